// Tile binning with a hand-written stable LSD radix sort.
//
// Two levels, so the long (view, tile, Gaussian) list is sorted on the tile
// bits only:
//   1. the (view, Gaussian) pairs are sorted by (view, FP32 depth bits); they
//      are emitted in Gaussian-index order and every pass is stable, so equal
//      depths keep the lower index first;
//   2. each visible pair, in that order, emits one entry per overlapped tile;
//   3. the entries are stable-sorted by (view, tile).
// The result is ordered by (view, tile, depth, Gaussian index), the list
// order of the rendering equation (Sec. 3: Gaussians sorted by depth).
#include <algorithm>

#include "common.cuh"
#include "reduce.cuh"

namespace lmrs {

// ---------------------------------------------------------------------------
// Exclusive prefix sum (recursive, 2048 elements per block).
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s, T* total) {
    // s: kScanBlock entries of shared memory
    const int tid = threadIdx.x;
    s[tid] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        T add = tid >= off ? s[tid - off] : T(0);
        __syncthreads();
        s[tid] += add;
        __syncthreads();
    }
    const T incl = s[tid];
    *total = s[kScanBlock - 1];
    __syncthreads();
    return incl - v;
}

template <typename T>
__global__ void k_scan_tiles(T* data, long long n, T* block_sums) {
    __shared__ T s[kScanBlock];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    T loc[kScanItems];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = base + k < n ? data[base + k] : T(0);
        sum += loc[k];
    }
    T total;
    T pre = block_exclusive_scan<T>(sum, s, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) data[base + k] = pre;
        pre += loc[k];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T* data, long long n, const T* block_offsets) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    const T off = block_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) data[base + k] += off;
}

template <typename T>
static size_t scan_tmp_elems(long long n) {
    size_t tot = 0;
    while (true) {
        long long nb = (n + kScanTile - 1) / kScanTile;
        tot += (size_t)nb + 1;
        if (nb <= 1) break;
        n = nb;
    }
    return tot;
}

// In-place exclusive scan; the total is written to total_dev.
template <typename T>
static void scan_rec(T* data, long long n, T* total_dev, T* tmp, cudaStream_t st) {
    const long long nb = (n + kScanTile - 1) / kScanTile;
    T* sums = tmp;
    LMRS_LAUNCH(k_scan_tiles<T>, (unsigned)nb, kScanBlock, 0, st, data, n, sums);
    if (nb == 1) {
        if (total_dev) cudaMemcpyAsync(total_dev, sums, sizeof(T), cudaMemcpyDeviceToDevice, st);
        return;
    }
    scan_rec<T>(sums, nb, total_dev, tmp + nb + 1, st);
    LMRS_LAUNCH(k_scan_add<T>, (unsigned)nb, kScanBlock, 0, st, data, n, sums);
}

size_t scan_u64_tmp_bytes(long long n) { return scan_tmp_elems<unsigned long long>(n) * sizeof(unsigned long long); }

void scan_u64(unsigned long long* data, long long n, unsigned long long* total_dev, void* tmp, size_t,
              cudaStream_t st) {
    scan_rec<unsigned long long>(data, n, total_dev, static_cast<unsigned long long*>(tmp), st);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of 32- or 64-bit keys with 32-bit values.  The key
// bits are split into the fewest passes of at most 8 bits, balanced (14 bits:
// two passes of 7), so each pass has as few buckets as possible.  Per pass:
//   1. per-block digit counts over tiles of kRadixTile elements, stored
//      digit-major so that one exclusive scan gives every (digit, block) its
//      output base;
//   2. the scatter: each warp ranks the digits of its contiguous 512
//      elements in element order (ballot multisplit + warp-private running
//      counts), the block combines the warps' counts into local digit starts,
//      places its tile sorted by digit in shared memory, and writes the tile
//      out in that order, so the stores of one digit's run are contiguous.
// ---------------------------------------------------------------------------
constexpr int kRadixBlock = 256;
constexpr int kRadixWarps = kRadixBlock / kWarp;
constexpr int kRadixRounds = 16;                           // 32-element rounds per warp
constexpr int kRadixTile = kRadixBlock * kRadixRounds;    // 4096 elements per block
constexpr int kRadixMaxBuckets = 256;

template <typename K>
constexpr size_t radix_smem_bytes() {
    return (size_t)kRadixTile * (sizeof(K) + sizeof(unsigned int)) +
           sizeof(unsigned int) * (kRadixWarps * kRadixMaxBuckets + 2 * kRadixMaxBuckets);
}

// Lanes of the warp whose digit equals this lane's (warp multisplit by
// ballots): the AND over the digit's bits of that bit's ballot or its
// complement, restricted to the valid lanes.  nbits <= 8, warp-uniform.
__device__ __forceinline__ unsigned digit_peers(unsigned d, int nbits, bool valid) {
    unsigned m = __ballot_sync(kFull, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b < nbits) {
            const bool bit = (d >> b) & 1u;
            const unsigned bb = __ballot_sync(kFull, bit);
            m &= bit ? bb : ~bb;
        }
    }
    return m;
}

template <typename K>
__global__ void __launch_bounds__(kRadixBlock) k_radix_hist(const K* keys, long long n, int shift, unsigned mask,
                                                           unsigned int* hist, int nblocks) {
    __shared__ unsigned int s[kRadixMaxBuckets];
    s[threadIdx.x] = 0u;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRadixTile;
#pragma unroll 4
    for (int r = 0; r < kRadixRounds; ++r) {
        const long long idx = base + r * kRadixBlock + threadIdx.x;
        if (idx < n) atomicAdd(&s[(unsigned)(keys[idx] >> shift) & mask], 1u);
    }
    __syncthreads();
    if (threadIdx.x <= mask) hist[(long long)threadIdx.x * nblocks + blockIdx.x] = s[threadIdx.x];
}

// Exclusive scan of v[0..256) in place by one block of 256 threads; returns
// nothing, v holds the exclusive prefix afterwards.
__device__ __forceinline__ void block_exclusive_scan256(unsigned int* v) {
    __shared__ unsigned int s_warp[kRadixWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned x = v[tid];
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < kRadixWarps ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < kRadixWarps; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kRadixWarps) s_warp[lane] = w;
    }
    __syncthreads();
    v[tid] = inc - x + (warp > 0 ? s_warp[warp - 1] : 0u);
    __syncthreads();
}

template <typename K>
__global__ void __launch_bounds__(kRadixBlock) k_radix_scatter(const K* kin, const unsigned int* vin, K* kout,
                                                              unsigned int* vout, long long n, int shift,
                                                              unsigned mask, const unsigned int* hist, int nblocks) {
    extern __shared__ __align__(16) unsigned char radix_smem[];
    K* s_key = reinterpret_cast<K*>(radix_smem);
    unsigned int* s_val = reinterpret_cast<unsigned int*>(s_key + kRadixTile);
    unsigned int* s_wc = s_val + kRadixTile;                        // [warp][bucket]
    unsigned int* s_start = s_wc + kRadixWarps * kRadixMaxBuckets;  // local digit starts
    unsigned int* s_gbase = s_start + kRadixMaxBuckets;            // output base per digit
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kRadixWarps * kRadixMaxBuckets; i += kRadixBlock) s_wc[i] = 0u;
    s_gbase[tid] = tid <= (int)mask ? hist[(long long)tid * nblocks + blockIdx.x] : 0u;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int nbits = __popc(mask);
    unsigned int* wc = s_wc + warp * kRadixMaxBuckets;
    const long long wbase = (long long)blockIdx.x * kRadixTile + warp * (kRadixRounds * kWarp);
    K key[kRadixRounds];
    unsigned int val[kRadixRounds], rank[kRadixRounds];
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        const long long idx = wbase + r * kWarp + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : K(0);
        val[r] = valid ? vin[idx] : 0u;
        const unsigned d = valid ? (unsigned)(key[r] >> shift) & mask : 0u;
        const unsigned peers = digit_peers(d, nbits, valid);
        const unsigned before = valid ? wc[d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: warp prefixes (in place) and the block total
    {
        unsigned run = 0u;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            const unsigned c = s_wc[w * kRadixMaxBuckets + tid];
            s_wc[w * kRadixMaxBuckets + tid] = run;
            run += c;
        }
        s_start[tid] = run;
    }
    __syncthreads();
    block_exclusive_scan256(s_start);
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        const long long idx = wbase + r * kWarp + lane;
        if (idx < n) {
            const unsigned d = (unsigned)(key[r] >> shift) & mask;
            const unsigned pos = s_start[d] + wc[d] + rank[r];
            s_key[pos] = key[r];
            s_val[pos] = val[r];
        }
    }
    __syncthreads();
    const long long cnt = min((long long)kRadixTile, n - (long long)blockIdx.x * kRadixTile);
    for (int i = tid; i < cnt; i += kRadixBlock) {
        const K k = s_key[i];
        const unsigned d = (unsigned)(k >> shift) & mask;
        const long long o = (long long)s_gbase[d] + (i - (long long)s_start[d]);
        kout[o] = k;
        vout[o] = s_val[i];
    }
}

size_t radix_tmp_bytes(long long n) {
    const long long nb = (n + kRadixTile - 1) / kRadixTile;
    const long long hist = (long long)kRadixMaxBuckets * (nb > 0 ? nb : 1);
    return (size_t)hist * sizeof(unsigned int) + scan_tmp_elems<unsigned int>(hist) * sizeof(unsigned int);
}

template <typename K>
static void radix_sort_impl(K* keys, unsigned int* vals, K* keys_alt, unsigned int* vals_alt, long long n, int bits,
                            void* tmp, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return;
    static_assert(radix_smem_bytes<unsigned long long>() <= 227 * 1024, "scatter tile exceeds shared memory");
    // the opt-in above 48 KB is a per-function attribute (idempotent)
    cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)radix_smem_bytes<K>());
    const int nb = (int)((n + kRadixTile - 1) / kRadixTile);
    unsigned int* hist = static_cast<unsigned int*>(tmp);
    unsigned int* stmp = hist + (long long)kRadixMaxBuckets * nb;
    K *ki = keys, *ko = keys_alt;
    unsigned int *vi = vals, *vo = vals_alt;
    const int passes = (bits + 7) / 8;
    const int width = (bits + passes - 1) / passes;
    for (int p = 0, shift = 0; p < passes; ++p, shift += width) {
        const int w = std::min(width, bits - shift);
        const unsigned mask = (1u << w) - 1u;
        LMRS_LAUNCH(k_radix_hist<K>, nb, kRadixBlock, 0, st, ki, n, shift, mask, hist, nb);
        scan_rec<unsigned int>(hist, (long long)(mask + 1) * nb, nullptr, stmp, st);
        LMRS_LAUNCH(k_radix_scatter<K>, nb, kRadixBlock, radix_smem_bytes<K>(), st, ki, vi, ko, vo, n, shift, mask,
                    hist, nb);
        K* tk = ki; ki = ko; ko = tk;
        unsigned int* tv = vi; vi = vo; vo = tv;
    }
    if (ki != keys) {
        cudaMemcpyAsync(keys, ki, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, vi, (size_t)n * sizeof(unsigned int), cudaMemcpyDeviceToDevice, st);
    }
}

void radix_sort(unsigned long long* keys, unsigned int* vals, unsigned long long* keys_alt, unsigned int* vals_alt,
                long long n, int bits, void* tmp, size_t, cudaStream_t st) {
    radix_sort_impl<unsigned long long>(keys, vals, keys_alt, vals_alt, n, bits, tmp, st);
}

void radix_sort32(unsigned int* keys, unsigned int* vals, unsigned int* keys_alt, unsigned int* vals_alt, long long n,
                  int bits, void* tmp, size_t, cudaStream_t st) {
    radix_sort_impl<unsigned int>(keys, vals, keys_alt, vals_alt, n, bits, tmp, st);
}

// ---------------------------------------------------------------------------
// Level 2: tile counts of the depth-sorted pairs and entry emission.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long rect_area(int4 rc) {
    return rc.x > rc.y ? 0ull : (unsigned long long)(rc.y - rc.x + 1) * (unsigned long long)(rc.w - rc.z + 1);
}

__global__ void k_sorted_counts(Ctx c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)c.nv * c.G) return;
    const long long slot = (long long)(c.dkeys[k] >> 32);
    c.cnt[k] = rect_area(c.rect[slot * c.G + c.dvals[k]]);
}

// Entries (view-tile key, Gaussian) of the depth-sorted pairs.  Each warp
// takes 32 consecutive pairs and writes them one pair at a time with all
// lanes, so the stores are contiguous and large rectangles do not serialise
// on one thread.
__global__ void k_emit(Ctx c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned slot = 0u, g = 0u;
    int4 rc = make_int4(1, 0, 1, 0);
    unsigned long long o = 0ull;
    if (k < (long long)c.nv * c.G) {
        slot = (unsigned)(c.dkeys[k] >> 32);
        g = c.dvals[k];
        rc = c.rect[(long long)slot * c.G + g];
        o = c.cnt[k];
    }
    for (int j = 0; j < 32; ++j) {
        const int x0 = __shfl_sync(0xffffffffu, rc.x, j), x1 = __shfl_sync(0xffffffffu, rc.y, j);
        const int y0 = __shfl_sync(0xffffffffu, rc.z, j), y1 = __shfl_sync(0xffffffffu, rc.w, j);
        const unsigned long long oj = __shfl_sync(0xffffffffu, o, j);
        const unsigned gj = __shfl_sync(0xffffffffu, g, j);
        const unsigned base = __shfl_sync(0xffffffffu, slot, j) * (unsigned)c.T;
        if (x0 > x1) continue;
        const int w = x1 - x0 + 1, area = w * (y1 - y0 + 1);
        for (int e = lane; e < area; e += 32) {
            const int ty = y0 + e / w, tx = x0 + e - (e / w) * w;
            c.keys[oj + e] = base + (unsigned)(ty * c.tiles_x + tx);
            c.ids[oj + e] = gj;
        }
    }
}

void launch_sorted_counts(const Ctx& c, cudaStream_t st) {
    const long long n = (long long)c.nv * c.G;
    LMRS_LAUNCH(k_sorted_counts, (unsigned)((n + 255) / 256), 256, 0, st, c);
}

void launch_emit(const Ctx& c, cudaStream_t st) {
    const long long n = (long long)c.nv * c.G;
    LMRS_LAUNCH(k_emit, (unsigned)((n + 127) / 128), 128, 0, st, c);
}

// ---------------------------------------------------------------------------
// Per-tile [begin, end) in the sorted list.
// ---------------------------------------------------------------------------
__global__ void k_ranges(Ctx c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= c.npairs) return;
    const unsigned vt = c.keys[k];
    if (k == 0 || c.keys[k - 1] != vt) c.ranges[vt].x = (int)k;
    if (k == c.npairs - 1 || c.keys[k + 1] != vt) c.ranges[vt].y = (int)(k + 1);
}

void launch_ranges(const Ctx& c, cudaStream_t st) {
    if (c.npairs <= 0) return;
    LMRS_LAUNCH(k_ranges, (unsigned)((c.npairs + 255) / 256), 256, 0, st, c);
}

// ---------------------------------------------------------------------------
// Direct stable binning (replaces the entry emission + tile sort when a
// view has at most kBinMaxTiles tiles).  In the depth-sorted pair array slot
// s occupies [s G, (s+1) G): its visible pairs by depth, then its culled ones
// (empty rectangles).  A block takes a chunk of kBinChunk consecutive pairs
// of one slot; warp w owns the w-th run of kBinRun pairs of the chunk and
// handles them in order, the tiles of one pair spread over the lanes (a pair
// touches each tile once, so the lanes never collide).
//   count : entries per (slot, tile, chunk), tile-major in mat;
//   scan  : exclusive prefix of mat = the output base of every (slot, tile,
//           chunk), the start of every tile list and the total;
//   place : per-warp counts per tile again, their prefix over the block's
//           warps, then each warp walks its run once more and writes each
//           entry's Gaussian index at base + warp prefix + running count.
// Per tile the entries come out by chunk, then warp, then pair order: the
// order of a stable sort on (slot, tile) of the depth-ordered entries.
// ---------------------------------------------------------------------------
constexpr int kBinWarps = 8;
constexpr int kBinRun = 256;
constexpr int kBinChunk = kBinWarps * kBinRun;
constexpr int kBinBlock = kBinWarps * kWarp;

int bin_chunks(const Ctx& c) { return (c.G + kBinChunk - 1) / kBinChunk; }

size_t bin_place_smem(int T) { return (size_t)T * (sizeof(unsigned) + kBinWarps * sizeof(unsigned short)); }

// Calls f(tile, gaussian) for every tile of every pair of [b, e) of slot's
// depth-ordered pairs, pairs in order, one __syncwarp between pairs.
template <class F>
__device__ __forceinline__ void for_run_tiles(const Ctx& c, int slot, long long b, long long e, F&& f) {
    const int lane = threadIdx.x & 31;
    for (long long base = b; base < e; base += 32) {
        const long long k = base + lane;
        int4 rc = make_int4(1, 0, 1, 0);
        unsigned g = 0u;
        if (k < e) {
            g = c.dvals[k];
            rc = c.rect[(long long)slot * c.G + g];
        }
        const int n = (int)min(32ll, e - base);
        for (int j = 0; j < n; ++j) {
            const int x0 = __shfl_sync(kFull, rc.x, j), x1 = __shfl_sync(kFull, rc.y, j);
            const int y0 = __shfl_sync(kFull, rc.z, j), y1 = __shfl_sync(kFull, rc.w, j);
            const unsigned gj = __shfl_sync(kFull, g, j);
            if (x0 <= x1) {
                const int w = x1 - x0 + 1, area = w * (y1 - y0 + 1);
                // row of q = floor((q + 0.5) / w): exact in FP32 for q < 2^22
                const float inv_w = 1.f / (float)w;
                for (int q = lane; q < area; q += 32) {
                    const int qy = (int)(((float)q + 0.5f) * inv_w);
                    f((y0 + qy) * c.tiles_x + x0 + (q - qy * w), gj);
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ void bin_run(const Ctx& c, long long& b, long long& e) {
    const long long s0 = (long long)blockIdx.y * c.G;
    b = s0 + (long long)blockIdx.x * kBinChunk + (long long)(threadIdx.x >> 5) * kBinRun;
    e = min(b + kBinRun, s0 + c.G);
}

__global__ void __launch_bounds__(kBinBlock) k_bin_count(Ctx c, int nchunk, unsigned* mat,
                                                         unsigned long long* total) {
    extern __shared__ unsigned bin_smem[];
    unsigned* s_cnt = bin_smem;  // [T]
    for (int t = threadIdx.x; t < c.T; t += kBinBlock) s_cnt[t] = 0u;
    __syncthreads();
    long long b, e;
    bin_run(c, b, e);
    unsigned mine = 0u;
    if (b < e)
        for_run_tiles(c, (int)blockIdx.y, b, e, [&](int t, unsigned) {
            atomicAdd(&s_cnt[t], 1u);
            ++mine;
        });
    __syncthreads();
    const long long row = (long long)blockIdx.y * c.T;
    for (int t = threadIdx.x; t < c.T; t += kBinBlock) mat[(row + t) * nchunk + blockIdx.x] = s_cnt[t];
    // exact 64-bit total (the scan of mat is 32-bit)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) mine += __shfl_xor_sync(kFull, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, (unsigned long long)mine);
}

__global__ void __launch_bounds__(kBinBlock) k_bin_place(Ctx c, int nchunk, const unsigned* mat) {
    extern __shared__ unsigned bin_smem[];
    unsigned* s_base = bin_smem;                                                  // [T]
    unsigned short* s_w = reinterpret_cast<unsigned short*>(bin_smem + c.T);     // [kBinWarps][T]
    for (int t = threadIdx.x; t < kBinWarps * c.T; t += kBinBlock) s_w[t] = 0;
    __syncthreads();
    long long b, e;
    bin_run(c, b, e);
    unsigned short* mine = s_w + (size_t)(threadIdx.x >> 5) * c.T;
    if (b < e) for_run_tiles(c, (int)blockIdx.y, b, e, [&](int t, unsigned) { ++mine[t]; });
    __syncthreads();
    const long long row = (long long)blockIdx.y * c.T;
    for (int t = threadIdx.x; t < c.T; t += kBinBlock) {
        unsigned run = 0u;
#pragma unroll
        for (int w = 0; w < kBinWarps; ++w) {
            const unsigned v = s_w[w * c.T + t];
            s_w[w * c.T + t] = (unsigned short)run;
            run += v;
        }
        s_base[t] = mat[(row + t) * nchunk + blockIdx.x];
    }
    __syncthreads();
    if (b < e)
        for_run_tiles(c, (int)blockIdx.y, b, e, [&](int t, unsigned g) {
            const unsigned pos = s_base[t] + mine[t];
            ++mine[t];
            c.ids[pos] = g;
        });
}

__global__ void k_bin_ranges(Ctx c, int nchunk, const unsigned* mat, const unsigned* total32) {
    const long long vt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nvt = (long long)c.nv * c.T;
    if (vt >= nvt) return;
    const unsigned b = mat[vt * nchunk];
    const unsigned e = vt + 1 < nvt ? mat[(vt + 1) * nchunk] : *total32;
    c.ranges[vt] = make_int2((int)b, (int)e);
}

size_t bin_mat_elems(const Ctx& c) { return (size_t)c.nv * c.T * bin_chunks(c); }

size_t bin_scan_tmp_bytes(long long n) { return scan_tmp_elems<unsigned int>(n) * sizeof(unsigned int); }

void launch_bin_count(const Ctx& c, unsigned* mat, unsigned long long* total, cudaStream_t st) {
    const dim3 grid(bin_chunks(c), c.nv);
    LMRS_LAUNCH(k_bin_count, grid, kBinBlock, sizeof(unsigned) * c.T, st, c, bin_chunks(c), mat, total);
}

void scan_bin_mat(unsigned* mat, long long n, unsigned* total32, void* tmp, cudaStream_t st) {
    scan_rec<unsigned int>(mat, n, total32, static_cast<unsigned int*>(tmp), st);
}

void launch_bin_place(const Ctx& c, const unsigned* mat, const unsigned* total32, cudaStream_t st) {
    const size_t smem = bin_place_smem(c.T);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_bin_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid(bin_chunks(c), c.nv);
    LMRS_LAUNCH(k_bin_place, grid, kBinBlock, smem, st, c, bin_chunks(c), mat);
    const long long nvt = (long long)c.nv * c.T;
    LMRS_LAUNCH(k_bin_ranges, (unsigned)((nvt + 255) / 256), 256, 0, st, c, bin_chunks(c), mat, total32);
}

}  // namespace lmrs
