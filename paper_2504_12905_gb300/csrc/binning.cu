// Tile binning with a hand-written stable LSD radix sort.
//
// The (view, Gaussian) pairs are first sorted by (view, FP32 depth bits);
// they are emitted in Gaussian-index order and every pass is stable, so equal
// depths keep the lower index first.  The tile lists are then built from the
// depth-ordered pairs, by one of two builders:
//   * the two-level placement (the main path, while a view's rows and columns
//     of tiles fit the shared-memory counters): each pair goes into the lists
//     of the tile rows its ellipse reaches, then each row entry into the
//     tiles of its span (see the section "Two-level stable binning" below);
//   * the fallback for wider or taller tile grids: each visible pair emits one
//     entry per tile it covers, and the entries are stable-sorted by (view,
//     tile).
// Either way the result is ordered by (view, tile, depth, Gaussian index),
// the list order of the rendering equation (Sec. 3: Gaussians sorted by
// depth).
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
// Tiles the list of pair i covers: the row spans of its rectangle.
__device__ __forceinline__ unsigned long long list_tiles(const Ctx& c, long long i) {
    const int4 rc = c.rect[i];
    if (rc.x > rc.y) return 0ull;
    const float4 e0 = c.ell[2 * i], e1 = c.ell[2 * i + 1];
    unsigned long long n = 0ull;
    for (int ty = rc.z; ty <= rc.w; ++ty) {
        int x0, x1;
        if (row_span(e0, e1, ty, rc, c.tile_w, c.tile_h, c.W, c.H, x0, x1)) n += (unsigned long long)(x1 - x0 + 1);
    }
    return n;
}

__global__ void k_sorted_counts(Ctx c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)c.nv * c.G) return;
    const long long slot = (long long)(c.dkeys[k] >> 32);
    c.cnt[k] = list_tiles(c, slot * c.G + c.dvals[k]);
}

// Entries (view-tile key, Gaussian) of the depth-sorted pairs.  Each warp
// takes 32 consecutive pairs and writes them one pair at a time with all
// lanes, row by row of its rectangle, so the stores are contiguous and large
// rectangles do not serialise on one thread.
__global__ void k_emit(Ctx c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned slot = 0u, g = 0u;
    unsigned long long o = 0ull;
    if (k < (long long)c.nv * c.G) {
        slot = (unsigned)(c.dkeys[k] >> 32);
        g = c.dvals[k];
        o = c.cnt[k];
    }
    for (int j = 0; j < 32; ++j) {
        if (k - lane + j >= (long long)c.nv * c.G) break;  // warp-uniform
        const unsigned gj = __shfl_sync(0xffffffffu, g, j);
        const unsigned sj = __shfl_sync(0xffffffffu, slot, j);
        unsigned long long oj = __shfl_sync(0xffffffffu, o, j);
        const long long i = (long long)sj * c.G + gj;
        const int4 rc = c.rect[i];
        if (rc.x > rc.y) continue;
        const float4 e0 = c.ell[2 * i], e1 = c.ell[2 * i + 1];
        const unsigned base = sj * (unsigned)c.T;
        for (int ty = rc.z; ty <= rc.w; ++ty) {
            int x0, x1;
            if (!row_span(e0, e1, ty, rc, c.tile_w, c.tile_h, c.W, c.H, x0, x1)) continue;
            for (int tx = x0 + lane; tx <= x1; tx += 32) {
                c.keys[oj + (tx - x0)] = base + (unsigned)(ty * c.tiles_x + tx);
                c.ids[oj + (tx - x0)] = gj;
            }
            oj += (unsigned long long)(x1 - x0 + 1);
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
// Two-level stable binning of the depth-sorted pairs into the tile lists
// (used while a view's rows and columns of tiles fit the shared-memory
// counters; the entry emission + tile sort above covers the rest).  In the
// depth-sorted pair array slot s occupies [s G, (s+1) G): its visible pairs
// by depth, then its culled ones (empty rectangles).
//   rows : each visible pair, in order, is placed into the list of every tile
//          row of its rectangle whose band meets its ellipse (band_meets),
//          with that row's tile columns (row_span, possibly none): counts
//          per (slot, row, chunk of kBinChunk pairs), an exclusive scan, then
//          the placement;
//   tiles: one block per (slot, row, segment of its row list) counts that
//          row's list per tile, an exclusive scan gives the tile lists'
//          starts, then one block per (slot, row, group of kColGroup tile
//          columns, segment) walks the segment in order and places each pair
//          whose span meets the group into the group's tiles it spans.
// A placement ranks a lane's pair among the warp's 32 pairs covering the same
// bin with a ballot, warps are ranked by their order in the chunk and chunks
// by the scan, so every list keeps the order it is read in: the tile lists
// equal a stable sort on (slot, tile) of the depth-ordered entries.  The
// lists a warp writes at a time are the rows of one view or the tiles of one
// row, so its stores stay within a few dozen runs.
// ---------------------------------------------------------------------------
constexpr int kBinWarps = 8;
constexpr int kBinRun = 256;                  // pairs per warp per chunk
constexpr int kBinChunk = kBinWarps * kBinRun;
constexpr int kBinBlock = kBinWarps * kWarp;

int bin_chunks(const Ctx& c) { return (c.G + kBinChunk - 1) / kBinChunk; }

__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// One round of a warp: lane l holds the l-th of 32 consecutive items, covering
// the bins [lo, hi] (lo > hi: none).  For every bin of the union, m = the
// lanes covering it; count(bin, m) runs on every lane (warp-uniform m), and
// place(bin, rank) on each covering lane, rank = its position among them.
template <class Count, class Place>
__device__ __forceinline__ void rank_round(int lo, int hi, Count&& count, Place&& place) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int ulo = warp_min_i(lo <= hi ? lo : 0x7fffffff);
    const int uhi = warp_max_i(lo <= hi ? hi : -1);
    for (int bin = ulo; bin <= uhi; ++bin) {
        const bool in = lo <= bin && bin <= hi;
        const unsigned m = __ballot_sync(kFull, in);
        if (m == 0u) continue;
        if (in) place(bin, __popc(m & lt));
        __syncwarp();
        count(bin, m);
        __syncwarp();
    }
}

// Rectangle and row-span ellipse of the depth-ordered pair k of slot s
// (empty when culled or past e).
__device__ __forceinline__ void pair_rect(const Ctx& c, long long s0, long long k, long long e, unsigned& g,
                                          int4& rc, float4& e0, float4& e1) {
    g = 0u;
    rc = make_int4(1, 0, 1, 0);
    e0 = e1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < e) {
        g = c.dvals[k];
        rc = c.rect[s0 + g];
        if (rc.x > rc.y) {
            rc = make_int4(1, 0, 1, 0);
        } else {
            e0 = c.ell[2 * (s0 + g)];
            e1 = c.ell[2 * (s0 + g) + 1];
        }
    }
}

// The rows of rc whose band meets the pair's ellipse: contiguous, since
// band_meets is monotone from both ends; lo > hi when there are none.
__device__ __forceinline__ void band_rows(const Ctx& c, int4 rc, float4 e0, float4 e1, int& lo, int& hi) {
    lo = rc.z;
    hi = rc.w;
    while (lo <= hi && !band_meets(e0, e1, lo, c.tile_h, c.H)) ++lo;
    while (hi >= lo && !band_meets(e0, e1, hi, c.tile_h, c.H)) --hi;
}

// Row counts per (slot, row, chunk, warp of the chunk): mat[((slot * tiles_y
// + row) * nchunk + chunk) * kBinWarps + warp], so that the scan over mat
// gives every warp of the placement its start in each row list.
__global__ void __launch_bounds__(kBinBlock) k_row_count(Ctx c, int nchunk, unsigned* mat) {
    extern __shared__ unsigned bin_smem[];
    const int ny = c.tiles_y;
    unsigned* s_cnt = bin_smem;  // [kBinWarps][tiles_y]
    for (int i = threadIdx.x; i < kBinWarps * ny; i += kBinBlock) s_cnt[i] = 0u;
    __syncthreads();
    unsigned* mine = s_cnt + (threadIdx.x >> 5) * ny;
    const int slot = blockIdx.y;
    const long long s0 = (long long)slot * c.G;
    const long long b = s0 + (long long)blockIdx.x * kBinChunk + (long long)(threadIdx.x >> 5) * kBinRun;
    const long long e = min(b + kBinRun, s0 + c.G);
    for (long long k = b + (threadIdx.x & 31); k < e; k += 32) {
        const long long i = s0 + c.dvals[k];
        const int4 rc = c.rect[i];
        if (rc.x > rc.y) continue;
        int lo, hi;
        band_rows(c, rc, c.ell[2 * i], c.ell[2 * i + 1], lo, hi);
        for (int r = lo; r <= hi; ++r) atomicAdd(&mine[r], 1u);
    }
    __syncthreads();
    const long long row0 = (long long)slot * ny;
    for (int i = threadIdx.x; i < kBinWarps * ny; i += kBinBlock) {
        const int w = i / ny, r = i - w * ny;
        mat[((row0 + r) * nchunk + blockIdx.x) * kBinWarps + w] = s_cnt[i];
    }
}

// A row-list entry: the Gaussian index and its tile columns x0..x1.
__device__ __forceinline__ unsigned long long row_entry(unsigned g, int x0, int x1) {
    return (unsigned long long)g | ((unsigned long long)(unsigned)x0 << 32) | ((unsigned long long)(unsigned)x1 << 48);
}
__device__ __forceinline__ void row_entry_unpack(unsigned long long v, unsigned& g, int& x0, int& x1) {
    g = (unsigned)v;
    x0 = (int)((v >> 32) & 0xFFFFu);
    x1 = (int)(v >> 48);
}

// Placement in windows of kRowWin rows: the ballots of a window fix every
// (pair, row) entry's slot (the warp's start in the row from the scanned
// counts, plus the entries it placed there before, plus the lane's rank),
// then each lane computes the tile columns of its own rows once (row_span)
// and writes their entries.
constexpr int kRowWin = 32;

__global__ void __launch_bounds__(kBinBlock) k_row_place(Ctx c, int nchunk, const unsigned* mat,
                                                         unsigned long long* rl) {
    extern __shared__ unsigned bin_smem[];
    const int ny = c.tiles_y;
    unsigned* s_pos = bin_smem;                   // [kBinWarps][ny]: each warp's next slot per row
    unsigned* s_dst = bin_smem + kBinWarps * ny;  // [kBinWarps][kRowWin][32]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int slot = blockIdx.y;
    const long long row0 = (long long)slot * ny;
    for (int i = threadIdx.x; i < kBinWarps * ny; i += kBinBlock) {
        const int w = i / ny, r = i - w * ny;
        s_pos[i] = mat[((row0 + r) * nchunk + blockIdx.x) * kBinWarps + w];
    }
    __syncthreads();
    const long long s0 = (long long)slot * c.G;
    const long long b = s0 + (long long)blockIdx.x * kBinChunk + (long long)wid * kBinRun;
    const long long e = min(b + kBinRun, s0 + c.G);
    unsigned* mine = s_pos + wid * ny;
    const auto count = [&](int r, unsigned m) { if (lane == 0) mine[r] += (unsigned)__popc(m); };
    unsigned* dst = s_dst + wid * kRowWin * 32;
    for (long long base = b; base < e; base += 32) {
        unsigned g;
        int4 rc;
        float4 e0, e1;
        pair_rect(c, s0, base + lane, e, g, rc, e0, e1);
        int lo, hi;
        band_rows(c, rc, e0, e1, lo, hi);
        const int ulo = warp_min_i(lo <= hi ? lo : 0x7fffffff);
        const int uhi = warp_max_i(lo <= hi ? hi : -1);
        for (int w0 = ulo; w0 <= uhi; w0 += kRowWin) {
            const int wl = max(lo, w0), wh = min(hi, w0 + kRowWin - 1);
            rank_round(wl, wh, count, [&](int r, int rank) { dst[(r - w0) * 32 + lane] = mine[r] + rank; });
            __syncwarp();
            for (int r = wl; r <= wh; ++r) {
                int x0, x1;  // no tile in this row: an empty entry the tile stage skips
                if (!row_span(e0, e1, r, rc, c.tile_w, c.tile_h, c.W, c.H, x0, x1)) x0 = 1, x1 = 0;
                rl[dst[(r - w0) * 32 + lane]] = row_entry(g, x0, x1);
            }
            __syncwarp();
        }
    }
}

// [begin, end) of the row list of (slot, row) index sr in rl.
__device__ __forceinline__ void row_range(const Ctx& c, int nchunk, const unsigned* mat, const unsigned* total,
                                          int sr, unsigned& b, unsigned& e) {
    b = mat[(long long)sr * nchunk * kBinWarps];
    e = sr + 1 < c.nv * c.tiles_y ? mat[(long long)(sr + 1) * nchunk * kBinWarps] : *total;
}

// A row list is placed in kRowSegs segments of its entries (in order), so
// that a dense row's work spreads over several blocks; every (tile, segment)
// has its own count and start, and a tile's list is its segments' runs one
// after the other, in row-list order.
constexpr int kRowSegs = 8;

__device__ __forceinline__ void seg_range(unsigned b, unsigned e, int seg, unsigned& sb, unsigned& se) {
    const unsigned long long n = e - b;
    sb = b + (unsigned)(n * (unsigned long long)seg / kRowSegs);
    se = b + (unsigned)(n * (unsigned long long)(seg + 1) / kRowSegs);
}

// Tile counts of one (slot, row, segment) per block: a difference array over
// the row's columns in shared memory (+1 at x0, -1 at x1 + 1 per entry), then
// its prefix, written as cnt[(slot * T + row * tiles_x + x) * kRowSegs + seg]
// (the scan over that order gives every segment's start in its tile's list).
__global__ void __launch_bounds__(kBinBlock) k_tile_count(Ctx c, int nchunk, const unsigned* mat,
                                                          const unsigned* rtotal, const unsigned long long* rl,
                                                          unsigned* cnt) {
    extern __shared__ unsigned bin_smem[];
    const int nx = c.tiles_x;
    int* s_d = reinterpret_cast<int*>(bin_smem);  // [nx + 1]
    for (int x = threadIdx.x; x <= nx; x += kBinBlock) s_d[x] = 0;
    __syncthreads();
    const int sr = blockIdx.x, slot = sr / c.tiles_y, row = sr - slot * c.tiles_y, seg = blockIdx.y;
    unsigned rb, re, b, e;
    row_range(c, nchunk, mat, rtotal, sr, rb, re);
    seg_range(rb, re, seg, b, e);
    for (unsigned k = b + threadIdx.x; k < e; k += kBinBlock) {
        unsigned g;
        int x0, x1;
        row_entry_unpack(rl[k], g, x0, x1);
        if (x0 > x1) continue;
        atomicAdd(&s_d[x0], 1);
        atomicAdd(&s_d[x1 + 1], -1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // prefix over the columns, 32 at a time
        const int lane = threadIdx.x;
        int carry = 0;
        unsigned* o = cnt + ((long long)slot * c.T + (long long)row * nx) * kRowSegs;
        for (int x0 = 0; x0 < nx; x0 += 32) {
            const int x = x0 + lane;
            int v = x < nx ? s_d[x] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(kFull, v, off);
                if (lane >= off) v += y;
            }
            if (x < nx) o[(long long)x * kRowSegs + seg] = (unsigned)(carry + v);
            carry += __shfl_sync(kFull, v, 31);
        }
    }
}

// One block per (slot, row, group of kColGroup columns, segment); warp w owns
// the group's columns x = x0g + w + kColWarps q (q < kColsPerWarp).  The
// block walks the segment of the row list kPlaceRound entries at a time:
// the warps load consecutive runs of them and keep, in order, the entries
// whose span meets the group (a ballot and a block-wide prefix of the
// warps' counts place them in shared memory); then every warp walks the
// kept entries 32 at a time, and per owned column one ballot of the entries
// covering it, each covering lane writing at the (column, segment)'s
// running offset + its rank.  Every column's list is appended in order.
// Splitting a row over column groups and segments spreads its work over
// several SMs; the keep step spares the column ballots the entries of the
// row that lie in other groups.
constexpr int kColWarps = 8;
constexpr int kColsPerWarp = 2;
constexpr int kColGroup = kColWarps * kColsPerWarp;
constexpr int kColRounds = 4;  // 32-entry loads per warp per round
constexpr int kColBlock = kColWarps * kWarp;
constexpr int kPlaceRound = kColBlock * kColRounds;  // entries the block walks per round

__global__ void __launch_bounds__(kColBlock) k_tile_place(Ctx c, int nchunk, const unsigned* mat,
                                                          const unsigned* rtotal, const unsigned long long* rl,
                                                          const unsigned* start) {
    __shared__ unsigned long long s_keep[kPlaceRound];
    __shared__ int s_wcnt[kColWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nx = c.tiles_x;
    const int sr = blockIdx.x, slot = sr / c.tiles_y, row = sr - slot * c.tiles_y, seg = blockIdx.z;
    const int x0g = blockIdx.y * kColGroup;
    const int x1g = min(x0g + kColGroup, nx) - 1;  // the group's last column
    const long long t0 = (long long)slot * c.T + (long long)row * nx;
    unsigned rb, re, b, e;
    row_range(c, nchunk, mat, rtotal, sr, rb, re);
    seg_range(rb, re, seg, b, e);
    // its columns inside the row (none for some warps of the last group):
    // the ballots of the others are skipped
    const int nq = x0g + wid < nx ? min(kColsPerWarp, (nx - 1 - x0g - wid) / kColWarps + 1) : 0;
    unsigned off[kColsPerWarp];
    int col[kColsPerWarp];
#pragma unroll
    for (int q = 0; q < kColsPerWarp; ++q) {
        col[q] = x0g + wid + kColWarps * q;
        off[q] = q < nq ? start[(t0 + col[q]) * kRowSegs + seg] : 0u;
    }
    for (unsigned base = b; base < e; base += kPlaceRound) {
        // keep, in order, the round's entries whose span meets the group
        unsigned long long v[kColRounds];
        unsigned m[kColRounds];
        int cnt = 0;
#pragma unroll
        for (int r = 0; r < kColRounds; ++r) {
            const unsigned k = base + (unsigned)(wid * kColRounds + r) * 32u + lane;
            v[r] = k < e ? rl[k] : row_entry(0u, 1, 0);
        }
#pragma unroll
        for (int r = 0; r < kColRounds; ++r) {
            unsigned g;
            int x0, x1;
            row_entry_unpack(v[r], g, x0, x1);
            m[r] = __ballot_sync(kFull, x0 <= x1 && x0 <= x1g && x1 >= x0g);
            cnt += __popc(m[r]);
        }
        if (lane == 0) s_wcnt[wid] = cnt;
        __syncthreads();
        int run = 0, n = 0;
#pragma unroll
        for (int w = 0; w < kColWarps; ++w) {
            const int t = s_wcnt[w];
            run += w < wid ? t : 0;
            n += t;
        }
#pragma unroll
        for (int r = 0; r < kColRounds; ++r) {
            if ((m[r] >> lane) & 1u) s_keep[run + __popc(m[r] & lt)] = v[r];
            run += __popc(m[r]);
        }
        __syncthreads();
        // the kept entries, 32 at a time: per owned column one ballot
        for (int j = 0; j < n; j += 32) {
            const int i = j + lane;
            unsigned g;
            int x0, x1;
            row_entry_unpack(i < n ? s_keep[i] : row_entry(0u, 1, 0), g, x0, x1);
#pragma unroll
            for (int q = 0; q < kColsPerWarp; ++q) {
                if (q >= nq) break;  // warp-uniform
                const bool in = x0 <= col[q] && col[q] <= x1;
                const unsigned mq = __ballot_sync(kFull, in);
                if (in) c.ids[off[q] + __popc(mq & lt)] = g;
                off[q] += __popc(mq);
            }
        }
        __syncthreads();  // s_keep and s_wcnt are rewritten by the next round
    }
}

__global__ void k_tile_ranges(Ctx c, const unsigned* start, const unsigned* total32) {
    const long long vt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nvt = (long long)c.nv * c.T;
    if (vt >= nvt) return;
    const unsigned b = start[vt * kRowSegs];
    const unsigned e = vt + 1 < nvt ? start[(vt + 1) * kRowSegs] : *total32;
    c.ranges[vt] = make_int2((int)b, (int)e);
    if (vt == 0) c.sc->n_list = *total32;
}

static size_t row_place_smem(const Ctx& c) {
    return ((size_t)kBinWarps * c.tiles_y + (size_t)kBinWarps * kRowWin * 32) * sizeof(unsigned);
}

bool bin_rows_fit(const Ctx& c) {
    return row_place_smem(c) <= 200 * 1024 && (size_t)(c.tiles_x + 1) * sizeof(int) <= 200 * 1024 &&
           c.tiles_x < 65536;
}

size_t bin_row_mat_elems(const Ctx& c) { return (size_t)c.nv * c.tiles_y * bin_chunks(c) * kBinWarps; }
size_t bin_tile_count_elems(const Ctx& c) { return (size_t)c.nv * c.T * kRowSegs; }
size_t bin_scan_tmp_bytes(long long n) { return scan_tmp_elems<unsigned int>(n) * sizeof(unsigned int); }

void bin_rows(const Ctx& c, unsigned* mat, unsigned long long* rl, unsigned* rtotal, void* tmp, cudaStream_t st) {
    const dim3 grid(bin_chunks(c), c.nv);
    const size_t csmem = sizeof(unsigned) * kBinWarps * c.tiles_y;
    if (csmem > 48 * 1024) cudaFuncSetAttribute(k_row_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
    LMRS_LAUNCH(k_row_count, grid, kBinBlock, csmem, st, c, bin_chunks(c), mat);
    scan_rec<unsigned int>(mat, (long long)bin_row_mat_elems(c), rtotal, static_cast<unsigned*>(tmp), st);
    const size_t smem = row_place_smem(c);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_row_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LMRS_LAUNCH(k_row_place, grid, kBinBlock, smem, st, c, bin_chunks(c), mat, rl);
}

void bin_tiles(const Ctx& c, const unsigned* mat, const unsigned* rtotal, const unsigned long long* rl, unsigned* cnt,
               unsigned* etotal, void* tmp, cudaStream_t st) {
    const unsigned rows = (unsigned)(c.nv * c.tiles_y);
    const size_t smem = sizeof(int) * (c.tiles_x + 1);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LMRS_LAUNCH(k_tile_count, dim3(rows, kRowSegs), kBinBlock, smem, st, c, bin_chunks(c), mat, rtotal, rl, cnt);
    const long long nvt = (long long)c.nv * c.T;
    scan_rec<unsigned int>(cnt, nvt * kRowSegs, etotal, static_cast<unsigned*>(tmp), st);
    const dim3 pgrid(rows, (unsigned)((c.tiles_x + kColGroup - 1) / kColGroup), kRowSegs);
    LMRS_LAUNCH(k_tile_place, pgrid, kColBlock, 0, st, c, bin_chunks(c), mat, rtotal, rl, cnt);
    LMRS_LAUNCH(k_tile_ranges, (unsigned)((nvt + 255) / 256), 256, 0, st, c, cnt, etotal);
}

}  // namespace lmrs
