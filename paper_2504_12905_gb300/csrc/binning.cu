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
#include "common.cuh"

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
// Stable LSD radix sort, 8-bit digits, 32- or 64-bit keys and 32-bit values.
// Per pass: a per-block digit histogram (digit-major, so one exclusive scan
// gives every block's output base per digit), then a stable scatter that
// ranks equal digits in element order with warp match masks and per-warp
// counters.
// ---------------------------------------------------------------------------
constexpr int kRadixBlock = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixBlock * kRadixItems;
constexpr int kRadixWarps = kRadixBlock / kWarp;

template <typename K>
__global__ void __launch_bounds__(kRadixBlock) k_radix_hist(const K* keys, long long n, int shift, unsigned int* hist,
                                                           int nblocks) {
    __shared__ unsigned int s[256];
    s[threadIdx.x] = 0u;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRadixTile;
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const long long idx = base + r * kRadixBlock + threadIdx.x;
        if (idx < n) atomicAdd(&s[(unsigned)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nblocks + blockIdx.x] = s[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kRadixBlock) k_radix_scatter(const K* kin, const unsigned int* vin, K* kout,
                                                              unsigned int* vout, long long n, int shift,
                                                              const unsigned int* hist, int nblocks) {
    __shared__ unsigned int s_base[256];
    __shared__ unsigned int s_wc[kRadixWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = hist[(long long)tid * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) s_wc[w][tid] = 0u;
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixItems; ++r) {
        const long long idx = base + r * kRadixBlock + tid;
        const bool valid = idx < n;
        K key = 0;
        unsigned int val = 0u;
        if (valid) {
            key = kin[idx];
            val = vin[idx];
        }
        const unsigned d = valid ? (unsigned)(key >> shift) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt_mask);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned pre = s_base[d];
            for (int w = 0; w < warp; ++w) pre += s_wc[w][d];
            kout[pre + rank] = key;
            vout[pre + rank] = val;
        }
        __syncthreads();
        unsigned add = 0u;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            add += s_wc[w][tid];
            s_wc[w][tid] = 0u;
        }
        s_base[tid] += add;
        __syncthreads();
    }
}

size_t radix_tmp_bytes(long long n) {
    const long long nb = (n + kRadixTile - 1) / kRadixTile;
    const long long hist = 256ll * (nb > 0 ? nb : 1);
    return (size_t)hist * sizeof(unsigned int) + scan_tmp_elems<unsigned int>(hist) * sizeof(unsigned int);
}

template <typename K>
static void radix_sort_impl(K* keys, unsigned int* vals, K* keys_alt, unsigned int* vals_alt, long long n, int bits,
                            void* tmp, cudaStream_t st) {
    if (n <= 1) return;
    const int nb = (int)((n + kRadixTile - 1) / kRadixTile);
    unsigned int* hist = static_cast<unsigned int*>(tmp);
    unsigned int* stmp = hist + 256ll * nb;
    K *ki = keys, *ko = keys_alt;
    unsigned int *vi = vals, *vo = vals_alt;
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        LMRS_LAUNCH(k_radix_hist<K>, nb, kRadixBlock, 0, st, ki, n, shift, hist, nb);
        scan_rec<unsigned int>(hist, 256ll * nb, nullptr, stmp, st);
        LMRS_LAUNCH(k_radix_scatter<K>, nb, kRadixBlock, 0, st, ki, vi, ko, vo, n, shift, hist, nb);
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

}  // namespace lmrs
