// Warp and block reductions shared by the kernels of liblmrs.
#pragma once

#include "common.cuh"

namespace lmrs {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

// Compensated FP32 dot product, Dot2 of Ogita, Rump and Oishi ("Accurate Sum
// and Dot Product", SIAM J. Sci. Comput. 26(6), 2005): TwoProduct through an
// FMA and Knuth's TwoSum, so a thread's partial sum is as accurate as if it
// were computed in twice the working precision.  FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU; per-thread partials are
// formed this way and only the cross-thread combination is FP64.  Every
// operation of the error-free transformations is rounded on its own.
struct Dot2 {
    float p = 0.f, s = 0.f;
    __device__ __forceinline__ void add(float x, float y) {
        const float h = __fmul_rn(x, y);
        const float r = __fmaf_rn(x, y, -h);  // x * y = h + r exactly
        const float t = __fadd_rn(p, h);
        const float z = __fsub_rn(t, p);
        const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));  // p + h = t + q exactly
        p = t;
        s += q + r;
    }
    __device__ __forceinline__ double value() const { return (double)p + (double)s; }
};

// Sum over the block, returned to every thread.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_w[BLOCK / kWarp];
    __shared__ double s_tot;
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < BLOCK / kWarp ? s_w[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) s_tot = t;
    }
    __syncthreads();
    double r = s_tot;
    __syncthreads();
    return r;
}

// Grid-wide FP64 sum in a fixed order: every block stores its partial, the
// last block to arrive adds the partials (in block order) and returns true
// with the total in *total (thread 0 writes it).  gridDim.x <= kMaxPartials.
template <int BLOCK>
__device__ __forceinline__ bool grid_sum_last(double v, double* partials, unsigned int* counter, double* total) {
    __shared__ bool s_last;
    double b = block_sum<BLOCK>(v);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += BLOCK) acc += ((volatile double*)partials)[i];
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) {
        *total = acc;
        *counter = 0u;
    }
    return true;
}

// Reduce-scatter of N values over the 32 lanes of a warp (recursive
// halving): on return v[0] of lane l holds the warp total of element
//   N == 32: l;    N == 16: (l >> 1) (lanes l and l^1 agree).
// N/2 + N/4 + ... shuffles instead of 5 N for one butterfly per value.
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[N]) {
    static_assert(N == 16 || N == 32, "16 or 32 values");
    const int lane = threadIdx.x & 31;
    int n = N;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        if (n > 1) {
            const bool upper = (lane & m) != 0;
#pragma unroll
            for (int i = 0; i < N / 2; ++i) {
                if (i < n / 2) {
                    float send = upper ? v[i] : v[i + n / 2];
                    float keep = upper ? v[i + n / 2] : v[i];
                    v[i] = keep + __shfl_xor_sync(kFull, send, m);
                }
            }
            n >>= 1;
        } else {
            v[0] += __shfl_xor_sync(kFull, v[0], m);
        }
    }
}

// Warp sum of 9 values per lane, scattered over the lanes: the 9 values
// (padded to 10) are halved over lane bits 16, 8, 4, 2 (5, 3, 2, 1
// shuffles), then the two partial sums of each pair of lanes are added
// across bit 1 -- 12 shuffles instead of 16 for the padded 16-value form.
// Returns the index of the value whose sum this lane holds, -1 when it
// holds padding (the even lanes 0, 2, 4, 8, 10, 16, 18, 20, 24 hold values
// 0..8; odd lanes hold a copy of their even neighbour's).  v[9] must be 0.
__device__ __forceinline__ int warp_reduce_scatter9(float (&v)[10]) {
    const int lane = threadIdx.x & 31;
    int base = 0, end = 9, n = 10;
#pragma unroll
    for (int m = 16; m >= 2; m >>= 1) {
        const int half = (n + 1) / 2;
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (i < half) {
                const float lo = v[i];
                const float hi = half + i < n ? v[half + i] : 0.f;
                v[i] = (up ? hi : lo) + __shfl_xor_sync(kFull, up ? lo : hi, m);
            }
        }
        if (up) base += half;
        else end = min(end, base + half);
        n = half;
    }
    v[0] += __shfl_xor_sync(kFull, v[0], 1);
    return base < end ? base : -1;
}

}  // namespace lmrs
