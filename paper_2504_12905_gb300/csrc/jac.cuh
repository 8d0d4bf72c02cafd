// Layout of the per-pair Jacobian cache, shared by the kernels that write it
// (preprocess.cu) and those that read it (preprocess.cu, raster.cu).
#pragma once

#include "common.cuh"

namespace lmrs {

template <int DEG>
struct Sh {
    static constexpr int K = (DEG + 1) * (DEG + 1);
};

// Per-pair Jacobian cache.  Within one LM step the map from a Gaussian's
// parameter tangent to the tangent of its 9 screen-space features in one view
// is linear and fixed, so it is formed once per step and the derivative
// kernels read it.  Layout (floats; jac_f4(DEG) float4 planes per pair):
//   [0, 6)    d(mu_x, mu_y) / dX                     (row-major 2 x 3)
//   [6, 36)   d(A, B, C) / d(X, log-scale, q)        (row-major 3 x 10)
//   [36]      d o / d logit = o (1 - o)
//   [37]      bit ch set: colour channel ch not clamped
//   [38, 47)  d colour / dX through the view direction (row-major 3 x 3, DEG > 0)
template <int DEG>
struct Jac {
    static constexpr int F4 = jac_f4(DEG);
    static constexpr int N = 4 * F4;
    static constexpr int kMu = 0, kCon = 6, kOp = 36, kMask = 37, kGx = 38;
};

// Blocked layout of the cache: pairs indexed slot * Gp + g (Gp = G rounded
// up to 32), blocks of 32 consecutive pairs, each block holding its F4
// planes one after the other ([block][q][32] float4).  The Jacobians of 32
// consecutive Gaussians in one view are one contiguous run of F4 x 512 B.
__device__ __forceinline__ long long jac_block(const Ctx& c, int slot, int g) {
    return ((long long)slot * ((c.G + 31) & ~31) + g) >> 5;
}

template <int DEG>
__device__ __forceinline__ long long jac_idx(const Ctx& c, int slot, int g, int q) {
    return (jac_block(c, slot, g) * Jac<DEG>::F4 + q) * 32 + (g & 31);
}

template <int DEG>
__device__ __forceinline__ void load_jac(const Ctx& c, int slot, int g, float* J) {
    const float4* base = c.pjac + jac_block(c, slot, g) * Jac<DEG>::F4 * 32 + (g & 31);
#pragma unroll
    for (int q = 0; q < Jac<DEG>::F4; ++q) {
        const float4 v = base[q * 32];
        J[4 * q] = v.x; J[4 * q + 1] = v.y; J[4 * q + 2] = v.z; J[4 * q + 3] = v.w;
    }
}

}  // namespace lmrs
