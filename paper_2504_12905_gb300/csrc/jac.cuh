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
// kernels read it.
//
// The features are those of the Gaussian's exponent as a quadratic in the
// offset (dx, dy) = mu - pixel centre,
//   power = -(A dx^2 + 2 B dx dy + C dy^2) / 2,
// whose derivative along any parameter tangent is
//   d power = dx e_1 + dy e_2 + dx^2 e_3 + dx dy e_4 + dy^2 e_5
// with e_1 = -(A dmu_x + B dmu_y), e_2 = -(B dmu_x + C dmu_y), e_3 = -dA / 2,
// e_4 = -dB, e_5 = -dC / 2 (dmu, dA, ... the tangents of the mean and conic);
// then log(o) and the colour (r, g, b).  So the tangent of the exponent at a
// pixel takes five operations, alpha = o e^power moves by alpha (d power +
// d log o), and the cotangents of e_1..e_5 and log(o) are the plain moments
// (sum pbar dx, sum pbar dy, sum pbar dx^2, ..., sum pbar) of the
// back-scatter.  Layout (floats; jac_f4(DEG) float4 planes per pair):
//   [0, 6)    d(e_1, e_2) / dX                       (row-major 2 x 3)
//   [6, 36)   d(e_3, e_4, e_5) / d(X, log-scale, q)  (row-major 3 x 10)
//   [36]      d log(o) / d logit = 1 - o
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
// planes two by two ([block][q / 2][32][2] float4).  The Jacobians of 32
// consecutive Gaussians in one view are one contiguous run of F4 x 512 B,
// read coalesced by the kernels whose lanes take consecutive Gaussians; a
// kernel that reads one pair's cache alone (k_diag, at a list entry) gets
// whole 32-byte sectors, not half of each (10% off k_diag against planes
// stored one by one).
__device__ __forceinline__ long long jac_block(const Ctx& c, int slot, int g) {
    return ((long long)slot * ((c.G + 31) & ~31) + g) >> 5;
}

template <int DEG>
__device__ __forceinline__ long long jac_idx(const Ctx& c, int slot, int g, int q) {
    static_assert(Jac<DEG>::F4 % 2 == 0, "planes are stored in pairs");
    return ((jac_block(c, slot, g) * (Jac<DEG>::F4 / 2) + (q >> 1)) * 32 + (g & 31)) * 2 + (q & 1);
}

template <int DEG>
__device__ __forceinline__ void load_jac(const Ctx& c, int slot, int g, float* J) {
    const float4* base = c.pjac + jac_block(c, slot, g) * Jac<DEG>::F4 * 32 + (g & 31) * 2;
#pragma unroll
    for (int q = 0; q < Jac<DEG>::F4; ++q) {
        const float4 v = base[(q >> 1) * 64 + (q & 1)];
        J[4 * q] = v.x; J[4 * q + 1] = v.y; J[4 * q + 2] = v.z; J[4 * q + 3] = v.w;
    }
}

}  // namespace lmrs
