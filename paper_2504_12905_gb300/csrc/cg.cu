// Vector kernels of the preconditioned CG solve (Alg. 1) and the LM update
// with the step-size rule (Sec. 4.5, App. D).  Inner products: per-thread
// partials in compensated FP32 (Dot2, twice-working-precision accuracy),
// combined across threads in FP64 by a fixed-order grid reduction whose last
// block also forms alpha or beta; no step of the solve goes through the host.
// The streaming kernels use 16-byte accesses when every vector is 16-byte
// aligned.
#include <cstddef>
#include <cstdint>

#include "common.cuh"
#include "reduce.cuh"

namespace lmrs {

constexpr int kVecBlock = 256;

static int vec_grid(long long n) {
    long long g = (n + kVecBlock - 1) / kVecBlock;
    if (g > 1216) g = 1216;  // 8 blocks per SM on 152 SMs; grid-stride beyond
    if (g < 1) g = 1;
    return (int)g;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Jacobi preconditioner 1 / diag(A) (Sec. 4.2): 1 / (D + lambda) for the
// identity damping, 1 / ((1 + lambda) D) for the diagonal damping (0 where
// D = 0: such a parameter touches no sampled pixel, its right-hand side is 0).
__global__ void k_precond(Ctx c, const float* D, float* minv) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < c.P; j += (long long)gridDim.x * blockDim.x) {
        const float d = c.damping_mode == 1 ? (1.f + c.lambda) * D[j] : D[j] + c.lambda;
        minv[j] = d > 0.f ? 1.f / d : 0.f;
    }
}

// Element range [lo, hi) of the scalar tail after the float4 body.
struct Span {
    long long n4, lo, hi, stride, first;
};
__device__ __forceinline__ Span span(long long P, bool vec) {
    Span s;
    s.stride = (long long)gridDim.x * blockDim.x;
    s.first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    s.n4 = vec ? P / 4 : 0;
    s.lo = 4 * s.n4;
    s.hi = P;
    return s;
}

// x0 = 0, r0 = b, z0 = M^-1 r0, p = 0 (the first direction update forms
// p0 = z0), rz = r0^T z0.
template <bool kVec>
__global__ void __launch_bounds__(kVecBlock) k_cg_init(Ctx c, const float* b, const float* minv, float* x, float* r,
                                                      float* z, float* p) {
    Dot2 dot;
    const Span s = span(c.P, kVec);
    if (kVec) {
        const float4* b4 = reinterpret_cast<const float4*>(b);
        const float4* m4 = reinterpret_cast<const float4*>(minv);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        for (long long j = s.first; j < s.n4; j += s.stride) {
            const float4 bj = b4[j], mj = m4[j];
            const float4 zj = make_float4(mj.x * bj.x, mj.y * bj.y, mj.z * bj.z, mj.w * bj.w);
            reinterpret_cast<float4*>(x)[j] = zero;
            reinterpret_cast<float4*>(r)[j] = bj;
            reinterpret_cast<float4*>(z)[j] = zj;
            reinterpret_cast<float4*>(p)[j] = zero;
            dot.add(bj.x, zj.x);
            dot.add(bj.y, zj.y);
            dot.add(bj.z, zj.z);
            dot.add(bj.w, zj.w);
        }
    }
    for (long long j = s.lo + s.first; j < s.hi; j += s.stride) {
        const float bj = b[j];
        const float zj = minv[j] * bj;
        x[j] = 0.f;
        r[j] = bj;
        z[j] = zj;
        p[j] = 0.f;
        dot.add(bj, zj);
    }
    double tot;
    if (grid_sum_last<kVecBlock>(dot.value(), c.partials, c.counter, &tot) && threadIdx.x == 0) {
        Scalars* sc = c.sc;
        sc->rz = tot;
        sc->rz0 = tot;
        sc->beta = 0.0;
        if (!isfinite(tot) || tot < 0.0) sc->numeric_error = 1u;
    }
}

// x += alpha p, r -= alpha A p, z = M^-1 r, beta = r'^T z' / r^T z.
template <bool kVec>
__global__ void __launch_bounds__(kVecBlock) k_cg_update(Ctx c, int iter, const float* p, const float* Ap,
                                                        const float* minv, float* x, float* r, float* z) {
    const float alpha = (float)c.sc->alpha;
    Dot2 dot;
    const Span s = span(c.P, kVec);
    if (kVec) {
        for (long long j = s.first; j < s.n4; j += s.stride) {
            const float4 pj = reinterpret_cast<const float4*>(p)[j];
            const float4 aj = reinterpret_cast<const float4*>(Ap)[j];
            const float4 mj = reinterpret_cast<const float4*>(minv)[j];
            float4 xj = reinterpret_cast<float4*>(x)[j];
            float4 rj = reinterpret_cast<float4*>(r)[j];
            xj.x += alpha * pj.x; xj.y += alpha * pj.y; xj.z += alpha * pj.z; xj.w += alpha * pj.w;
            rj.x -= alpha * aj.x; rj.y -= alpha * aj.y; rj.z -= alpha * aj.z; rj.w -= alpha * aj.w;
            const float4 zj = make_float4(mj.x * rj.x, mj.y * rj.y, mj.z * rj.z, mj.w * rj.w);
            reinterpret_cast<float4*>(x)[j] = xj;
            reinterpret_cast<float4*>(r)[j] = rj;
            reinterpret_cast<float4*>(z)[j] = zj;
            dot.add(rj.x, zj.x);
            dot.add(rj.y, zj.y);
            dot.add(rj.z, zj.z);
            dot.add(rj.w, zj.w);
        }
    }
    for (long long j = s.lo + s.first; j < s.hi; j += s.stride) {
        x[j] += alpha * p[j];
        const float rj = r[j] - alpha * Ap[j];
        r[j] = rj;
        const float zj = minv[j] * rj;
        z[j] = zj;
        dot.add(rj, zj);
    }
    double tot;
    if (grid_sum_last<kVecBlock>(dot.value(), c.partials, c.counter, &tot) && threadIdx.x == 0) {
        Scalars* sc = c.sc;
        sc->rz_new = tot;
        sc->beta = sc->rz != 0.0 ? tot / sc->rz : 0.0;
        if (iter < 64) {
            sc->alpha_hist[iter] = sc->alpha;
            sc->beta_hist[iter] = sc->beta;
        }
        sc->rz = tot;
        if (!isfinite(tot)) sc->numeric_error = 1u;
    }
}

// max |x| over the SH degree-0 entries (the colour parameters of Sec. 4.5).
__global__ void __launch_bounds__(kVecBlock) k_max_dc(Ctx c, const float* x) {
    float m = 0.f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < c.G; g += gridDim.x * blockDim.x) {
        const float* e = x + 11ll * c.G + (long long)g * c.K * 3;
        m = fmaxf(m, fmaxf(fabsf(e[0]), fmaxf(fabsf(e[1]), fabsf(e[2]))));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&c.sc->max_dc_bits, __float_as_uint(m));
}

__device__ __forceinline__ double step_size(long long lm_step, double lr_warm, double lr_cap, double color_bound,
                                            int warm_iters, unsigned int max_bits) {
    if (lm_step < warm_iters) return lr_warm;
    const double m = (double)__uint_as_float(max_bits);
    if (m == 0.0) return lr_cap;
    return fmin(lr_cap, color_bound / m);
}

// beta <- beta - eta x; a solve that met a non-finite or non-positive
// curvature (numeric_error) leaves the parameters as they were, eta = 0
__global__ void __launch_bounds__(kVecBlock) k_lm_update(Ctx c, long long lm_step, double lr_warm, double lr_cap,
                                                        double color_bound, int warm_iters, const float* x,
                                                        float* params) {
    const bool failed = c.sc->numeric_error != 0u;
    const double eta = failed ? 0.0 : step_size(lm_step, lr_warm, lr_cap, color_bound, warm_iters, c.sc->max_dc_bits);
    if (blockIdx.x == 0 && threadIdx.x == 0) c.sc->eta = eta;
    if (failed) return;
    const float e = (float)eta;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < c.P; j += (long long)gridDim.x * blockDim.x)
        params[j] -= e * x[j];
}

// ---------------------------------------------------------------------------
// Batched CG: every scene of a batch in one launch per phase.  Chunks never
// cross a scene; the per-scene scalars of iteration i are
//   rz[i] = r_i^T z_i (accumulated by init / the previous update),
//   pAp[i] = p_i^T A p_i (accumulated by kb_prep_vjp),
// so alpha_i = rz[i] / pAp[i] and beta_i = rz[i+1] / rz[i] are formed where
// they are used.  The history arrays start at zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void b_precond_init(const BatchTables& t) {
    const int n = t.counts[1];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.vchunks[k];
        const Ctx& c = t.ctxs[ch.x];
        const BatchVec& bv = t.vecs[ch.x];
        if (ch.y == 0 && threadIdx.x == 0) {
            c.sc->max_dc_bits = 0u;
            c.sc->numeric_error = 0u;
        }
        const int mode = c.damping_mode;
        const float lam = c.lambda;
        Dot2 dot;
        for (long long j = ch.y + threadIdx.x; j < ch.z; j += kBatchBlock) {
            const float d = mode == 1 ? (1.f + lam) * bv.D[j] : bv.D[j] + lam;
            const float m = d > 0.f ? 1.f / d : 0.f;
            const float bj = bv.b[j];
            const float zj = m * bj;
            bv.minv[j] = m;
            bv.x[j] = 0.f;
            bv.r[j] = bj;
            bv.z[j] = zj;
            bv.p[j] = 0.f;
            dot.add(bj, zj);
        }
        const double tot = block_sum<kBatchBlock>(dot.value());
        if (threadIdx.x == 0) atomicAdd(&bv.rz[0], tot);
    }
}
__global__ void __launch_bounds__(kBatchBlock) kb_precond_init(BatchTables t) { b_precond_init(t); }


__device__ __forceinline__ void b_direction(const BatchTables& t, int iter) {
    const int n = t.counts[1];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.vchunks[k];
        const BatchVec& bv = t.vecs[ch.x];
        const double prev = iter > 0 ? bv.rz[iter - 1] : 0.0;
        const float beta = prev != 0.0 ? (float)(bv.rz[iter] / prev) : 0.f;
        for (long long j = ch.y + threadIdx.x; j < ch.z; j += kBatchBlock) bv.p[j] = bv.z[j] + beta * bv.p[j];
    }
}
__global__ void __launch_bounds__(kBatchBlock) kb_direction(BatchTables t, int iter) { b_direction(t, iter); }


__device__ __forceinline__ void b_update(const BatchTables& t, int iter) {
    const int n = t.counts[1];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.vchunks[k];
        const Ctx& c = t.ctxs[ch.x];
        const BatchVec& bv = t.vecs[ch.x];
        const double rz = bv.rz[iter], pap = bv.pAp[iter];
        float alpha = 0.f;
        if (rz != 0.0) {
            if (pap > 0.0 && isfinite(pap)) alpha = (float)(rz / pap);
            else if (threadIdx.x == 0) c.sc->numeric_error = 1u;
        }
        Dot2 dot;
        for (long long j = ch.y + threadIdx.x; j < ch.z; j += kBatchBlock) {
            bv.x[j] += alpha * bv.p[j];
            const float rj = bv.r[j] - alpha * bv.Ap[j];
            bv.r[j] = rj;
            const float zj = bv.minv[j] * rj;
            bv.z[j] = zj;
            dot.add(rj, zj);
        }
        const double tot = block_sum<kBatchBlock>(dot.value());
        if (threadIdx.x == 0) atomicAdd(&bv.rz[iter + 1], tot);
    }
}
__global__ void __launch_bounds__(kBatchBlock) kb_update(BatchTables t, int iter) { b_update(t, iter); }


__device__ __forceinline__ void b_max_dc(const BatchTables& t) {
    const int n = t.counts[0];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.gchunks[k];
        const Ctx& c = t.ctxs[ch.x];
        const int g = ch.y + threadIdx.x;
        float m = 0.f;
        if (g < ch.z) {
            const float* e = t.vecs[ch.x].x + 11ll * c.G + (long long)g * c.K * 3;
            m = fmaxf(fabsf(e[0]), fmaxf(fabsf(e[1]), fabsf(e[2])));
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
        if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&c.sc->max_dc_bits, __float_as_uint(m));
    }
}
__global__ void __launch_bounds__(kBatchBlock) kb_max_dc(BatchTables t) { b_max_dc(t); }


__device__ __forceinline__ void b_lm_update(const BatchTables& t) {
    const int n = t.counts[1];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.vchunks[k];
        const Ctx& c = t.ctxs[ch.x];
        const BatchVec& bv = t.vecs[ch.x];
        const bool failed = c.sc->numeric_error != 0u;
        const double eta = failed ? 0.0 : step_size(bv.lm_step, bv.lr_warm, bv.lr_cap, bv.color_bound,
                                                    bv.warm_iters, c.sc->max_dc_bits);
        if (ch.y == 0 && threadIdx.x == 0) c.sc->eta = eta;
        if (failed) continue;  // the scene's parameters stay as they were
        const float e = (float)eta;
        for (long long j = ch.y + threadIdx.x; j < ch.z; j += kBatchBlock) bv.params[j] -= e * bv.x[j];
    }
}
__global__ void __launch_bounds__(kBatchBlock) kb_lm_update(BatchTables t) { b_lm_update(t); }


void launch_b_precond_init(const BatchTables& t, int grid, cudaStream_t st) {
    LMRS_LAUNCH(kb_precond_init, grid, kBatchBlock, 0, st, t);
}
void launch_b_direction(const BatchTables& t, int iter, int grid, cudaStream_t st) {
    LMRS_LAUNCH(kb_direction, grid, kBatchBlock, 0, st, t, iter);
}
void launch_b_update(const BatchTables& t, int iter, int grid, cudaStream_t st) {
    LMRS_LAUNCH(kb_update, grid, kBatchBlock, 0, st, t, iter);
}
void launch_b_lm_update(const BatchTables& t, int, int grid, cudaStream_t st) {
    LMRS_LAUNCH(kb_max_dc, grid, kBatchBlock, 0, st, t);
    LMRS_LAUNCH(kb_lm_update, grid, kBatchBlock, 0, st, t);
}

void launch_precond(const Ctx& c, const float* D, float* minv, cudaStream_t st) {
    LMRS_LAUNCH(k_precond, vec_grid(c.P), kVecBlock, 0, st, c, D, minv);
}
void launch_cg_init(const Ctx& c, const float* b, const float* minv, float* x, float* r, float* z, float* p,
                    cudaStream_t st) {
    const bool vec = aligned16(b) && aligned16(minv) && aligned16(x) && aligned16(r) && aligned16(z) && aligned16(p);
    if (vec) LMRS_LAUNCH(k_cg_init<true>, vec_grid(c.P / 4 + 1), kVecBlock, 0, st, c, b, minv, x, r, z, p);
    else LMRS_LAUNCH(k_cg_init<false>, vec_grid(c.P), kVecBlock, 0, st, c, b, minv, x, r, z, p);
}
void launch_cg_update(const Ctx& c, int iter, const float* p, const float* Ap, const float* minv, float* x, float* r,
                      float* z, cudaStream_t st) {
    const bool vec = aligned16(p) && aligned16(Ap) && aligned16(minv) && aligned16(x) && aligned16(r) && aligned16(z);
    if (vec) LMRS_LAUNCH(k_cg_update<true>, vec_grid(c.P / 4 + 1), kVecBlock, 0, st, c, iter, p, Ap, minv, x, r, z);
    else LMRS_LAUNCH(k_cg_update<false>, vec_grid(c.P), kVecBlock, 0, st, c, iter, p, Ap, minv, x, r, z);
}
void launch_max_dc(const Ctx& c, const float* x, cudaStream_t st) {
    LMRS_LAUNCH(k_max_dc, vec_grid(c.G), kVecBlock, 0, st, c, x);
}
void launch_lm_update(const Ctx& c, long long lm_step, double lr_warm, double lr_cap, double color_bound,
                      int warm_iters, const float* x, float* params, cudaStream_t st) {
    LMRS_LAUNCH(k_lm_update, vec_grid(c.P), kVecBlock, 0, st, c, lm_step, lr_warm, lr_cap, color_bound, warm_iters, x,
                params);
}
void launch_zero_scalars(const Ctx& c, cudaStream_t st) {
    cudaMemsetAsync(c.sc, 0, offsetof(Scalars, loss_num), st);
}

}  // namespace lmrs
