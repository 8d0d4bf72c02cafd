// Rasterisation kernels of the LM-RS hot path.  One warp handles one work
// item: up to 32 sampled pixels of one (view, tile) (Sec. 4.4: per-tile
// stratified samples), front to back over the tile's depth-sorted list
// (Eq. 4, Alg. 2).  Gaussian records are staged 32 at a time into the warp's
// shared-memory slice with coalesced id loads and 16-byte record loads.
//
//   k_fwd_samples  render + residual (Eq. 7) + per-sample caches; also the
//                  work item's compact list: the entries at which at least
//                  one of its live pixels has alpha >= 1/255 (every other
//                  entry is skipped by all of them, so dropping it changes no
//                  pixel), and each pixel's stopping position in it
//   k_full         full frames (all pixels)
//   k_jvp          u = J v, dual-number style tangent compositing (Alg. 3)
//   k_vjp          back-scatter of a per-sample cotangent (App. A, J^T v
//                  kernel, first launch) using the cached final colour and
//                  stopping position
//   k_jtj          fused: JVP pass then VJP pass of w * (J v) per work item
//   k_diag         diag(J^T W J) row by row into per-pair slots (App. A, Diag
//                  kernel; completed by k_prep_diag), optionally with the
//                  right-hand side's back-scatter in the same walk
//   k_ssim         the diagonal SSIM term at every sample (from full frames)
// k_vjp, k_jtj and k_diag walk the compact lists.  Back-scatter: the lanes
// first write per-(entry, sample) values to shared memory in list order, then
// the lanes take the entries and sum over the samples, so each (work item,
// list entry) adds its cotangents with a few vector atomics and no warp
// reduction (backward_pass).
#include "common.cuh"
#include "jac.cuh"
#include "reduce.cuh"

namespace lmrs {

constexpr int kRasterWarps = 4;
constexpr int kRasterBlock = kRasterWarps * kWarp;

// 2^x on the special-function unit.  The records carry the conic scaled by
// -log2(e)/2 (A, C) and -log2(e) (B), so e^power = 2^(dx (A' dx + B' dy) +
// C' dy^2) takes five FP32 operations and one 2^x.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// e^power at offset d = mu - pixel centre from the third float4 of a pair's
// record, (b, B', A', C'): (A' dx, C' dy) is one paired multiply.
__device__ __forceinline__ float gauss_ex2(float4 r2, float2 d) {
    const float2 ac = __fmul2_rn(make_float2(r2.z, r2.w), d);
    return ex2_approx(fmaf(ac.y, d.y, d.x * fmaf(r2.y, d.y, ac.x)));
}

struct Pix {
    int vt, slot, tile, chunk;
    long long si;
    bool active;
    float pcx, pcy;
    float2 npc;  // -(pcx, pcy)
    int px, py;
    float w;
};

__device__ __forceinline__ void setup_item(const Ctx& c, int item, Pix& p) {
    const int lane = threadIdx.x & 31;
    const int2 wk = c.work[item];
    p.vt = wk.x;
    p.chunk = wk.y >> 5;
    p.slot = p.vt / c.T;
    p.tile = p.vt - p.slot * c.T;
    const int tx = p.tile % c.tiles_x, ty = p.tile / c.tiles_x;
    const int vw = min(c.tile_w, c.W - tx * c.tile_w);
    const int s0 = c.tile_off[p.vt], s1 = c.tile_off[p.vt + 1];
    p.si = (long long)s0 + wk.y + lane;
    p.active = p.si < s1;
    const int o = p.active ? c.off[p.si] : 0;
    p.px = tx * c.tile_w + o % vw;
    p.py = ty * c.tile_h + o / vw;
    p.pcx = p.px + 0.5f;
    p.pcy = p.py + 0.5f;
    p.npc = make_float2(-p.pcx, -p.pcy);
    p.w = c.wsample ? (p.active ? c.wsample[p.si] : 0.f) : c.wtile[p.vt];
}

// Weight of the sample's channel-ch row in J^T W J: w, times 1 + ssim_weight
// d^2 with the SSIM term (its row is d times the colour's).
__device__ __forceinline__ float row_weight(const Ctx& c, const Pix& p, int ch) {
    if (!c.ssim_d || !p.active) return p.w;
    const float d = c.ssim_d[3 * p.si + ch];
    return p.w * fmaf(c.ssim_weight * d, d, 1.f);
}

// The list a kernel walks: ids[b, e).
struct List {
    const unsigned* ids;
    int b, e;
};

// Compact list of a work item: capacity max_items * (tile list length) per
// tile, chunk q at offset max_items * begin + q * length.
__device__ __forceinline__ long long compact_base(const Ctx& c, const Pix& p, int2 rg) {
    return (long long)c.max_items * rg.x + (long long)p.chunk * (rg.y - rg.x);
}

__device__ __forceinline__ List compact_list(const Ctx& c, const Pix& p) {
    const int2 rg = c.ranges[p.vt];
    List L;
    L.ids = c.cids + compact_base(c, p, rg);
    L.b = 0;
    L.e = c.clen[(long long)p.vt * c.max_items + p.chunk];
    return L;
}

__device__ __forceinline__ List tile_list(const Ctx& c, const Pix& p) {
    const int2 rg = c.ranges[p.vt];
    List L;
    L.ids = c.ids;
    L.b = rg.x;
    L.e = rg.y;
    return L;
}

template <int NF4, int W, int R = 32>
__device__ __forceinline__ int stage_batch(const Ctx& c, int slot, const unsigned* ids, int b, int end,
                                           float4 (*s_rec)[W], unsigned* s_id) {
    static_assert(NF4 <= W, "staged row too narrow");
    const int lane = threadIdx.x & 31;
    const int k = b + lane;
    if (lane < R && k < end) {
        unsigned id = ids[k];
        LMRS_DCHECK_INDEX(c, id, c.G, kCheckStagedId);
        const long long pr = (long long)slot * c.G + id;
#pragma unroll
        for (int q = 0; q < NF4; ++q) s_rec[lane][q] = q < kPrimF4 ? c.rec[pr * kPrimF4 + q] : c.tan[pr * kTanF4 + q - kPrimF4];
        if (s_id) s_id[lane] = id;
    }
    __syncwarp();
    return min(R, end - b);
}

// Front-to-back pass.  With kTan also the tangent of the colour (Alg. 3).
// ncons = entries of the walked list consumed before termination (all of
// them if none).  With kCompact the needed entries are appended to out_ids
// and ncons counts them instead; *out_len receives their number.
template <bool kTan, bool kCompact>
__device__ __forceinline__ void forward_pass(const Ctx& c, const Pix& p, List L, float4 (*s_rec)[kRecF4],
                                             unsigned* s_id, float C[3], float& T, float dC[3], int& ncons,
                                             unsigned* out_ids = nullptr, int* out_len = nullptr,
                                             int* n_comp = nullptr) {
    const int lane = threadIdx.x & 31;
    T = 1.f;
    float dT = 0.f;
    C[0] = C[1] = C[2] = 0.f;
    dC[0] = dC[1] = dC[2] = 0.f;
    bool done = !p.active;
    ncons = L.e - L.b;
    int kept = 0;
    for (int b = L.b; b < L.e; b += 32) {
        if (__all_sync(kFull, done)) break;
        const int n = stage_batch<kTan ? 6 : 3>(c, p.slot, L.ids, b, L.e, s_rec, s_id);
        for (int j = 0; j < n; ++j) {
            const float4 r0 = s_rec[j][0], r1 = s_rec[j][1], r2 = s_rec[j][2];
            const float2 d = __fadd2_rn(make_float2(r0.x, r0.y), p.npc);
            const float dx = d.x, dy = d.y;
            const float gval = gauss_ex2(r2, d);
            const float raw = r1.y * gval;
            float alpha = fminf(kAlphaMax, raw);
            bool need = !done && alpha >= kAlphaMin;
            if (kCompact) {
                const bool any = __any_sync(kFull, need);
                if (any && lane == 0) {
                    int slot_k = kept;
                    LMRS_DCHECK_INDEX(c, slot_k, L.e - L.b, kCheckCompactWrite);
                    out_ids[slot_k] = s_id[j];
                }
                if (need) {
                    const float Tn = T * (1.f - alpha);
                    if (Tn < kTMin) {
                        done = true;
                        ncons = kept;
                    } else {
                        const float wgt = alpha * T;
                        C[0] += r1.z * wgt;
                        C[1] += r1.w * wgt;
                        C[2] += r2.x * wgt;
                        T = Tn;
                        if (n_comp) ++*n_comp;
                    }
                }
                if (any) ++kept;
                continue;
            }
            // branch-free: an entry the lane does not composite takes alpha = 0,
            // which leaves T, C and their tangents unchanged
            const float Tn0 = T * (1.f - alpha);
            const bool stop = need && Tn0 < kTMin;
            if (stop) {
                done = true;
                ncons = b + j - L.b;
            }
            const bool comp = need && !stop;
            alpha = comp ? alpha : 0.f;
            const float Tn = T * (1.f - alpha);
            const float col2 = r2.x;
            const float wgt = alpha * T;
            if (kTan) {
                // tangent record (e_1, e_2, e_3, e_4 | e_5, log o, r, g | b):
                // alpha moves by raw (dx e_1 + dy e_2 + dx^2 e_3 + dx dy e_4 +
                // dy^2 e_5 + d log o) where it is not clamped
                const float4 t0 = s_rec[j][3], t1 = s_rec[j][4];
                const float dcol2 = s_rec[j][5].x;
                const float dlin = fmaf(dx, fmaf(t0.z, dx, fmaf(t0.w, dy, t0.x)), fmaf(dy, fmaf(t1.x, dy, t0.y), t1.y));
                const float dalpha = (comp && raw <= kAlphaMax) ? raw * dlin : 0.f;
                const float dw = dalpha * T + alpha * dT;
                dC[0] += t1.z * wgt + r1.z * dw;
                dC[1] += t1.w * wgt + r1.w * dw;
                dC[2] += dcol2 * wgt + col2 * dw;
                dT = dT * (1.f - alpha) - T * dalpha;
            }
            C[0] += r1.z * wgt;
            C[1] += r1.w * wgt;
            C[2] += col2 * wgt;
            T = Tn;
            if (n_comp && comp) ++*n_comp;
        }
        __syncwarp();
    }
    if (kCompact) {
        if (!done) ncons = kept;
        if (out_len && lane == 0) *out_len = kept;
    }
}

// Back-scatter of the cotangent ub of each lane's colour into the 9 feature
// cotangents of every contributing Gaussian (reverse mode through Eq. 4 with
// the final colour Cf known: dC/dalpha_n = T_n c_n - (Cf - C_<=n)/(1 - alpha_n)).
// Lane stops after its first ncons entries of the list.
//
// Two phases per kBwdE staged entries, so that no warp reduction is needed:
//   A  lane = sample, in list order: alpha, T and the running sum give, per
//      entry, pbar = <ub, dC/dalpha> raw (0 where alpha is clamped: alpha
//      then does not move with the features) and wgt = alpha T, written to
//      pw[entry][lane];
//   B  lane = (entry e, half hh of the samples): the lane sums its entry's
//      moments over its samples (dx = mu_x - pixel x, dy likewise)
//        Mx = sum pbar dx, My = sum pbar dy, Mxx = sum pbar dx^2,
//        Mxy = sum pbar dx dy, Myy = sum pbar dy^2, M5 = sum pbar,
//        Mc_ch = sum ub_ch wgt,
//      the two halves are added with one shuffle per moment; the moments
//      are the cotangents of the exponent's coefficients e_1..e_5 (jac.cuh):
//        (Mx, My, Mxx, Mxy, Myy);  log o: M5 (alpha = o e^power, so
//        d alpha / d log o = raw);  colour: Mc,
//      added with two 4-wide and one scalar atomic.
constexpr int kBwdE = 16;  // entries per phase; lanes e and e + 16 share entry e

struct BwdSmem {
    // pbar and wgt per (entry, sample), planar; row stride 34 (even, for the
    // sample-pair loads, and 2 mod 32) keeps phase B's reads conflict-free
    float pb[kBwdE][34], wt[kBwdE][34];
    float npx[32], npy[32];  // per sample: minus the pixel centre
    float u0[32], u1[32], u2[32];
};

// One staged batch per warp, plus the back-scatter's exchange area.  The
// batch's Gaussian ids are read back from the list where they are needed.
constexpr int kJtjRows = 16;  // list entries staged at a time by k_jtj and k_vjp
constexpr int kJtjF4 = 5;     // float4 per staged row (the JVP pass's layout)
struct WarpSmem {
    float4 rec[kJtjRows][kJtjF4];
    BwdSmem bw;
};

__device__ __forceinline__ float2 ld2(const float* a) { return *reinterpret_cast<const float2*>(a); }

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void backward_pass(const Ctx& c, const Pix& p, List L, WarpSmem& sm, const float ub[3],
                                              const float Cf[3], int ncons) {
    const int lane = threadIdx.x & 31;
    const float S_tot = ub[0] * Cf[0] + ub[1] * Cf[1] + ub[2] * Cf[2];
    float s = 0.f, T = 1.f;
    const int lane_end = p.active ? L.b + ncons : L.b;
    int warp_end = lane_end;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) warp_end = max(warp_end, __shfl_xor_sync(kFull, warp_end, m));
    // the live samples are lanes [0, nact)
    const int nact = __popc(__ballot_sync(kFull, p.active));
    sm.bw.npx[lane] = -p.pcx;
    sm.bw.npy[lane] = -p.pcy;
    sm.bw.u0[lane] = ub[0];
    sm.bw.u1[lane] = ub[1];
    sm.bw.u2[lane] = ub[2];
    float* cot_base = c.cot + (long long)p.slot * c.G * kCotF;
    const int e = lane & (kBwdE - 1), hh = lane >> 4;
    for (int b = L.b; b < warp_end; b += kJtjRows) {
        const int n = stage_batch<3, kJtjF4, kJtjRows>(c, p.slot, L.ids, b, warp_end, sm.rec, nullptr);
        for (int h0 = 0; h0 < n; h0 += kBwdE) {
            const int m = min(kBwdE, n - h0);
            // phase A
            for (int jj = 0; jj < m; ++jj) {
                const int j = h0 + jj;
                const float4 r0 = sm.rec[j][0], r1 = sm.rec[j][1], r2 = sm.rec[j][2];
                const float col2 = r2.x;
                const float gval = gauss_ex2(r2, __fadd2_rn(make_float2(r0.x, r0.y), p.npc));
                const float raw = r1.y * gval;
                float alpha = fminf(kAlphaMax, raw);
                // branch-free: an entry the lane does not composite (past its
                // stop, or alpha < 1/255) takes alpha = 0, which leaves T and s
                // unchanged and gives pb = wt = 0
                const bool on = (b + j < lane_end) && alpha >= kAlphaMin;
                alpha = on ? alpha : 0.f;
                const float ucol = ub[0] * r1.z + ub[1] * r1.w + ub[2] * col2;
                const float wt = alpha * T;
                s += ucol * wt;
                const float abar = T * ucol - __fdividef(S_tot - s, 1.f - alpha);  // 1 - alpha >= 0.01
                const float pb = (on && raw <= kAlphaMax) ? abar * raw : 0.f;
                T *= 1.f - alpha;
                sm.bw.pb[jj][lane] = pb;
                sm.bw.wt[jj][lane] = wt;
            }
            __syncwarp();
            // phase B, in paired FP32 operations (f32x2: two lanes of
            // arithmetic per issued instruction, each rounded as alone) over
            // sample pairs (i, i + 1): samples past the live ones hold
            // pbar = wgt = 0 (phase A writes every lane), so the pairs run to
            // an even count; the two lanes of an entry take alternate pairs
            float2 M[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) M[k] = make_float2(0.f, 0.f);
            const int j = h0 + e;
            if (e < m) {
                const float2 mx = make_float2(sm.rec[j][0].x, sm.rec[j][0].x);
                const float2 my = make_float2(sm.rec[j][0].y, sm.rec[j][0].y);
                for (int i = 2 * hh; i < nact; i += 4) {
                    const float2 q = ld2(&sm.bw.pb[e][i]), w = ld2(&sm.bw.wt[e][i]);
                    const float2 dx = __fadd2_rn(mx, ld2(&sm.bw.npx[i]));
                    const float2 dy = __fadd2_rn(my, ld2(&sm.bw.npy[i]));
                    const float2 pdx = __fmul2_rn(q, dx), pdy = __fmul2_rn(q, dy);
                    M[0] = __fadd2_rn(M[0], pdx);
                    M[1] = __fadd2_rn(M[1], pdy);
                    M[2] = __ffma2_rn(pdx, dx, M[2]);
                    M[3] = __ffma2_rn(pdx, dy, M[3]);
                    M[4] = __ffma2_rn(pdy, dy, M[4]);
                    M[5] = __fadd2_rn(M[5], q);
                    M[6] = __ffma2_rn(ld2(&sm.bw.u0[i]), w, M[6]);
                    M[7] = __ffma2_rn(ld2(&sm.bw.u1[i]), w, M[7]);
                    M[8] = __ffma2_rn(ld2(&sm.bw.u2[i]), w, M[8]);
                }
            }
            float Ms[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                Ms[k] = M[k].x + M[k].y;
                Ms[k] += __shfl_xor_sync(kFull, Ms[k], 16);
            }
            if (hh == 0 && e < m) {
                unsigned id = L.ids[b + j];
                LMRS_DCHECK_INDEX(c, id, c.G, kCheckScatterId);
                float* dst = cot_base + (long long)id * kCotF;
                red_add_v4(dst, Ms[0], Ms[1], Ms[2], Ms[3]);
                red_add_v4(dst + 4, Ms[4], Ms[5], Ms[6], Ms[7]);
                atomicAdd(dst + 8, Ms[8]);
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ void load_cache(const Ctx& c, long long si, float Cf[3], int& ncons) {
    if (c.cache_bf16) {
        Cf[0] = __bfloat162float(c.cacheCh[3 * si]);
        Cf[1] = __bfloat162float(c.cacheCh[3 * si + 1]);
        Cf[2] = __bfloat162float(c.cacheCh[3 * si + 2]);
    } else {
        Cf[0] = c.cacheC[3 * si];
        Cf[1] = c.cacheC[3 * si + 1];
        Cf[2] = c.cacheC[3 * si + 2];
    }
    ncons = c.cacheN[si];
}

#define LMRS_RASTER_PROLOGUE                                                    \
    __shared__ float4 s_rec_all[kRasterWarps][32][kRecF4];                      \
    __shared__ unsigned s_id_all[kRasterWarps][32];                             \
    const int wid = threadIdx.x >> 5;                                           \
    const int item = blockIdx.x * kRasterWarps + wid;                           \
    if (item >= c.nwork) return;                                                \
    float4(*s_rec)[kRecF4] = s_rec_all[wid];                                    \
    unsigned* s_id = s_id_all[wid];                                             \
    Pix p;                                                                      \
    setup_item(c, item, p);

__global__ void __launch_bounds__(kRasterBlock) k_fwd_samples(Ctx c) {
    LMRS_RASTER_PROLOGUE
    const int2 rg = c.ranges[p.vt];
    float C[3], T, dC[3];
    int ncons;
    int* len_out = c.clen + (long long)p.vt * c.max_items + p.chunk;
    int n_comp = 0;
    forward_pass<false, true>(c, p, tile_list(c, p), s_rec, s_id, C, T, dC, ncons,
                              c.cids + compact_base(c, p, rg), len_out, &n_comp);
    double num = 0.0, den = 0.0;
    if (p.active) {
        const long long si = p.si;
        float r[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float tgt = 0.f;
            if (c.targets) {
                const int cam = c.views[p.slot];
                tgt = c.targets[(((long long)cam * c.H + p.py) * c.W + p.px) * 3 + ch];
            }
            r[ch] = C[ch] - tgt;
            c.resid[3 * si + ch] = r[ch];
        }
        if (c.cache_bf16) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) c.cacheCh[3 * si + ch] = __float2bfloat16_rn(C[ch]);
            c.cacheTh[si] = __float2bfloat16_rn(T);
        } else {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) c.cacheC[3 * si + ch] = C[ch];
            c.cacheT[si] = T;
        }
        c.cacheN[si] = ncons;
        num = (double)p.w * ((double)r[0] * r[0] + (double)r[1] * r[1] + (double)r[2] * r[2]);
        den = 3.0 * p.w;
    }
    // traversal length of this work item in the kernels that walk the compact list
    if ((threadIdx.x & 31) == 0 && c.item_cost) c.item_cost[item] = *len_out;
    num = warp_sum(num);
    den = warp_sum(den);
    unsigned long long ne = p.active ? (unsigned long long)n_comp : 0ull;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) ne += __shfl_xor_sync(kFull, ne, o);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&c.sc->loss_num, num);
        atomicAdd(&c.sc->loss_den, den);
        atomicAdd(&c.sc->n_eval, ne);
        atomicAdd(&c.sc->n_walk, (unsigned long long)*len_out);
    }
}

__global__ void __launch_bounds__(kRasterBlock) k_jvp(Ctx c, float* u) {
    LMRS_RASTER_PROLOGUE
    float C[3], T, dC[3];
    int ncons;
    forward_pass<true, false>(c, p, tile_list(c, p), s_rec, s_id, C, T, dC, ncons);
    if (p.active) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) u[3 * p.si + ch] = dC[ch];
    }
}

__global__ void __launch_bounds__(kRasterBlock) k_vjp(Ctx c, const float* u) {
    __shared__ WarpSmem s_warp[kRasterWarps];
    const int wid = threadIdx.x >> 5;
    const int item = blockIdx.x * kRasterWarps + wid;
    if (item >= c.nwork) return;
    Pix p;
    setup_item(c, item, p);
    float ub[3] = {0.f, 0.f, 0.f}, Cf[3] = {0.f, 0.f, 0.f};
    int ncons = 0;
    if (p.active) {
        load_cache(c, p.si, Cf, ncons);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (u) {
                ub[ch] = u[3 * p.si + ch];
            } else {
                // J^T W r, plus ssim_weight * w * d * s for the SSIM rows
                float r = c.resid[3 * p.si + ch];
                if (c.ssim_s) r = fmaf(c.ssim_weight * c.ssim_d[3 * p.si + ch], c.ssim_s[3 * p.si + ch], r);
                ub[ch] = p.w * r;
            }
        }
    }
    backward_pass(c, p, compact_list(c, p), s_warp[wid], ub, Cf, ncons);
}

// The JVP pass of k_jtj (Alg. 3 over the compact list).  Within an LM step
// the primal is fixed, so each lane's stopping position (lane_end, from the
// forward render's cache) replaces the termination test, and the final
// colour comes from the cache: the pass carries T and the tangents only.
// With kColour it also accumulates the primal colour C, for the BF16 cache
// mode, whose cached colour is too coarse for the back-scatter's suffix
// Cf - C_<=n.  alpha >= 1/255 is tested on raw: the clamp at 0.99 is above
// the threshold, so the decision is the same.
//
// Its own staged layout, five float4 per entry, puts each channel's colour
// tangent beside its colour, so that dC_ch = sum dc_ch wgt + c_ch dw is one
// paired FMA per channel into (sum dc_ch wgt, sum c_ch dw):
//   (mu_x, mu_y, A', C') (dr, r, dg, g) (db, b, B', o) (e_1..e_4) (e_5, d log o, -, -)

__device__ __forceinline__ void stage_jvp(const Ctx& c, int slot, const unsigned* ids, int b, int end,
                                          float4 (*s)[kJtjF4]) {
    const int lane = threadIdx.x & 31;
    const int k = b + lane;
    if (lane < kJtjRows && k < end) {
        unsigned id = ids[k];
        LMRS_DCHECK_INDEX(c, id, c.G, kCheckStagedId);
        const long long pr = (long long)slot * c.G + id;
        const float4 a0 = c.rec[pr * kPrimF4], a1 = c.rec[pr * kPrimF4 + 1], a2 = c.rec[pr * kPrimF4 + 2];
        const float4 t0 = c.tan[pr * kTanF4], t1 = c.tan[pr * kTanF4 + 1];
        const float tb = reinterpret_cast<const float*>(c.tan + pr * kTanF4 + 2)[0];
        s[lane][0] = make_float4(a0.x, a0.y, a2.z, a2.w);
        s[lane][1] = make_float4(t1.z, a1.z, t1.w, a1.w);
        s[lane][2] = make_float4(tb, a2.x, a2.y, a1.y);
        s[lane][3] = t0;
        s[lane][4] = make_float4(t1.x, t1.y, 0.f, 0.f);
    }
    __syncwarp();
}

template <bool kColour>
__device__ __forceinline__ void jvp_pass(const Ctx& c, const Pix& p, List L, int lane_end, int warp_end,
                                         float4 (*s_rec)[kJtjF4], float C[3], float dC[3]) {
    float T = 1.f, dT = 0.f;
    C[0] = C[1] = C[2] = 0.f;
    float2 dCp[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int b = L.b; b < warp_end; b += kJtjRows) {
        stage_jvp(c, p.slot, L.ids, b, warp_end, s_rec);
        const int n = min(kJtjRows, warp_end - b);
        const int rem = lane_end - b;
        for (int j = 0; j < n; ++j) {
            const float4 s0 = s_rec[j][0], s1 = s_rec[j][1], s2 = s_rec[j][2];
            const float2 d = __fadd2_rn(make_float2(s0.x, s0.y), p.npc);
            const float2 ac = __fmul2_rn(make_float2(s0.z, s0.w), d);
            const float raw = s2.w * ex2_approx(fmaf(ac.y, d.y, d.x * fmaf(s2.z, d.y, ac.x)));
            // alpha = 0 where the lane does not composite the entry: T, C and
            // the tangents stay as they are
            const bool on = j < rem && raw >= kAlphaMin;
            const float alpha = on ? fminf(kAlphaMax, raw) : 0.f;
            const float4 t0 = s_rec[j][3];
            const float2 t1 = make_float2(s_rec[j][4].x, s_rec[j][4].y);
            const float dx = d.x, dy = d.y;
            const float dlin = fmaf(dx, fmaf(t0.z, dx, fmaf(t0.w, dy, t0.x)), fmaf(dy, fmaf(t1.x, dy, t0.y), t1.y));
            const float dalpha = (on && raw <= kAlphaMax) ? raw * dlin : 0.f;
            const float2 wd = make_float2(alpha * T, fmaf(dalpha, T, alpha * dT));  // (wgt, dw)
            dCp[0] = __ffma2_rn(make_float2(s1.x, s1.y), wd, dCp[0]);
            dCp[1] = __ffma2_rn(make_float2(s1.z, s1.w), wd, dCp[1]);
            dCp[2] = __ffma2_rn(make_float2(s2.x, s2.y), wd, dCp[2]);
            if (kColour) {
                C[0] = fmaf(s1.y, wd.x, C[0]);
                C[1] = fmaf(s1.w, wd.x, C[1]);
                C[2] = fmaf(s2.y, wd.x, C[2]);
            }
            const float om = 1.f - alpha;
            dT = dT * om - T * dalpha;
            T *= om;
        }
        __syncwarp();
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dC[ch] = dCp[ch].x + dCp[ch].y;
}

__device__ __forceinline__ void jtj_item(const Ctx& c, int item, WarpSmem& sm) {
    Pix p;
    setup_item(c, item, p);
    const List L = compact_list(c, p);
    float Cf[3] = {0.f, 0.f, 0.f}, C[3], dC[3];
    int ncons = 0;
    if (p.active) {
        ncons = c.cacheN[p.si];
        if (!c.cache_bf16) {
            Cf[0] = c.cacheC[3 * p.si];
            Cf[1] = c.cacheC[3 * p.si + 1];
            Cf[2] = c.cacheC[3 * p.si + 2];
        }
    }
    const int lane_end = p.active ? L.b + ncons : L.b;
    int warp_end = lane_end;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) warp_end = max(warp_end, __shfl_xor_sync(kFull, warp_end, m));
    if (c.cache_bf16) {
        jvp_pass<true>(c, p, L, lane_end, warp_end, sm.rec, C, dC);
        Cf[0] = C[0], Cf[1] = C[1], Cf[2] = C[2];
    } else {
        jvp_pass<false>(c, p, L, lane_end, warp_end, sm.rec, C, dC);
    }
    const float ub[3] = {row_weight(c, p, 0) * dC[0], row_weight(c, p, 1) * dC[1], row_weight(c, p, 2) * dC[2]};
    __syncwarp();
    backward_pass(c, p, L, sm, ub, Cf, ncons);
}

__global__ void __launch_bounds__(kRasterBlock, 8) k_jtj(Ctx c) {
    __shared__ WarpSmem s_warp[kRasterWarps];
    const int wid = threadIdx.x >> 5;
    const int item = blockIdx.x * kRasterWarps + wid;
    if (item < c.nwork) jtj_item(c, item, s_warp[wid]);
}

// The same for every scene of a batch: chunks of at most kRasterWarps work
// items of one scene, one item per warp.
__device__ __forceinline__ void b_jtj(const BatchTables& t, WarpSmem* s_warp) {
    static_assert(kRasterBlock == kBatchBlock, "one warp per work item of a chunk");
    const int wid = threadIdx.x >> 5;
    const int n = t.counts[2];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.wchunks[k];
        const int item = ch.y + wid;
        if (item < ch.z) jtj_item(t.ctxs[ch.x], item, s_warp[wid]);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kRasterBlock) kb_jtj(BatchTables t) {
    __shared__ WarpSmem s_warp[kRasterWarps];
    b_jtj(t, s_warp);
}

void launch_b_jtj(const BatchTables& t, int grid, cudaStream_t st) {
    LMRS_LAUNCH(kb_jtj, grid, kRasterBlock, 0, st, t);
}

// diag(J^T W J) row by row (App. A, Diag kernel), optionally with the right-
// hand side J^T W r in the same walk.  Per contributing (sample, Gaussian)
// and channel, the row of J restricted to the Gaussian's geometric parameter
// k is
//   hr_ch (et . a_k) + q acol_ch,k
// with q = alpha T, h_ch = dC_ch/dalpha, hr_ch = h_ch raw (0 where alpha is
// clamped), et = d power / d(mu_x, mu_y, A, B, C) (= -(A dx + B dy),
// -(B dx + C dy), -dx^2/2, -dx dy, -dy^2/2), a_k column k of the pair's
// Jacobian cache and acol its colour-through-direction part (DEG > 0).  Its
// square, weighted by the channel's row weight w_ch, is added to the pair's
// slot: every term is non-negative, so each entry of D keeps its own relative
// accuracy however small it is next to the rest of its Gaussian's block.
// Slot (kDiagF floats): [0, 10) the 10 parameters X, log-scale, q; [10] the
// opacity logit, (1 - o)^2 sum_ch w_ch hr_ch^2 (dalpha/dlogit = raw (1 - o));
// [11, 14) sum w_ch q^2 per channel, which k_prep_diag turns into the SH
// entries (colour ch moves by Y_k per unit of coefficient (k, ch)).
// Two phases per kBwdE staged entries as in backward_pass: A (lane = sample)
// writes (q, hr_0, hr_1, hr_2); B (lane = (entry, half of the samples)) sums
// the rows over the samples with the entry's Jacobian in registers, and the
// halves are added with one shuffle per value.
struct DiagSmem {
    float4 rec[32][kPrimF4];
    unsigned id[32];
    float4 qh[kBwdE][33];  // (q, hr_0, hr_1, hr_2) per (entry, sample)
    float4 pix0[32];       // pixel centre x, y, w_0, w_1
    float4 pix1[32];       // w_2, ub_0, ub_1, ub_2 (right-hand side cotangent)
};

template <int DEG, bool kRhs>
__global__ void __launch_bounds__(kRasterBlock) k_diag(Ctx c) {
    using LJ = Jac<DEG>;
    __shared__ DiagSmem s_warp[kRasterWarps];
    const int wid = threadIdx.x >> 5;
    const int item = blockIdx.x * kRasterWarps + wid;
    if (item >= c.nwork) return;
    DiagSmem& sm = s_warp[wid];
    Pix p;
    setup_item(c, item, p);
    const List L = compact_list(c, p);
    const int lane = threadIdx.x & 31;
    float Cf[3] = {0.f, 0.f, 0.f};
    int ncons = 0;
    if (p.active) load_cache(c, p.si, Cf, ncons);
    float ub[3] = {0.f, 0.f, 0.f};
    if (kRhs && p.active)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float r = c.resid[3 * p.si + ch];
            if (c.ssim_s) r = fmaf(c.ssim_weight * c.ssim_d[3 * p.si + ch], c.ssim_s[3 * p.si + ch], r);
            ub[ch] = p.w * r;
        }
    sm.pix0[lane] = make_float4(p.pcx, p.pcy, row_weight(c, p, 0), row_weight(c, p, 1));
    sm.pix1[lane] = make_float4(row_weight(c, p, 2), ub[0], ub[1], ub[2]);
    const int nact = __popc(__ballot_sync(kFull, p.active));
    const int lane_end = p.active ? L.b + ncons : L.b;
    int warp_end = lane_end;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) warp_end = max(warp_end, __shfl_xor_sync(kFull, warp_end, m));
    float acc[3] = {0.f, 0.f, 0.f}, T = 1.f;
    float* dbase = c.dslot + (long long)p.slot * c.G * kDiagF;
    float* cbase = c.cot + (long long)p.slot * c.G * kCotF;
    const int e = lane & (kBwdE - 1), hh = lane >> 4;
    for (int b = L.b; b < warp_end; b += 32) {
        const int n = stage_batch<3>(c, p.slot, L.ids, b, warp_end, sm.rec, sm.id);
        for (int h0 = 0; h0 < n; h0 += kBwdE) {
            const int m = min(kBwdE, n - h0);
            // phase A
            for (int jj = 0; jj < m; ++jj) {
                const int j = h0 + jj;
                const float4 r0 = sm.rec[j][0], r1 = sm.rec[j][1], r2 = sm.rec[j][2];
                const float col[3] = {r1.z, r1.w, r2.x};
                const float gval = gauss_ex2(r2, __fadd2_rn(make_float2(r0.x, r0.y), p.npc));
                const float raw = r1.y * gval;
                float alpha = fminf(kAlphaMax, raw);
                // branch-free as in backward_pass: alpha = 0 where the lane
                // does not composite the entry, so q = hr = 0 there
                const bool on = (b + j < lane_end) && alpha >= kAlphaMin;
                alpha = on ? alpha : 0.f;
                const float q = alpha * T;
                const float inv = __fdividef(1.f, 1.f - alpha);  // 1 - alpha >= 0.01
                const float rr = (on && raw <= kAlphaMax) ? raw : 0.f;
                float hr[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    acc[ch] += col[ch] * q;
                    hr[ch] = rr * (T * col[ch] - (Cf[ch] - acc[ch]) * inv);
                }
                sm.qh[jj][lane] = make_float4(q, hr[0], hr[1], hr[2]);
                T *= 1.f - alpha;
            }
            __syncwarp();
            // phase B
            float D[14], M[9];
#pragma unroll
            for (int k = 0; k < 14; ++k) D[k] = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) M[k] = 0.f;
            const int j = h0 + e;
            if (e < m) {
                float J[LJ::N];
                load_jac<DEG>(c, p.slot, (int)sm.id[j], J);
                const float4 r0 = sm.rec[j][0];
                const unsigned bits = __float_as_uint(J[LJ::kMask]);
                float acol[3][3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                    for (int k = 0; k < 3; ++k) acol[ch][k] = (DEG > 0 && ((bits >> ch) & 1u)) ? J[LJ::kGx + 3 * ch + k] : 0.f;
                for (int i = hh; i < nact; i += 2) {
                    const float4 qh = sm.qh[e][i];
                    const float4 x0 = sm.pix0[i], x1 = sm.pix1[i];
                    const float dx = r0.x - x0.x, dy = r0.y - x0.y;
                    // d power = dx e_1 + dy e_2 + dx^2 e_3 + dx dy e_4 + dy^2 e_5 (jac.cuh)
                    const float et0 = dx, et1 = dy, et2 = dx * dx, et3 = dx * dy, et4 = dy * dy;
                    const float W = x0.z * qh.y * qh.y + x0.w * qh.z * qh.z + x1.x * qh.w * qh.w;
#pragma unroll
                    for (int k = 3; k < 10; ++k) {
                        const float ea = et2 * J[LJ::kCon + k] + et3 * J[LJ::kCon + 10 + k] + et4 * J[LJ::kCon + 20 + k];
                        D[k] = fmaf(W * ea, ea, D[k]);
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float ea = et0 * J[LJ::kMu + k] + et1 * J[LJ::kMu + 3 + k] + et2 * J[LJ::kCon + k] +
                                         et3 * J[LJ::kCon + 10 + k] + et4 * J[LJ::kCon + 20 + k];
                        if constexpr (DEG == 0) {
                            D[k] = fmaf(W * ea, ea, D[k]);
                        } else {
                            const float t0 = fmaf(qh.y, ea, qh.x * acol[0][k]);
                            const float t1 = fmaf(qh.z, ea, qh.x * acol[1][k]);
                            const float t2 = fmaf(qh.w, ea, qh.x * acol[2][k]);
                            D[k] = fmaf(x0.z * t0, t0, fmaf(x0.w * t1, t1, fmaf(x1.x * t2, t2, D[k])));
                        }
                    }
                    D[10] += W;
                    const float q2 = qh.x * qh.x;
                    D[11] = fmaf(x0.z, q2, D[11]);
                    D[12] = fmaf(x0.w, q2, D[12]);
                    D[13] = fmaf(x1.x, q2, D[13]);
                    if (kRhs) {
                        const float pb = x1.y * qh.y + x1.z * qh.z + x1.w * qh.w;
                        const float pdx = pb * dx, pdy = pb * dy;
                        M[0] += pdx;
                        M[1] += pdy;
                        M[2] = fmaf(pdx, dx, M[2]);
                        M[3] = fmaf(pdx, dy, M[3]);
                        M[4] = fmaf(pdy, dy, M[4]);
                        M[5] += pb;
                        M[6] = fmaf(x1.y, qh.x, M[6]);
                        M[7] = fmaf(x1.z, qh.x, M[7]);
                        M[8] = fmaf(x1.w, qh.x, M[8]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 14; ++k) D[k] += __shfl_xor_sync(kFull, D[k], 16);
            if (kRhs)
#pragma unroll
                for (int k = 0; k < 9; ++k) M[k] += __shfl_xor_sync(kFull, M[k], 16);
            if (hh == 0 && e < m) {
                const float4 r1 = sm.rec[j][1];
                const float om = 1.f - r1.y;
                unsigned id = sm.id[j];
                LMRS_DCHECK_INDEX(c, id, c.G, kCheckScatterId);
                float* dst = dbase + (long long)id * kDiagF;
                red_add_v4(dst, D[0], D[1], D[2], D[3]);
                red_add_v4(dst + 4, D[4], D[5], D[6], D[7]);
                red_add_v4(dst + 8, D[8], D[9], om * om * D[10], D[11]);
                red_add_v4(dst + 12, D[12], D[13], 0.f, 0.f);
                if (kRhs) {
                    float* cdst = cbase + (long long)id * kCotF;
                    red_add_v4(cdst, M[0], M[1], M[2], M[3]);
                    red_add_v4(cdst + 4, M[4], M[5], M[6], M[7]);
                    atomicAdd(cdst + 8, M[8]);
                }
            }
            __syncwarp();
        }
    }
}

// Full frames: one block per (slot, tile), one warp per 32 pixels.
__global__ void __launch_bounds__(256) k_full(Ctx c, float* images) {
    __shared__ float4 s_rec_all[8][32][kRecF4];
    __shared__ unsigned s_id_all[8][32];
    const int vt = blockIdx.x;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = vt / c.T, tile = vt - slot * c.T;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int vw = min(c.tile_w, c.W - tx * c.tile_w), vh = min(c.tile_h, c.H - ty * c.tile_h);
    const int nvalid = vw * vh;
    const int first = wid * 32;
    if (first >= nvalid) return;
    Pix p;
    p.vt = vt;
    p.slot = slot;
    p.tile = tile;
    p.chunk = 0;
    const int o = first + lane;
    p.active = o < nvalid;
    p.si = 0;
    p.px = tx * c.tile_w + (p.active ? o % vw : 0);
    p.py = ty * c.tile_h + (p.active ? o / vw : 0);
    p.pcx = p.px + 0.5f;
    p.pcy = p.py + 0.5f;
    p.npc = make_float2(-p.pcx, -p.pcy);
    p.w = 1.f;
    float C[3], T, dC[3];
    int ncons;
    forward_pass<false, false>(c, p, tile_list(c, p), s_rec_all[wid], s_id_all[wid], C, T, dC, ncons);
    if (p.active) {
        float* dst = images + (((long long)slot * c.H + p.py) * c.W + p.px) * 3;
        dst[0] = C[0];
        dst[1] = C[1];
        dst[2] = C[2];
    }
}

// Diagonal SSIM term at every sample (supplementary material: SSIM of
// Wang et al. 2004 with an 11 x 11 Gaussian window, sigma 1.5, out-of-image
// pixels counting as 0, C1 = 0.01^2, C2 = 0.03^2).  One warp per work item,
// one sample per lane, over the full frame and the target.  Two passes over
// the window: the means mx, my and dm = mean of X - Y, then the centred
// second moments vx, vy, cxy and vd = Var(X - Y), so nothing is formed as
// E[X^2] - mx^2.  With A1 = 2 mx my + C1, A2 = 2 cxy + C2, B1 = mx^2 + my^2 +
// C1, B2 = vx + vy + C2, D1 = dm^2 = B1 - A1 and D2 = vd = B2 - A2:
//   s = 1 - A1 A2 / (B1 B2) = (A1 D2 + B2 D1) / (B1 B2),
// a sum of non-negative terms.  The derivative through the pixel's own
// colour (g0 the centre weight: dA1 = 2 g0 my, dB1 = 2 g0 mx, dA2 =
// 2 g0 (Y_i - my), dB2 = 2 g0 (X_i - mx)) is d = -N / (B1 B2) with
//   N = dA1 A2 + A1 dA2 - (1 - s)(dB1 B2 + B1 dB2)
//     = (dA1 - dB1) A2 - dB1 D2 + A1 (dA2 - dB2) - D1 dB2 + s (dB1 B2 + B1 dB2),
// dA1 - dB1 = -2 g0 dm and dA2 - dB2 = -2 g0 ((X_i - Y_i) - dm) taken directly.
constexpr int kSsimRad = 5;

// s and d of one sample's three channels; returns sum_ch s^2.
__device__ float ssim_sample(const Ctx& c, const Pix& p) {
    // normalised 1D window; the 2D weights are the products g1[a] g1[b]
    float g1[2 * kSsimRad + 1], z = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kSsimRad; ++k) {
        const float t = (float)(k - kSsimRad);
        g1[k] = expf(-t * t * (1.f / 4.5f));
        z += g1[k];
    }
#pragma unroll
    for (int k = 0; k <= 2 * kSsimRad; ++k) g1[k] /= z;
    const int cam = c.views[p.slot];
    const float* X = c.frames + (long long)p.slot * c.H * c.W * 3;
    const float* Y = c.targets ? c.targets + (long long)cam * c.H * c.W * 3 : nullptr;
    float mx[3] = {0.f, 0.f, 0.f}, my[3] = {0.f, 0.f, 0.f}, dm[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a <= 2 * kSsimRad; ++a) {
        const int y = p.py + a - kSsimRad;
        if (y < 0 || y >= c.H) continue;
        float rx[3] = {0.f, 0.f, 0.f}, ry[3] = {0.f, 0.f, 0.f}, rd[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b <= 2 * kSsimRad; ++b) {
            const int x = p.px + b - kSsimRad;
            if (x < 0 || x >= c.W) continue;
            const long long o = ((long long)y * c.W + x) * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float xv = X[o + ch], yv = Y ? Y[o + ch] : 0.f;
                rx[ch] = fmaf(g1[b], xv, rx[ch]);
                ry[ch] = fmaf(g1[b], yv, ry[ch]);
                rd[ch] = fmaf(g1[b], xv - yv, rd[ch]);
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            mx[ch] = fmaf(g1[a], rx[ch], mx[ch]);
            my[ch] = fmaf(g1[a], ry[ch], my[ch]);
            dm[ch] = fmaf(g1[a], rd[ch], dm[ch]);
        }
    }
    float vx[3] = {0.f, 0.f, 0.f}, vy[3] = {0.f, 0.f, 0.f}, cxy[3] = {0.f, 0.f, 0.f}, vd[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a <= 2 * kSsimRad; ++a) {
        const int y = p.py + a - kSsimRad;
        const bool yin = y >= 0 && y < c.H;
        float rx[3] = {0.f, 0.f, 0.f}, ry[3] = {0.f, 0.f, 0.f}, rc[3] = {0.f, 0.f, 0.f}, rd[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b <= 2 * kSsimRad; ++b) {
            const int x = p.px + b - kSsimRad;
            const bool in = yin && x >= 0 && x < c.W;
            const long long o = ((long long)y * c.W + x) * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float xv = in ? X[o + ch] : 0.f;
                const float yv = (in && Y) ? Y[o + ch] : 0.f;
                const float ex = xv - mx[ch], ey = yv - my[ch], ed = (xv - yv) - dm[ch];
                rx[ch] = fmaf(g1[b] * ex, ex, rx[ch]);
                ry[ch] = fmaf(g1[b] * ey, ey, ry[ch]);
                rc[ch] = fmaf(g1[b] * ex, ey, rc[ch]);
                rd[ch] = fmaf(g1[b] * ed, ed, rd[ch]);
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            vx[ch] = fmaf(g1[a], rx[ch], vx[ch]);
            vy[ch] = fmaf(g1[a], ry[ch], vy[ch]);
            cxy[ch] = fmaf(g1[a], rc[ch], cxy[ch]);
            vd[ch] = fmaf(g1[a], rd[ch], vd[ch]);
        }
    }
    constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const float g0 = g1[kSsimRad] * g1[kSsimRad];
    const long long pix = ((long long)p.py * c.W + p.px) * 3;
    float sq = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float xi = X[pix + ch], yi = Y ? Y[pix + ch] : 0.f;
        const float A1 = 2.f * mx[ch] * my[ch] + C1, A2 = 2.f * cxy[ch] + C2;
        const float B1 = mx[ch] * mx[ch] + my[ch] * my[ch] + C1, B2 = vx[ch] + vy[ch] + C2;
        const float D1 = dm[ch] * dm[ch], D2 = vd[ch];
        const float BB = B1 * B2;
        const float sv = (A1 * D2 + B2 * D1) / BB;
        const float dB1 = 2.f * g0 * mx[ch], dB2 = 2.f * g0 * (xi - mx[ch]);
        const float dA1mB1 = -2.f * g0 * dm[ch], dA2mB2 = -2.f * g0 * ((xi - yi) - dm[ch]);
        const float N = dA1mB1 * A2 - dB1 * D2 + A1 * dA2mB2 - D1 * dB2 + sv * (dB1 * B2 + B1 * dB2);
        c.ssim_s[3 * p.si + ch] = sv;
        c.ssim_d[3 * p.si + ch] = -N / BB;
        sq = fmaf(sv, sv, sq);
    }
    return sq;
}

__global__ void __launch_bounds__(kRasterBlock) k_ssim(Ctx c) {
    const int wid = threadIdx.x >> 5;
    const int item = blockIdx.x * kRasterWarps + wid;
    if (item >= c.nwork) return;
    Pix p;
    setup_item(c, item, p);
    // the term's share of the sampled loss: ssim_weight * w * sum_ch s^2
    double part = p.active ? (double)c.ssim_weight * (double)p.w * (double)ssim_sample(c, p) : 0.0;
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) atomicAdd(&c.sc->loss_num, part);
}

void launch_ssim(const Ctx& c, cudaStream_t st) {
    if (c.nwork > 0) LMRS_LAUNCH(k_ssim, (unsigned)((c.nwork + kRasterWarps - 1) / kRasterWarps), kRasterBlock, 0, st, c);
}

// Importance draws of the pixel sampler (modes 1, 2), one block per (view,
// tile): every valid pixel is rendered and weighted -- e^{|r_p|}, |r_p| the
// Euclidean norm of its RGB residual, or the number of Gaussians it
// composites --, the weights are prefix-summed in FP64 in pixel order, and
// draw i takes the first pixel whose cumulative weight exceeds u_i x total,
// u_i = (output i of the tile's SplitMix64 stream >> 11) 2^-53; its weight
// is total / (K_t x the pixel's weight) = 1 / (K_t q).  A tile whose total is
// 0 is drawn uniformly with weight n_valid / K_t.
__global__ void __launch_bounds__(256) k_importance(Ctx c, long long lm_step, unsigned long long seed) {
    __shared__ float4 s_rec_all[8][32][kRecF4];
    __shared__ unsigned s_id_all[8][32];
    __shared__ double s_cdf[256];
    __shared__ float s_a[256];
    const int vt = blockIdx.x;
    const int wid = threadIdx.x >> 5, o = threadIdx.x;
    const int slot = vt / c.T, tile = vt - slot * c.T;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int vw = min(c.tile_w, c.W - tx * c.tile_w), vh = min(c.tile_h, c.H - ty * c.tile_h);
    const int nvalid = vw * vh;
    const int cam = c.views[slot];
    float a = 0.f;
    if (wid * 32 < nvalid) {
        Pix p;
        p.vt = vt;
        p.slot = slot;
        p.tile = tile;
        p.chunk = 0;
        p.active = o < nvalid;
        p.si = 0;
        p.px = tx * c.tile_w + (p.active ? o % vw : 0);
        p.py = ty * c.tile_h + (p.active ? o / vw : 0);
        p.pcx = p.px + 0.5f;
        p.pcy = p.py + 0.5f;
        p.npc = make_float2(-p.pcx, -p.pcy);
        p.w = 1.f;
        float C[3], T, dC[3];
        int ncons, ncomp = 0;
        forward_pass<false, false>(c, p, tile_list(c, p), s_rec_all[wid], s_id_all[wid], C, T, dC, ncons, nullptr,
                                   nullptr, &ncomp);
        if (p.active) {
            if (c.sample_dist == 1) {
                float r2 = 0.f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float tg = c.targets ? c.targets[(((long long)cam * c.H + p.py) * c.W + p.px) * 3 + ch] : 0.f;
                    const float d = C[ch] - tg;
                    r2 += d * d;
                }
                a = expf(sqrtf(r2));
            } else {
                a = (float)ncomp;
            }
        }
    }
    s_a[o] = a;
    s_cdf[o] = (double)a;
    __syncthreads();
    for (int d = 1; d < 256; d <<= 1) {
        const double v = o >= d ? s_cdf[o - d] : 0.0;
        __syncthreads();
        s_cdf[o] += v;
        __syncthreads();
    }
    const double total = s_cdf[nvalid - 1];
    const int b = c.tile_off[vt], K = c.tile_off[vt + 1] - b;
    if (o < K) {
        const unsigned long long r =
            sm64_mix(tile_stream(seed, lm_step, cam, tile) + (unsigned long long)(o + 1) * kSm64Gamma);
        const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
        int sel;
        float w;
        if (!(total > 0.0)) {
            sel = min(nvalid - 1, (int)floor(u * nvalid));
            w = (float)nvalid / (float)K;
        } else {
            const double thr = u * total;
            int lo = 0, hi = nvalid - 1;  // the first index whose cumulative weight exceeds thr
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_cdf[mid] > thr) hi = mid;
                else lo = mid + 1;
            }
            sel = lo;
            w = (float)(total / ((double)K * (double)s_a[sel]));
        }
        c.off[b + o] = (unsigned char)sel;
        c.wsample[b + o] = w;
    }
}

void launch_importance(const Ctx& c, long long lm_step, unsigned long long seed, cudaStream_t st) {
    LMRS_LAUNCH(k_importance, (unsigned)(c.nv * c.T), 256, 0, st, c, lm_step, seed);
}

static unsigned raster_grid(const Ctx& c) { return (unsigned)((c.nwork + kRasterWarps - 1) / kRasterWarps); }

// Longest-first order of the work items (load balance only): 16-bit keys,
// ascending key = descending cost; items of 65,535 or more list entries tie
// and keep their index order.
constexpr int kOrderBits = 16;

__global__ void k_order_keys(const int* cost, int n, unsigned long long* keys, unsigned int* vals) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const unsigned cmax = (1u << kOrderBits) - 1u;
    keys[k] = cmax - min((unsigned)max(cost[k], 0), cmax);
    vals[k] = (unsigned int)k;
}

__global__ void k_gather_work(const int2* work, const unsigned int* order, int n, int2* sorted) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) sorted[k] = work[order[k]];
}

void launch_order_work(const Ctx& c, unsigned long long* keys, unsigned int* vals, unsigned long long* keys_alt,
                       unsigned int* vals_alt, void* tmp, size_t tmp_bytes, int2* sorted, cudaStream_t st) {
    if (c.nwork <= 0) return;
    const unsigned grid = (unsigned)((c.nwork + 255) / 256);
    LMRS_LAUNCH(k_order_keys, grid, 256, 0, st, c.item_cost, c.nwork, keys, vals);
    radix_sort(keys, vals, keys_alt, vals_alt, c.nwork, kOrderBits, tmp, tmp_bytes, st);
    LMRS_LAUNCH(k_gather_work, grid, 256, 0, st, c.work, vals, c.nwork, sorted);
}

void launch_raster_fwd_samples(const Ctx& c, cudaStream_t st) {
    if (c.nwork > 0) LMRS_LAUNCH(k_fwd_samples, raster_grid(c), kRasterBlock, 0, st, c);
}
// Sum over the preprocessed views of |frame - target|^2 (full frames, slot
// order), added into *out in FP64.
__global__ void __launch_bounds__(256) k_frame_sqerr(Ctx c, const float* frames, double* out) {
    const long long per = (long long)c.H * c.W * 3;
    const long long n = (long long)c.nv * per;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(i / per);
        const float d = frames[i] - c.targets[(long long)c.views[slot] * per + (i - (long long)slot * per)];
        acc += (double)(d * d);
    }
    acc = block_sum<256>(acc);
    if (threadIdx.x == 0) atomicAdd(out, acc);
}

void launch_frame_sqerr(const Ctx& c, const float* frames, double* out, cudaStream_t st) {
    LMRS_LAUNCH(k_frame_sqerr, 152 * 8, 256, 0, st, c, frames, out);
}

void launch_raster_full(const Ctx& c, float* images, cudaStream_t st) {
    LMRS_LAUNCH(k_full, (unsigned)(c.nv * c.T), 256, 0, st, c, images);
}
void launch_raster_jvp(const Ctx& c, float* u, cudaStream_t st) {
    if (c.nwork > 0) LMRS_LAUNCH(k_jvp, raster_grid(c), kRasterBlock, 0, st, c, u);
}
void launch_raster_vjp(const Ctx& c, const float* u, cudaStream_t st) {
    if (c.nwork > 0) LMRS_LAUNCH(k_vjp, raster_grid(c), kRasterBlock, 0, st, c, u);
}
void launch_raster_jtj(const Ctx& c, cudaStream_t st) {
    if (c.nwork > 0) LMRS_LAUNCH(k_jtj, raster_grid(c), kRasterBlock, 0, st, c);
}
template <bool kRhs>
static void diag_deg(const Ctx& c, cudaStream_t st) {
    const unsigned grid = raster_grid(c);
    const char* name = kRhs ? "k_diag<rhs>" : "k_diag";
    switch (c.deg) {
        case 0: LMRS_LAUNCH_AS(name, (k_diag<0, kRhs>), grid, kRasterBlock, 0, st, c); break;
        case 1: LMRS_LAUNCH_AS(name, (k_diag<1, kRhs>), grid, kRasterBlock, 0, st, c); break;
        case 2: LMRS_LAUNCH_AS(name, (k_diag<2, kRhs>), grid, kRasterBlock, 0, st, c); break;
        default: LMRS_LAUNCH_AS(name, (k_diag<3, kRhs>), grid, kRasterBlock, 0, st, c); break;
    }
}
void launch_raster_diag(const Ctx& c, cudaStream_t st) {
    if (c.nwork > 0) diag_deg<false>(c, st);
}
void launch_raster_diag_rhs(const Ctx& c, cudaStream_t st) {
    if (c.nwork > 0) diag_deg<true>(c, st);
}

}  // namespace lmrs
