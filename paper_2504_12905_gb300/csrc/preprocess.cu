// Per-(view, Gaussian) preprocessing of the LM-RS hot path.
//
//   k_sample        per-tile stratified pixel sampling (Sec. 4.4)
//   k_prep_gauss    view-independent 3D state per Gaussian (scale, normalised
//                   quaternion, R, M = R S, Sigma = M M^T, opacity), once per
//                   LM step (Sec. 3, Eq. 3)
//   k_prep_fwd      projection (Sec. 3, Eqs. 2-4): list decisions in FP32 with
//                   a fixed operation order, 2D features, and the per-pair
//                   Jacobian of the 9 features w.r.t. the Gaussian's
//                   parameters (forward mode on unit tangents, Alg. 3)
//   k_prep_jvp      tangents of the 2D features from the Jacobian cache (the
//                   "preprocessing" half of the Jv kernel, App. A)
//   k_prep_vjp      the transposed map from the per-pair 2D cotangents to the
//                   3D parameters (second launch of the J^T v kernel, App. A),
//                   plus the damping of Eq. 8 and p^T A p in FP64
//   k_prep_diag     diag(J^T W J): the per-pair row sums of k_diag summed over
//                   the views (App. A "Diag")
// Kernels are instantiated per SH degree (0..3) so coefficient arrays live
// in registers.
#include <cmath>

#include "common.cuh"
#include "jac.cuh"
#include "reduce.cuh"

namespace lmrs {

// Real SH normalisation constants (degree <= 3), computed on the host from
// K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for m != 0.
__constant__ float c_sh[10];

void set_sh_constants() {
    const double pi = 3.14159265358979323846;
    float h[10] = {
        (float)std::sqrt(1.0 / (4.0 * pi)),     // 0: l=0
        (float)std::sqrt(3.0 / (4.0 * pi)),     // 1: l=1
        (float)std::sqrt(15.0 / (4.0 * pi)),    // 2: xy, yz, xz
        (float)std::sqrt(5.0 / (16.0 * pi)),    // 3: 3z^2 - 1
        (float)std::sqrt(15.0 / (16.0 * pi)),   // 4: x^2 - y^2
        (float)std::sqrt(35.0 / (32.0 * pi)),   // 5: l=3, |m|=3
        (float)std::sqrt(105.0 / (4.0 * pi)),   // 6: xyz
        (float)std::sqrt(21.0 / (32.0 * pi)),   // 7: l=3, |m|=1
        (float)std::sqrt(7.0 / (16.0 * pi)),    // 8: l=3, m=0
        (float)std::sqrt(105.0 / (16.0 * pi)),  // 9: z (x^2 - y^2)
    };
    cudaMemcpyToSymbol(c_sh, h, sizeof(h));
}

// Basis values, index l^2 + l + m.
template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
    Y[0] = c_sh[0];
    if (DEG < 1) return;
    Y[1] = c_sh[1] * y;
    Y[2] = c_sh[1] * z;
    Y[3] = c_sh[1] * x;
    if (DEG < 2) return;
    Y[4] = c_sh[2] * x * y;
    Y[5] = c_sh[2] * y * z;
    Y[6] = c_sh[3] * (3.f * z * z - 1.f);
    Y[7] = c_sh[2] * x * z;
    Y[8] = c_sh[4] * (x * x - y * y);
    if (DEG < 3) return;
    Y[9] = c_sh[5] * y * (3.f * x * x - y * y);
    Y[10] = c_sh[6] * x * y * z;
    Y[11] = c_sh[7] * y * (5.f * z * z - 1.f);
    Y[12] = c_sh[8] * z * (5.f * z * z - 3.f);
    Y[13] = c_sh[7] * x * (5.f * z * z - 1.f);
    Y[14] = c_sh[9] * z * (x * x - y * y);
    Y[15] = c_sh[5] * x * (x * x - 3.f * y * y);
}

// gY[k] = grad Y_k(x, y, z) . d  (directional derivative of each basis function).
template <int DEG>
__device__ __forceinline__ void sh_dir_deriv(float x, float y, float z, const float d[3], float* gY) {
    gY[0] = 0.f;
    if (DEG < 1) return;
    const float k1 = c_sh[1];
    gY[1] = k1 * d[1];
    gY[2] = k1 * d[2];
    gY[3] = k1 * d[0];
    if (DEG < 2) return;
    const float k2 = c_sh[2], k20 = c_sh[3], k22 = c_sh[4];
    gY[4] = k2 * (d[0] * y + x * d[1]);
    gY[5] = k2 * (d[1] * z + y * d[2]);
    gY[6] = 6.f * k20 * z * d[2];
    gY[7] = k2 * (d[0] * z + x * d[2]);
    gY[8] = 2.f * k22 * (x * d[0] - y * d[1]);
    if (DEG < 3) return;
    const float k33 = c_sh[5], k32a = c_sh[6], k31 = c_sh[7], k30 = c_sh[8], k32 = c_sh[9];
    gY[9] = k33 * (6.f * x * y * d[0] + 3.f * (x * x - y * y) * d[1]);
    gY[10] = k32a * (y * z * d[0] + x * z * d[1] + x * y * d[2]);
    gY[11] = k31 * ((5.f * z * z - 1.f) * d[1] + 10.f * y * z * d[2]);
    gY[12] = k30 * (15.f * z * z - 3.f) * d[2];
    gY[13] = k31 * ((5.f * z * z - 1.f) * d[0] + 10.f * x * z * d[2]);
    gY[14] = k32 * (2.f * x * z * d[0] - 2.f * y * z * d[1] + (x * x - y * y) * d[2]);
    gY[15] = k33 * (3.f * (x * x - y * y) * d[0] - 6.f * x * y * d[1]);
}

// ---------------------------------------------------------------------------
// Primal quantities.
// ---------------------------------------------------------------------------
struct Prim {
    // per Gaussian (cache)
    float s[3], qn, qh[4];
    float R[9], M[9], S[9];
    float o;
    float tau;  // level of the alpha >= 1/255 ellipse (row_span)
    bool valid;
    // per (view, Gaussian)
    float t[3];
    float ux, uy;
    bool clx, cly;
    float j00, j02, j11, j12;
    float T[6], V[6];
    float a, b, c, det;
    float mux, muy;
    float A, B, C;
    float dir[3], dn;
    float col[3];
    bool clamped[3];
};

__device__ __forceinline__ float rm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ra(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rd(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ void load_mean(const float* p, int g, float X[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) X[k] = p[3ll * g + k];
}

// View-independent 3D state in the fixed FP32 operation order of the list
// decisions: s = binary32(exp_fp64(log-scale)), q / |q|, R(q), M = R S,
// Sigma = M M^T; every operation rounded on its own.
__global__ void k_prep_gauss(Ctx c) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= c.G) return;
    const float* p = c.params;
    const long long G = c.G;
    float s[3], q[4];
#pragma unroll
    for (int j = 0; j < 3; ++j) s[j] = (float)exp((double)p[3 * G + 3ll * g + j]);
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = p[6 * G + 4ll * g + k];
    const float qq = ra(ra(ra(rm(q[0], q[0]), rm(q[1], q[1])), rm(q[2], q[2])), rm(q[3], q[3]));
    const bool valid = qq > 0.f;
    const float qn = valid ? __fsqrt_rn(qq) : 1.f;
    const float w = rd(q[0], qn), x = rd(q[1], qn), y = rd(q[2], qn), z = rd(q[3], qn);
    float r[9];
    r[0] = rs(1.f, rm(2.f, ra(rm(y, y), rm(z, z))));
    r[1] = rm(2.f, rs(rm(x, y), rm(w, z)));
    r[2] = rm(2.f, ra(rm(x, z), rm(w, y)));
    r[3] = rm(2.f, ra(rm(x, y), rm(w, z)));
    r[4] = rs(1.f, rm(2.f, ra(rm(x, x), rm(z, z))));
    r[5] = rm(2.f, rs(rm(y, z), rm(w, x)));
    r[6] = rm(2.f, rs(rm(x, z), rm(w, y)));
    r[7] = rm(2.f, ra(rm(y, z), rm(w, x)));
    r[8] = rs(1.f, rm(2.f, ra(rm(x, x), rm(y, y))));
    float m[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m[3 * i + j] = rm(r[3 * i + j], s[j]);
    float S[6];  // S00 S01 S02 S11 S12 S22
    int k = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            S[k++] = ra(ra(rm(m[3 * i], m[3 * j]), rm(m[3 * i + 1], m[3 * j + 1])), rm(m[3 * i + 2], m[3 * j + 2]));
    const float o = 1.f / (1.f + expf(-p[10 * G + g]));
    // alpha = o exp(-q / 2) >= 1/255 iff q <= 2 ln(255 o); with a slack of
    // 0.02, in double, rounded once
    const double od = 1.0 / (1.0 + exp(-(double)p[10 * G + g]));
    const float tau = (float)__dadd_rn(__dmul_rn(2.0, log(255.0 * od)), 0.02);
    float4* gc = c.gcache;
    gc[0 * G + g] = make_float4(s[0], s[1], s[2], qn);
    gc[1 * G + g] = make_float4(w, x, y, z);
    gc[2 * G + g] = make_float4(r[0], r[1], r[2], r[3]);
    gc[3 * G + g] = make_float4(r[4], r[5], r[6], r[7]);
    gc[4 * G + g] = make_float4(r[8], m[0], m[1], m[2]);
    gc[5 * G + g] = make_float4(m[3], m[4], m[5], m[6]);
    gc[6 * G + g] = make_float4(m[7], m[8], S[0], S[1]);
    gc[7 * G + g] = make_float4(S[2], S[3], S[4], S[5]);
    gc[8 * G + g] = make_float4(o, valid ? 1.f : 0.f, tau, 0.f);
}

__device__ __forceinline__ void load_gauss(const Ctx& c, int g, Prim& P) {
    const long long G = c.G;
    const float4* gc = c.gcache;
    float4 v = gc[0 * G + g];
    P.s[0] = v.x; P.s[1] = v.y; P.s[2] = v.z; P.qn = v.w;
    v = gc[1 * G + g];
    P.qh[0] = v.x; P.qh[1] = v.y; P.qh[2] = v.z; P.qh[3] = v.w;
    v = gc[2 * G + g];
    P.R[0] = v.x; P.R[1] = v.y; P.R[2] = v.z; P.R[3] = v.w;
    v = gc[3 * G + g];
    P.R[4] = v.x; P.R[5] = v.y; P.R[6] = v.z; P.R[7] = v.w;
    v = gc[4 * G + g];
    P.R[8] = v.x; P.M[0] = v.y; P.M[1] = v.z; P.M[2] = v.w;
    v = gc[5 * G + g];
    P.M[3] = v.x; P.M[4] = v.y; P.M[5] = v.z; P.M[6] = v.w;
    v = gc[6 * G + g];
    P.M[7] = v.x; P.M[8] = v.y; P.S[0] = v.z; P.S[1] = v.w;
    v = gc[7 * G + g];
    P.S[2] = v.x; P.S[4] = v.y; P.S[5] = v.z; P.S[8] = v.w;
    P.S[3] = P.S[1]; P.S[6] = P.S[2]; P.S[7] = P.S[5];
    v = gc[8 * G + g];
    P.o = v.x;
    P.valid = v.y != 0.f;
    P.tau = v.z;
}

// Per-(view, Gaussian) projection with the list decisions, continuing the
// fixed FP32 operation order of k_prep_gauss (so visibility, depth key, tile
// rectangle and the ellipse that picks each row's tiles are reproducible bit
// for bit).  Returns false when culled.
__device__ __forceinline__ bool prim_project(const float X[3], const CamDev& cam, int tiles_x, int tiles_y, int tw,
                                             int th, Prim& P, int4* rect_out, float* depth_out,
                                             float4* ell_out = nullptr) {
    const float* R = cam.R;
    P.t[0] = ra(ra(ra(rm(R[0], X[0]), rm(R[1], X[1])), rm(R[2], X[2])), cam.t[0]);
    P.t[1] = ra(ra(ra(rm(R[3], X[0]), rm(R[4], X[1])), rm(R[5], X[2])), cam.t[1]);
    P.t[2] = ra(ra(ra(rm(R[6], X[0]), rm(R[7], X[1])), rm(R[8], X[2])), cam.t[2]);
    if (!(P.t[2] > cam.znear)) return false;
    if (!P.valid) return false;
    P.ux = rd(P.t[0], P.t[2]);
    P.uy = rd(P.t[1], P.t[2]);
    const float cux = fminf(fmaxf(P.ux, -cam.limx), cam.limx);
    const float cuy = fminf(fmaxf(P.uy, -cam.limy), cam.limy);
    P.clx = cux != P.ux;
    P.cly = cuy != P.uy;
    P.j00 = rd(cam.fx, P.t[2]);
    P.j02 = -rd(rm(cam.fx, cux), P.t[2]);
    P.j11 = rd(cam.fy, P.t[2]);
    P.j12 = -rd(rm(cam.fy, cuy), P.t[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P.T[k] = ra(rm(P.j00, R[k]), rm(P.j02, R[6 + k]));
        P.T[3 + k] = ra(rm(P.j11, R[3 + k]), rm(P.j12, R[6 + k]));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            P.V[3 * i + k] = ra(ra(rm(P.T[3 * i], P.S[k]), rm(P.T[3 * i + 1], P.S[3 + k])), rm(P.T[3 * i + 2], P.S[6 + k]));
    P.a = ra(ra(ra(rm(P.V[0], P.T[0]), rm(P.V[1], P.T[1])), rm(P.V[2], P.T[2])), 0.3f);
    P.b = ra(ra(rm(P.V[0], P.T[3]), rm(P.V[1], P.T[4])), rm(P.V[2], P.T[5]));
    P.c = ra(ra(ra(rm(P.V[3], P.T[3]), rm(P.V[4], P.T[4])), rm(P.V[5], P.T[5])), 0.3f);
    P.det = rs(rm(P.a, P.c), rm(P.b, P.b));
    if (!(P.det > 0.f)) return false;
    P.mux = ra(rm(cam.fx, P.ux), cam.cx);
    P.muy = ra(rm(cam.fy, P.uy), cam.cy);
    if (rect_out) {
        const float mid = rm(0.5f, ra(P.a, P.c));
        const float disc = fmaxf(rs(rm(mid, mid), P.det), 0.1f);
        const float lam = ra(mid, __fsqrt_rn(disc));
        const float rad = ceilf(rm(3.0f, __fsqrt_rn(lam)));
        const float fx0 = floorf(rd(rs(P.mux, rad), (float)tw));
        const float fx1 = floorf(rd(ra(P.mux, rad), (float)tw));
        const float fy0 = floorf(rd(rs(P.muy, rad), (float)th));
        const float fy1 = floorf(rd(ra(P.muy, rad), (float)th));
        if (fx1 < 0.f || fx0 > (float)(tiles_x - 1) || fy1 < 0.f || fy0 > (float)(tiles_y - 1)) return false;
        rect_out->x = (int)fmaxf(fx0, 0.f);
        rect_out->y = (int)fminf(fx1, (float)(tiles_x - 1));
        rect_out->z = (int)fmaxf(fy0, 0.f);
        rect_out->w = (int)fminf(fy1, (float)(tiles_y - 1));
        *depth_out = P.t[2];
        if (ell_out) {
            // (dx - kx dy)^2 <= pq - qq dy^2 with kx = b / c, pq = (det / c) tau,
            // qq = det / c^2; |dy| <= sqrt(tau c); extreme points at dy = +-b sqrt(tau / a)
            float kx = 0.f, dys = 0.f, pq = 0.f, qq = 0.f, ey = -1.f;
            if (P.tau > 0.f) {
                const float sv = rd(P.det, P.c);
                kx = rd(P.b, P.c);
                pq = rm(sv, P.tau);
                qq = rd(sv, P.c);
                ey = __fsqrt_rn(rm(P.tau, P.c));
                dys = rm(P.b, __fsqrt_rn(rd(P.tau, P.a)));
            }
            ell_out[0] = make_float4(P.mux, P.muy, kx, dys);
            ell_out[1] = make_float4(pq, qq, ey, 0.f);
        }
    }
    return true;
}

// 2D conic and view-dependent colour.
template <int DEG>
__device__ __forceinline__ void prim_features(const float X[3], const float* sh, const CamDev& cam, Prim& P) {
    const float inv = 1.f / P.det;
    P.A = P.c * inv;
    P.B = -P.b * inv;
    P.C = P.a * inv;
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = X[k] - cam.centre[k];
    P.dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float idn = 1.f / P.dn;
#pragma unroll
    for (int k = 0; k < 3; ++k) P.dir[k] = d[k] * idn;
    constexpr int K = Sh<DEG>::K;
    float Y[K];
    sh_eval<DEG>(P.dir[0], P.dir[1], P.dir[2], Y);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc += sh[3 * k + ch] * Y[k];
        P.clamped[ch] = acc < 0.f;
        P.col[ch] = P.clamped[ch] ? 0.f : acc;
    }
}

// ---------------------------------------------------------------------------
// Forward-mode tangent of the features (mu_x, mu_y, A, B, C) and of the colour
// through the view direction, along a tangent with one non-zero parameter
// group: kTanMean (dX), kTanScale (d log-scale) or kTanRot (dq), as the
// Jacobian cache's columns need.  The terms the other groups would add are
// exactly zero and are not formed (IEEE arithmetic cannot drop a product with
// a zero factor by itself).  out[5] (opacity) is 0; the colour out[6..8] is
// formed for the mean group only (the other columns do not move it).
// ---------------------------------------------------------------------------
struct GTan {
    float X[3], ls[3], q[4], th;
};

constexpr int kTanMean = 1, kTanScale = 2, kTanRot = 4;

template <int DEG, int kGroup>
__device__ __forceinline__ void prim_tangent(const Prim& P, const CamDev& cam, const GTan& d, const float* sh,
                                             float out[9]) {
    constexpr bool kX = kGroup == kTanMean, kS = kGroup == kTanScale, kQ = kGroup == kTanRot;
    static_assert(kX || kS || kQ, "one parameter group");
    const float* W = cam.R;
    const float* V = P.V;
    const float* T = P.T;
    float da, db, dc, dux = 0.f, duy = 0.f;
    if constexpr (kX) {
        float dt[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) dt[k] = W[3 * k] * d.X[0] + W[3 * k + 1] * d.X[1] + W[3 * k + 2] * d.X[2];
        const float it2 = 1.f / P.t[2];
        dux = (dt[0] - P.ux * dt[2]) * it2;
        duy = (dt[1] - P.uy * dt[2]) * it2;
        const float dcux = P.clx ? 0.f : dux, dcuy = P.cly ? 0.f : duy;
        const float dj00 = -P.j00 * dt[2] * it2;
        const float dj02 = -cam.fx * dcux * it2 - P.j02 * dt[2] * it2;
        const float dj11 = -P.j11 * dt[2] * it2;
        const float dj12 = -cam.fy * dcuy * it2 - P.j12 * dt[2] * it2;
        float dT[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dT[k] = dj00 * W[k] + dj02 * W[6 + k];
            dT[3 + k] = dj11 * W[3 + k] + dj12 * W[6 + k];
        }
        // d(T Sigma T^T) = dT V^T + V dT^T  with V = T Sigma
        da = 2.f * (dT[0] * V[0] + dT[1] * V[1] + dT[2] * V[2]);
        db = dT[0] * V[3] + dT[1] * V[4] + dT[2] * V[5] + V[0] * dT[3] + V[1] * dT[4] + V[2] * dT[5];
        dc = 2.f * (dT[3] * V[3] + dT[4] * V[4] + dT[5] * V[5]);
    } else {
        // dM = d(R S): R dS with dS = S d log-scale, or dR S with dR from the
        // normalised quaternion's tangent dqh = (dq - qh (qh . dq)) / |q|
        float dM[9];
        if constexpr (kS) {
            float ds[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) ds[j] = P.s[j] * d.ls[j];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) dM[3 * i + j] = P.R[3 * i + j] * ds[j];
        } else {
            const float* qh = P.qh;
            const float proj = qh[0] * d.q[0] + qh[1] * d.q[1] + qh[2] * d.q[2] + qh[3] * d.q[3];
            const float iqn = 1.f / P.qn;
            const float dw = (d.q[0] - qh[0] * proj) * iqn, dx = (d.q[1] - qh[1] * proj) * iqn;
            const float dy = (d.q[2] - qh[2] * proj) * iqn, dz = (d.q[3] - qh[3] * proj) * iqn;
            const float w = qh[0], x = qh[1], y = qh[2], z = qh[3];
            float dR[9];
            dR[0] = -4.f * (y * dy + z * dz);
            dR[1] = 2.f * (dx * y + x * dy - dw * z - w * dz);
            dR[2] = 2.f * (dx * z + x * dz + dw * y + w * dy);
            dR[3] = 2.f * (dx * y + x * dy + dw * z + w * dz);
            dR[4] = -4.f * (x * dx + z * dz);
            dR[5] = 2.f * (dy * z + y * dz - dw * x - w * dx);
            dR[6] = 2.f * (dx * z + x * dz - dw * y - w * dy);
            dR[7] = 2.f * (dy * z + y * dz + dw * x + w * dx);
            dR[8] = -4.f * (x * dx + y * dy);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) dM[3 * i + j] = dR[3 * i + j] * P.s[j];
        }
        // dSigma = dM M^T + M dM^T
        float dS[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float v = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) v += dM[3 * i + k] * P.M[3 * j + k] + P.M[3 * i + k] * dM[3 * j + k];
                dS[3 * i + j] = v;
            }
        // d(T Sigma T^T) = T dSigma T^T
        float TdS[6];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                TdS[3 * i + k] = T[3 * i] * dS[k] + T[3 * i + 1] * dS[3 + k] + T[3 * i + 2] * dS[6 + k];
        da = TdS[0] * T[0] + TdS[1] * T[1] + TdS[2] * T[2];
        db = TdS[0] * T[3] + TdS[1] * T[4] + TdS[2] * T[5];
        dc = TdS[3] * T[3] + TdS[4] * T[4] + TdS[5] * T[5];
    }
    const float ddet = da * P.c + P.a * dc - 2.f * P.b * db;
    const float idet = 1.f / P.det;
    out[0] = cam.fx * dux;
    out[1] = cam.fy * duy;
    out[2] = (dc - P.A * ddet) * idet;
    out[3] = (-db - P.B * ddet) * idet;
    out[4] = (da - P.C * ddet) * idet;
    out[5] = 0.f;
    // colour through the view direction (mean group only):
    // dc_ch = sum_k sh_k,ch (grad Y_k . ddir), coefficients streamed from memory
    constexpr int K = Sh<DEG>::K;
    float v3[3] = {0.f, 0.f, 0.f};
    if constexpr (DEG > 0 && kX) {
        const float idn = 1.f / P.dn;
        const float pd = P.dir[0] * d.X[0] + P.dir[1] * d.X[1] + P.dir[2] * d.X[2];
        float ddir[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) ddir[k] = (d.X[k] - P.dir[k] * pd) * idn;
        float gY[K];
        sh_dir_deriv<DEG>(P.dir[0], P.dir[1], P.dir[2], ddir, gY);
#pragma unroll
        for (int k = 1; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) v3[ch] += sh[3 * k + ch] * gY[k];
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) out[6 + ch] = P.clamped[ch] ? 0.f : v3[ch];
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
__global__ void k_sample(Ctx c, long long lm_step, unsigned long long seed) {
    const int vt = blockIdx.x * blockDim.x + threadIdx.x;
    if (vt >= c.nv * c.T) return;
    const int slot = vt / c.T, tile = vt % c.T;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int vw = min(c.tile_w, c.W - tx * c.tile_w), vh = min(c.tile_h, c.H - ty * c.tile_h);
    const int n = vw * vh;
    const int b = c.tile_off[vt], k = c.tile_off[vt + 1] - b;
    unsigned char a[256];
    for (int i = 0; i < n; ++i) a[i] = (unsigned char)i;
    unsigned long long h = tile_stream(seed, lm_step, c.views[slot], tile);
    for (int i = 0; i < k; ++i) {
        h += kSm64Gamma;
        const unsigned long long r = sm64_mix(h);
        const int j = i + (int)(r % (unsigned long long)(n - i));
        const unsigned char t = a[i];
        a[i] = a[j];
        a[j] = t;
        c.off[b + i] = a[i];
    }
}

// ---------------------------------------------------------------------------
// Per-pair Jacobian cache (layout in jac.cuh), formed from the verified
// tangent code on unit tangents: column j is the tangent of the mean, conic,
// opacity and colour along geometric parameter j, turned into the tangents
// of the exponent's coefficients e_1..e_5 with the pair's conic.
// ---------------------------------------------------------------------------
template <int DEG>
__device__ __forceinline__ void pair_jacobian(const Prim& P, const CamDev& cam, const float* sh, float* J) {
    using L = Jac<DEG>;
#pragma unroll
    for (int k = 0; k < L::N; ++k) J[k] = 0.f;
#pragma unroll
    for (int col = 0; col < 10; ++col) {
        GTan d;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d.X[k] = col == k ? 1.f : 0.f;
            d.ls[k] = col == 3 + k ? 1.f : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) d.q[k] = col == 6 + k ? 1.f : 0.f;
        d.th = 0.f;
        float out[9];
        if (col < 3)
            prim_tangent<DEG, kTanMean>(P, cam, d, sh, out);
        else if (col < 6)
            prim_tangent<DEG, kTanScale>(P, cam, d, sh, out);
        else
            prim_tangent<DEG, kTanRot>(P, cam, d, sh, out);
        if (col < 3) {
            J[L::kMu + col] = -(P.A * out[0] + P.B * out[1]);
            J[L::kMu + 3 + col] = -(P.B * out[0] + P.C * out[1]);
            if (DEG > 0) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) J[L::kGx + 3 * ch + col] = out[6 + ch];
            }
        }
        J[L::kCon + col] = -0.5f * out[2];
        J[L::kCon + 10 + col] = -out[3];
        J[L::kCon + 20 + col] = -0.5f * out[4];
    }
    J[L::kOp] = 1.f - P.o;  // d log(o) / d logit
    unsigned bits = 0u;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
        if (!P.clamped[ch]) bits |= 1u << ch;
    J[L::kMask] = __uint_as_float(bits);
}

// SH basis values Y_k of the pair's view direction, recomputed from the
// Gaussian's mean X and the camera centre with the arithmetic of
// prim_features (the cache does not hold them: at SH3 they would be a
// quarter of its bytes).  DEG 0: the constant Y_0.
template <int DEG>
__device__ __forceinline__ void pair_Y(const CamDev& cam, const float X[3], float* Y) {
    if constexpr (DEG == 0) {
        Y[0] = c_sh[0];
    } else {
        float d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = X[k] - cam.centre[k];
        const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float idn = 1.f / dn;
        sh_eval<DEG>(d[0] * idn, d[1] * idn, d[2] * idn, Y);
    }
}

template <int DEG>
__global__ void k_prep_fwd(Ctx c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)c.nv * c.G) return;
    const int slot = (int)(i / c.G), g = (int)(i % c.G);
    const CamDev& cam = c.cams[c.views[slot]];
    float X[3];
    load_mean(c.params, g, X);
    Prim P;
    load_gauss(c, g, P);
    int4 rect;
    float depth;
    float4 ell[2];
    const bool vis = prim_project(X, cam, c.tiles_x, c.tiles_y, c.tile_w, c.tile_h, P, &rect, &depth, ell);
    // visible pairs, the binning's row-list entries (the rectangle rows whose
    // band meets the ellipse), and a bound on the tile-list entries (those
    // rows times the rectangle's width; the binning counts the exact number)
    const unsigned active = __activemask();
    const unsigned ballot = __ballot_sync(active, vis);
    unsigned rows = 0u;
    if (vis)
        for (int ty = rect.z; ty <= rect.w; ++ty) rows += band_meets(ell[0], ell[1], ty, c.tile_h, c.H) ? 1u : 0u;
    const unsigned area = vis ? rows * (unsigned)(rect.y - rect.x + 1) : 0u;
    const unsigned sum_rows = __reduce_add_sync(active, rows), sum_area = __reduce_add_sync(active, area);
    if ((threadIdx.x & 31) == __ffs(active) - 1 && ballot) {
        atomicAdd(c.n_visible, (unsigned long long)__popc(ballot));
        atomicAdd(c.n_entries, (unsigned long long)sum_area);
        atomicAdd(c.n_rowent, (unsigned long long)sum_rows);
    }
    // depth key in (slot, Gaussian) order: the stable depth sort keeps index order on ties
    c.dvals[i] = (unsigned int)g;
    if (!vis) {
        c.rect[i] = make_int4(1, 0, 1, 0);
        c.dkeys[i] = ((unsigned long long)slot << 32) | 0xFFFFFFFFull;
        return;
    }
    const float* sh = c.params + 11ll * c.G + (long long)g * 3 * Sh<DEG>::K;
    prim_features<DEG>(X, sh, cam, P);
    float4* r = c.rec + i * kPrimF4;
    r[0] = make_float4(P.mux, P.muy, P.A, P.B);
    r[1] = make_float4(P.C, P.o, P.col[0], P.col[1]);
    // the conic scaled for the rasterizer's 2^x (the primal record's spare slots)
    const float L2E = 1.4426950408889634f;
    r[2] = make_float4(P.col[2], -L2E * P.B, -0.5f * L2E * P.A, -0.5f * L2E * P.C);
    c.rect[i] = rect;
    c.ell[2 * i] = ell[0];
    c.ell[2 * i + 1] = ell[1];
    c.dkeys[i] = ((unsigned long long)slot << 32) | __float_as_uint(depth);
    float J[Jac<DEG>::N];
    pair_jacobian<DEG>(P, cam, sh, J);
#pragma unroll
    for (int q = 0; q < Jac<DEG>::F4; ++q)
        c.pjac[jac_idx<DEG>(c, slot, g, q)] = make_float4(J[4 * q], J[4 * q + 1], J[4 * q + 2], J[4 * q + 3]);
}

// tangent of the 11 geometric parameters of Gaussian g
__device__ __forceinline__ void load_geo_tangent(const float* v, int G, int g, GTan& d) {
    const long long GG = G;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d.X[k] = v[3ll * g + k];
        d.ls[k] = v[3 * GG + 3ll * g + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) d.q[k] = v[6 * GG + 4ll * g + k];
    d.th = v[10 * GG + g];
}

// One thread per (Gaussian, view) pair, Gaussian-major (consecutive threads
// are the views of one Gaussian, so its parameters and tangent are loaded
// once per warp through L1).  Writes the tangent half of the pair record and
// clears the pair's cotangent slot.
// Tangent half of the pair records of Gaussian g in views slot0, slot0 +
// dslot, ... (visible ones), from the Jacobian cache, and cleared cotangent
// slots.  The lanes of a warp take consecutive Gaussians, so every plane
// load and record store is one contiguous run.
// dsh: the Gaussian's 3K SH tangent values (global memory, or a staged copy
// in shared memory).
template <int DEG>
__device__ __forceinline__ void prep_jvp_gauss(const Ctx& c, const GTan& d, const float* dsh, int g, int slot0,
                                               int dslot) {
    using L = Jac<DEG>;
    constexpr int K = Sh<DEG>::K;
    const float u[10] = {d.X[0], d.X[1], d.X[2], d.ls[0], d.ls[1], d.ls[2], d.q[0], d.q[1], d.q[2], d.q[3]};
    float X[3] = {0.f, 0.f, 0.f};
    if (DEG > 0) load_mean(c.params, g, X);
    for (int slot = slot0; slot < c.nv; slot += dslot) {
        const long long pair = (long long)slot * c.G + g;
        const int4 rc = c.rect[pair];
        if (rc.x > rc.y) continue;
        float J[L::N];
        load_jac<DEG>(c, slot, g, J);
        float Y[K];
        pair_Y<DEG>(c.cams[c.views[slot]], X, Y);
        float o[9];
        o[0] = J[L::kMu] * d.X[0] + J[L::kMu + 1] * d.X[1] + J[L::kMu + 2] * d.X[2];
        o[1] = J[L::kMu + 3] * d.X[0] + J[L::kMu + 4] * d.X[1] + J[L::kMu + 5] * d.X[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 10; ++k) a += J[L::kCon + 10 * r + k] * u[k];
            o[2 + r] = a;
        }
        o[5] = J[L::kOp] * d.th;  // tangent of log(o)
        const unsigned bits = __float_as_uint(J[L::kMask]);
        float v3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) v3[ch] += Y[k] * dsh[3 * k + ch];
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (DEG > 0)
                v3[ch] += J[L::kGx + 3 * ch] * d.X[0] + J[L::kGx + 3 * ch + 1] * d.X[1] + J[L::kGx + 3 * ch + 2] * d.X[2];
            o[6 + ch] = (bits >> ch) & 1u ? v3[ch] : 0.f;
        }
        float4* r = c.tan + pair * kTanF4;
        r[0] = make_float4(o[0], o[1], o[2], o[3]);
        r[1] = make_float4(o[4], o[5], o[6], o[7]);
        r[2] = make_float4(o[8], 0.f, 0.f, 0.f);
        float4* ct = reinterpret_cast<float4*>(c.cot + pair * kCotF);
        ct[0] = ct[1] = ct[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Blocks of 32 Gaussians (lanes) x kJvpWarps warps, warp w taking views w,
// w + kJvpWarps, ...: several warps per Gaussian for latency hiding.  The
// block's tangent values are contiguous runs of the P-vector (32 x 3K SH
// values; 3, 3, 4 and 1 geometric values per Gaussian in the four geometric
// groups): the block stages them once, coalesced, into shared memory (row
// strides 3K + 1 and 11, odd, so the lanes' reads of their own rows hit
// distinct banks).  With z given, the staged tangent is the PCG direction
// p <- z + beta p (Alg. 1, beta from the device scalars), written back to p
// by the thread that read it; otherwise it is v = p as given.
constexpr int kJvpWarps = 4;

// Position in the P-vector, and in the staging area, of the i-th of the
// 11 ng geometric values of Gaussians g0 .. g0 + ng - 1 (their runs in the
// means, log-scale, quaternion and opacity groups, in that order).
__device__ __forceinline__ void geo_slot(long long G, int g0, int ng, int i, long long& idx, int& at) {
    int row, k;
    if (i < 3 * ng) {
        idx = 3ll * g0 + i, row = i / 3, k = i % 3;
    } else if (i < 6 * ng) {
        const int o = i - 3 * ng;
        idx = 3 * G + 3ll * g0 + o, row = o / 3, k = 3 + o % 3;
    } else if (i < 10 * ng) {
        const int o = i - 6 * ng;
        idx = 6 * G + 4ll * g0 + o, row = o / 4, k = 6 + o % 4;
    } else {
        const int o = i - 10 * ng;
        idx = 10 * G + g0 + o, row = o, k = 10;
    }
    at = row * 11 + k;
}

template <int DEG>
__global__ void __launch_bounds__(32 * kJvpWarps) k_prep_jvp(Ctx c, const float* __restrict__ z, float* p) {
    constexpr int K3 = 3 * Sh<DEG>::K;
    constexpr int kThreads = 32 * kJvpWarps;
    constexpr int kShPer = (32 * K3 + kThreads - 1) / kThreads;  // SH values per thread
    constexpr int kGeoPer = (32 * 11 + kThreads - 1) / kThreads;
    __shared__ float s_dsh[32 * (K3 + 1)];
    __shared__ float s_geo[32 * 11];
    const int g0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31;
    const int ng = min(32, c.G - g0);
    const float beta = z ? (float)c.sc->beta : 0.f;
    const long long G = c.G;
    const long long sh0 = 11 * G + (long long)g0 * K3;
    const int nsh = ng * K3, ngeo = 11 * ng;
    // every load of the thread first, then the direction and the stores
    float vs[kShPer], vg[kGeoPer], zs[kShPer], zg[kGeoPer];
    long long gidx[kGeoPer];
    int gat[kGeoPer];
#pragma unroll
    for (int k = 0; k < kShPer; ++k) {
        const int i = threadIdx.x + k * kThreads;
        vs[k] = i < nsh ? p[sh0 + i] : 0.f;
        zs[k] = (z && i < nsh) ? z[sh0 + i] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kGeoPer; ++k) {
        const int i = threadIdx.x + k * kThreads;
        gidx[k] = 0;
        gat[k] = 0;
        if (i < ngeo) geo_slot(G, g0, ng, i, gidx[k], gat[k]);
        vg[k] = i < ngeo ? p[gidx[k]] : 0.f;
        zg[k] = (z && i < ngeo) ? z[gidx[k]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kShPer; ++k) {
        const int i = threadIdx.x + k * kThreads;
        if (i >= nsh) continue;
        float val = vs[k];
        if (z) {
            val = zs[k] + beta * val;
            p[sh0 + i] = val;
        }
        s_dsh[(i / K3) * (K3 + 1) + i % K3] = val;
    }
#pragma unroll
    for (int k = 0; k < kGeoPer; ++k) {
        const int i = threadIdx.x + k * kThreads;
        if (i >= ngeo) continue;
        float val = vg[k];
        if (z) {
            val = zg[k] + beta * val;
            p[gidx[k]] = val;
        }
        s_geo[gat[k]] = val;
    }
    __syncthreads();
    const int g = g0 + lane;
    if (g < c.G) {
        const float* sg = s_geo + lane * 11;
        GTan d;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d.X[k] = sg[k];
            d.ls[k] = sg[3 + k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) d.q[k] = sg[6 + k];
        d.th = sg[10];
        prep_jvp_gauss<DEG>(c, d, s_dsh + lane * (K3 + 1), g, threadIdx.x >> 5, kJvpWarps);
    }
}

// The same for every scene of a batch: Gaussian chunks, tangent = the scene's p.
template <int DEG>
__device__ __forceinline__ void b_prep_jvp(const BatchTables& t) {
    static_assert(kBatchBlock == 32 * kJvpWarps, "one lane per Gaussian, one warp per view class");
    const int n = t.counts[0];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.gchunks[k];
        for (int g = ch.y + (int)(threadIdx.x & 31); g < ch.z; g += 32) {
            const Ctx& c = t.ctxs[ch.x];
            const float* v = t.vecs[ch.x].p;
            GTan d;
            load_geo_tangent(v, c.G, g, d);
            prep_jvp_gauss<DEG>(c, d, v + 11ll * c.G + (long long)g * 3 * Sh<DEG>::K, g, threadIdx.x >> 5, kJvpWarps);
        }
    }
}
template <int DEG>
__global__ void __launch_bounds__(kBatchBlock) kb_prep_jvp(BatchTables t) { b_prep_jvp<DEG>(t); }


constexpr int kPrepBlock = 128;

// out[idx] = val + the damping of v (when v is given), v^T out into dot.
template <bool kDot>
__device__ __forceinline__ void damp_put(const Ctx& c, float* out, const float* v, const float* D, long long idx,
                                         float val, Dot2& dot) {
    if (v) {
        const float damp = c.damping_mode == 1 ? c.lambda * D[idx] : c.lambda;
        val += damp * v[idx];
        if (kDot) dot.add(v[idx], val);
    }
    out[idx] = val;
}

// J^T of Gaussian g's cotangent slots over its visible views slot0, slot0 +
// dslot, ...: gu (X, log-scale, q), gth (opacity logit), gsh (3K SH values).
template <int DEG>
__device__ __forceinline__ void vjp_views(const Ctx& c, int g, int slot0, int dslot, float gu[10], float& gth,
                                          float* gsh) {
    using L = Jac<DEG>;
    constexpr int K = Sh<DEG>::K;
    constexpr int K3 = 3 * K;
#pragma unroll
    for (int k = 0; k < 10; ++k) gu[k] = 0.f;
    gth = 0.f;
#pragma unroll
    for (int k = 0; k < K3; ++k) gsh[k] = 0.f;
    float X[3] = {0.f, 0.f, 0.f};
    if (DEG > 0) load_mean(c.params, g, X);
    for (int slot = slot0; slot < c.nv; slot += dslot) {
        const long long i = (long long)slot * c.G + g;
        // the cache and cotangent slots exist for culled pairs too: their
        // loads go out with the rectangle's, and a culled pair's values are
        // replaced by zeros (they are stale there)
        float J[L::N];
        load_jac<DEG>(c, slot, g, J);
        const float4* ct = reinterpret_cast<const float4*>(c.cot + i * kCotF);
        const float4 c0 = ct[0], c1 = ct[1], c2 = ct[2];
        const int4 rc = c.rect[i];
        const bool vis = rc.x <= rc.y;
#pragma unroll
        for (int k = 0; k < L::N; ++k) J[k] = vis ? J[k] : 0.f;
        float Y[K];
        pair_Y<DEG>(c.cams[c.views[slot]], X, Y);
        const float cot[9] = {vis ? c0.x : 0.f, vis ? c0.y : 0.f, vis ? c0.z : 0.f, vis ? c0.w : 0.f, vis ? c1.x : 0.f,
                              vis ? c1.y : 0.f, vis ? c1.z : 0.f, vis ? c1.w : 0.f, vis ? c2.x : 0.f};
        const unsigned bits = __float_as_uint(J[L::kMask]);
        float ccol[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) ccol[ch] = (bits >> ch) & 1u ? cot[6 + ch] : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float a = J[L::kMu + k] * cot[0] + J[L::kMu + 3 + k] * cot[1];
            if (DEG > 0) a += J[L::kGx + k] * ccol[0] + J[L::kGx + 3 + k] * ccol[1] + J[L::kGx + 6 + k] * ccol[2];
            gu[k] += a;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k)
            gu[k] += J[L::kCon + k] * cot[2] + J[L::kCon + 10 + k] * cot[3] + J[L::kCon + 20 + k] * cot[4];
        gth += J[L::kOp] * cot[5];
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gsh[3 * k + ch] += Y[k] * ccol[ch];
        }
    }
}

// The geometric entries of Gaussian g: out = gu, gth (+ lambda damping of v
// when v is given; v^T out accumulated into dot).  Entries [k0, k1) of the 11.
template <bool kDot>
__device__ __forceinline__ void put_geo(const Ctx& c, int g, float* out, const float* v, const float* D,
                                        const float gu[10], float gth, Dot2& dot, int k0 = 0, int k1 = 11) {
    const long long G = c.G;
    const long long idx[11] = {3ll * g, 3ll * g + 1, 3ll * g + 2, 3 * G + 3ll * g, 3 * G + 3ll * g + 1,
                               3 * G + 3ll * g + 2, 6 * G + 4ll * g, 6 * G + 4ll * g + 1, 6 * G + 4ll * g + 2,
                               6 * G + 4ll * g + 3, 10 * G + g};
#pragma unroll
    for (int k = 0; k < 11; ++k)
        if (k >= k0 && k < k1) damp_put<kDot>(c, out, v, D, idx[k], k < 10 ? gu[k] : gth, dot);
}

// The whole map for Gaussian g, every view, one thread.
template <int DEG, bool kDot>
__device__ __forceinline__ void prep_vjp_gauss(const Ctx& c, int g, float* out, const float* v, const float* D,
                                               Dot2& dot) {
    constexpr int K3 = 3 * Sh<DEG>::K;
    float gu[10], gth, gsh[K3];
    vjp_views<DEG>(c, g, 0, 1, gu, gth, gsh);
    put_geo<kDot>(c, g, out, v, D, gu, gth, dot);
#pragma unroll
    for (int k = 0; k < K3; ++k) damp_put<kDot>(c, out, v, D, 11ll * c.G + (long long)g * K3 + k, gsh[k], dot);
}

// One warp per 32 consecutive Gaussians (grid-stride over warp groups).  The
// SH entries of the 32 Gaussians are one contiguous run of out, v and D: each
// lane stages its 3K entries in shared memory (row stride 3K + 1), then the
// warp stores the run coalesced, with the damping and the dot product.  (A
// lane pair per Gaussian, each lane taking half of the views, measured
// slower: 134 against 108 us on the 200k-Gaussian workload.)
template <int DEG, bool kDot>
__global__ void __launch_bounds__(kPrepBlock) k_prep_vjp(Ctx c, float* out, const float* v, const float* D) {
    constexpr int K3 = 3 * Sh<DEG>::K;
    __shared__ float s_sh[kPrepBlock / 32][32 * (K3 + 1)];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* stage = s_sh[wid];
    Dot2 dot;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long gw = (long long)blockIdx.x * blockDim.x + wid * 32; gw < c.G; gw += stride) {
        const int g = (int)gw + lane;
        if (g < c.G) {
            float gu[10], gth, gsh[K3];
            vjp_views<DEG>(c, g, 0, 1, gu, gth, gsh);
            put_geo<kDot>(c, g, out, v, D, gu, gth, dot);
            float* row = stage + lane * (K3 + 1);
#pragma unroll
            for (int k = 0; k < K3; ++k) row[k] = gsh[k];
        }
        __syncwarp();
        const int n = (int)min(32ll, (long long)c.G - gw) * K3;
        const long long base = 11ll * c.G + gw * K3;
        // the run's v and D first (out may alias neither, but the compiler
        // cannot know: loaded after a store, each would be a round trip)
        float vv[K3], dv[K3];
#pragma unroll
        for (int k = 0; k < K3; ++k) {
            const int i = k * 32 + lane;
            vv[k] = (v && i < n) ? v[base + i] : 0.f;
            dv[k] = (v && c.damping_mode == 1 && i < n) ? D[base + i] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < K3; ++k) {
            const int i = k * 32 + lane;
            if (i >= n) continue;
            float val = stage[(i / K3) * (K3 + 1) + i % K3];
            if (v) {
                val += (c.damping_mode == 1 ? c.lambda * dv[k] : c.lambda) * vv[k];
                if (kDot) dot.add(vv[k], val);
            }
            out[base + i] = val;
        }
        __syncwarp();
    }
    if (kDot) {
        double tot;
        if (grid_sum_last<kPrepBlock>(dot.value(), c.partials, c.counter, &tot) && threadIdx.x == 0) {
            Scalars* s = c.sc;
            s->pAp = tot;
            if (s->rz == 0.0) {
                s->alpha = 0.0;
            } else if (!(tot > 0.0) || !isfinite(tot)) {
                s->numeric_error = 1u;
                s->alpha = 0.0;
            } else {
                s->alpha = s->rz / tot;
            }
        }
    }
}

// The same for every scene of a batch: Ap = J^T W J p + damping, and
// p^T A p of iteration `iter` accumulated into the scene's history (the
// per-thread Dot2 partials of one chunk are summed in FP64 over the block).
template <int DEG>
__device__ __forceinline__ void b_prep_vjp(const BatchTables& t, int iter) {
    const int n = t.counts[0];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 ch = t.gchunks[k];
        const Ctx& c = t.ctxs[ch.x];
        const BatchVec& bv = t.vecs[ch.x];
        Dot2 dot;
        const int g = ch.y + threadIdx.x;
        if (g < ch.z) prep_vjp_gauss<DEG, true>(c, g, bv.Ap, bv.p, bv.D, dot);
        const double tot = block_sum<kBatchBlock>(dot.value());
        if (threadIdx.x == 0) atomicAdd(&bv.pAp[iter], tot);
    }
}
template <int DEG>
__global__ void __launch_bounds__(kBatchBlock) kb_prep_vjp(BatchTables t, int iter) { b_prep_vjp<DEG>(t, iter); }


// diag(J^T W J) for Gaussian g: the sum over its visible views of the
// pair slots k_diag filled (the 11 geometric entries directly; SH
// coefficient (k, ch) moves only colour ch, by Y_k, so its entry is
// Y_k^2 sum w_ch q^2 where channel ch is not clamped).
template <int DEG>
__global__ void __launch_bounds__(kPrepBlock) k_prep_diag(Ctx c, float* D) {
    using L = Jac<DEG>;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= c.G) return;
    constexpr int K = Sh<DEG>::K;
    constexpr int K3 = 3 * K;
    float dgeo[11];
#pragma unroll
    for (int j = 0; j < 11; ++j) dgeo[j] = 0.f;
    float dsh[K3];
#pragma unroll
    for (int k = 0; k < K3; ++k) dsh[k] = 0.f;
    float X[3] = {0.f, 0.f, 0.f};
    if (DEG > 0) load_mean(c.params, g, X);
    for (int slot = 0; slot < c.nv; ++slot) {
        const long long i = (long long)slot * c.G + g;
        // loads before the visibility test; a culled pair's (stale) slot and
        // mask are replaced by zeros
        const float4* src = reinterpret_cast<const float4*>(c.dslot + i * kDiagF);
        const float4 s0 = src[0], s1 = src[1], s2 = src[2], s3 = src[3];
        static_assert(L::kMask % 4 == 1, "the clamp mask is the .y of its plane");
        const float maskf = c.pjac[jac_idx<DEG>(c, slot, g, L::kMask / 4)].y;
        const int4 rc = c.rect[i];
        const bool vis = rc.x <= rc.y;
        const float v[14] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w, s2.x, s2.y, s2.z, s2.w, s3.x, s3.y};
#pragma unroll
        for (int j = 0; j < 11; ++j) dgeo[j] += vis ? v[j] : 0.f;
        const unsigned bits = vis ? __float_as_uint(maskf) : 0u;
        float Y[K];
        pair_Y<DEG>(c.cams[c.views[slot]], X, Y);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float y2 = Y[k] * Y[k];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                if ((bits >> ch) & 1u) dsh[3 * k + ch] = fmaf(y2, v[11 + ch], dsh[3 * k + ch]);
        }
    }
    const long long G = c.G;
#pragma unroll
    for (int k = 0; k < 3; ++k) D[3ll * g + k] = dgeo[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) D[3 * G + 3ll * g + k] = dgeo[3 + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) D[6 * G + 4ll * g + k] = dgeo[6 + k];
    D[10 * G + g] = dgeo[10];
#pragma unroll
    for (int k = 0; k < K3; ++k) D[11 * G + (long long)g * K3 + k] = dsh[k];
}

// ---------------------------------------------------------------------------
// Launchers (dispatch on the SH degree)
// ---------------------------------------------------------------------------
void launch_sample(const Ctx& c, long long lm_step, unsigned long long seed, cudaStream_t st) {
    const int n = c.nv * c.T;
    LMRS_LAUNCH(k_sample, (n + 127) / 128, 128, 0, st, c, lm_step, seed);
}

void launch_prep_gauss(const Ctx& c, cudaStream_t st) {
    LMRS_LAUNCH(k_prep_gauss, (c.G + 255) / 256, 256, 0, st, c);
}

template <int DEG>
static void prep_fwd_deg(const Ctx& c, cudaStream_t st) {
    const long long n = (long long)c.nv * c.G;
    LMRS_LAUNCH_AS("k_prep_fwd", k_prep_fwd<DEG>, (unsigned)((n + 127) / 128), 128, 0, st, c);
}
template <int DEG>
static void prep_jvp_deg(const Ctx& c, const float* z, float* p, cudaStream_t st) {
    LMRS_LAUNCH_AS("k_prep_jvp", k_prep_jvp<DEG>, (unsigned)((c.G + 31) / 32), 32 * kJvpWarps, 0, st, c, z, p);
}
template <int DEG>
static void prep_vjp_deg(const Ctx& c, float* g, const float* v, const float* D, bool dot, cudaStream_t st) {
    int grid = (c.G + kPrepBlock - 1) / kPrepBlock;
    if (dot) {
        if (grid > kMaxPartials) grid = kMaxPartials;
        LMRS_LAUNCH_AS("k_prep_vjp<dot>", (k_prep_vjp<DEG, true>), grid, kPrepBlock, 0, st, c, g, v, D);
    } else {
        LMRS_LAUNCH_AS("k_prep_vjp", (k_prep_vjp<DEG, false>), grid, kPrepBlock, 0, st, c, g, v, D);
    }
}
template <int DEG>
static void prep_diag_deg(const Ctx& c, float* D, cudaStream_t st) {
    LMRS_LAUNCH_AS("k_prep_diag", k_prep_diag<DEG>, (c.G + kPrepBlock - 1) / kPrepBlock, kPrepBlock, 0, st, c, D);
}

void launch_prep_fwd(const Ctx& c, cudaStream_t st) {
    switch (c.deg) {
        case 0: prep_fwd_deg<0>(c, st); break;
        case 1: prep_fwd_deg<1>(c, st); break;
        case 2: prep_fwd_deg<2>(c, st); break;
        default: prep_fwd_deg<3>(c, st); break;
    }
}

void launch_prep_jvp(const Ctx& c, const float* v, cudaStream_t st) {
    // read only: k_prep_jvp writes p only when z is given
    float* p = const_cast<float*>(v);
    switch (c.deg) {
        case 0: prep_jvp_deg<0>(c, nullptr, p, st); break;
        case 1: prep_jvp_deg<1>(c, nullptr, p, st); break;
        case 2: prep_jvp_deg<2>(c, nullptr, p, st); break;
        default: prep_jvp_deg<3>(c, nullptr, p, st); break;
    }
}

void launch_prep_jvp_direction(const Ctx& c, const float* z, float* p, cudaStream_t st) {
    switch (c.deg) {
        case 0: prep_jvp_deg<0>(c, z, p, st); break;
        case 1: prep_jvp_deg<1>(c, z, p, st); break;
        case 2: prep_jvp_deg<2>(c, z, p, st); break;
        default: prep_jvp_deg<3>(c, z, p, st); break;
    }
}

void launch_prep_vjp(const Ctx& c, float* g, const float* v, const float* D, bool dot, cudaStream_t st) {
    switch (c.deg) {
        case 0: prep_vjp_deg<0>(c, g, v, D, dot, st); break;
        case 1: prep_vjp_deg<1>(c, g, v, D, dot, st); break;
        case 2: prep_vjp_deg<2>(c, g, v, D, dot, st); break;
        default: prep_vjp_deg<3>(c, g, v, D, dot, st); break;
    }
}

void launch_b_prep_jvp(const BatchTables& t, int deg, int grid, cudaStream_t st) {
    switch (deg) {
        case 0: LMRS_LAUNCH(kb_prep_jvp<0>, grid, kBatchBlock, 0, st, t); break;
        case 1: LMRS_LAUNCH(kb_prep_jvp<1>, grid, kBatchBlock, 0, st, t); break;
        case 2: LMRS_LAUNCH(kb_prep_jvp<2>, grid, kBatchBlock, 0, st, t); break;
        default: LMRS_LAUNCH(kb_prep_jvp<3>, grid, kBatchBlock, 0, st, t); break;
    }
}

void launch_b_prep_vjp(const BatchTables& t, int deg, int iter, int grid, cudaStream_t st) {
    switch (deg) {
        case 0: LMRS_LAUNCH(kb_prep_vjp<0>, grid, kBatchBlock, 0, st, t, iter); break;
        case 1: LMRS_LAUNCH(kb_prep_vjp<1>, grid, kBatchBlock, 0, st, t, iter); break;
        case 2: LMRS_LAUNCH(kb_prep_vjp<2>, grid, kBatchBlock, 0, st, t, iter); break;
        default: LMRS_LAUNCH(kb_prep_vjp<3>, grid, kBatchBlock, 0, st, t, iter); break;
    }
}

void launch_prep_diag(const Ctx& c, float* D, cudaStream_t st) {
    switch (c.deg) {
        case 0: prep_diag_deg<0>(c, D, st); break;
        case 1: prep_diag_deg<1>(c, D, st); break;
        case 2: prep_diag_deg<2>(c, D, st); break;
        default: prep_diag_deg<3>(c, D, st); break;
    }
}

}  // namespace lmrs
