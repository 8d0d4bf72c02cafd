// FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see lmrs_oracle.h).
//
// Plain and slow on purpose.  The forward model is written once, templated on
// its scalar type: `double` gives values, `Dual` (value + tangent, the
// dual numbers of Alg. 3, App. A) gives Jacobian-vector products by forward
// mode.  The reverse pass through alpha compositing is written by hand from
// the rendering equation (Eq. 4), and the chain back to the 3D parameters uses
// the preprocessing Jacobian obtained column by column with dual numbers.
//
// Build flags must include -ffp-contract=off: the FP32 decision pass relies on
// every operation being rounded on its own, and the double and Dual
// instantiations must take identical discrete decisions.
#include "lmrs_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// --------------------------------------------------------------------------
// Dual numbers (Alg. 3): a value and its directional derivative.
// --------------------------------------------------------------------------
struct Dual {
    double v, d;
    Dual() : v(0.0), d(0.0) {}
    Dual(double x) : v(x), d(0.0) {}
    Dual(double x, double y) : v(x), d(y) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.v * b.d + a.d * b.v); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual sqrt(Dual a) { double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
inline double val(double x) { return x; }
inline double val(float x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double tan_of(double) { return 0.0; }
inline double tan_of(const Dual& x) { return x.d; }
using std::exp;
using std::sqrt;

constexpr double kPi = 3.14159265358979323846;
constexpr double kAlphaMin = 1.0 / 255.0;  // skip threshold (3DGS convention)
constexpr double kAlphaMax = 0.99;         // alpha clamp
constexpr double kTMin = 1e-4;             // termination threshold
constexpr double kDilation = 0.3;          // low-pass added to the 2D covariance

// --------------------------------------------------------------------------
// Real spherical harmonics up to degree 3, written in Cartesian form on the
// unit sphere.  Normalisation K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!),
// sqrt(2) K for m != 0, no Condon-Shortley phase; index l^2 + l + m.
// The colour of Sec. 4.5 is c = Y_0 * sh_dc + ... + 0.5.
// --------------------------------------------------------------------------
struct ShConst {
    double k00, k1, k2a, k20, k22, k33, k32a, k31, k30, k32;
    ShConst() {
        k00 = std::sqrt(1.0 / (4.0 * kPi));
        k1 = std::sqrt(3.0 / (4.0 * kPi));
        k2a = std::sqrt(15.0 / (4.0 * kPi));
        k20 = std::sqrt(5.0 / (16.0 * kPi));
        k22 = std::sqrt(15.0 / (16.0 * kPi));
        k33 = std::sqrt(35.0 / (32.0 * kPi));
        k32a = std::sqrt(105.0 / (4.0 * kPi));
        k31 = std::sqrt(21.0 / (32.0 * kPi));
        k30 = std::sqrt(7.0 / (16.0 * kPi));
        k32 = std::sqrt(105.0 / (16.0 * kPi));
    }
};
const ShConst kSh;

template <class S>
void sh_basis(int deg, S x, S y, S z, S* Y) {
    Y[0] = S(kSh.k00);
    if (deg >= 1) {
        Y[1] = S(kSh.k1) * y;
        Y[2] = S(kSh.k1) * z;
        Y[3] = S(kSh.k1) * x;
    }
    if (deg >= 2) {
        Y[4] = S(kSh.k2a) * x * y;
        Y[5] = S(kSh.k2a) * y * z;
        Y[6] = S(kSh.k20) * (S(3.0) * z * z - S(1.0));
        Y[7] = S(kSh.k2a) * x * z;
        Y[8] = S(kSh.k22) * (x * x - y * y);
    }
    if (deg >= 3) {
        Y[9] = S(kSh.k33) * y * (S(3.0) * x * x - y * y);
        Y[10] = S(kSh.k32a) * x * y * z;
        Y[11] = S(kSh.k31) * y * (S(5.0) * z * z - S(1.0));
        Y[12] = S(kSh.k30) * z * (S(5.0) * z * z - S(3.0));
        Y[13] = S(kSh.k31) * x * (S(5.0) * z * z - S(1.0));
        Y[14] = S(kSh.k32) * z * (x * x - y * y);
        Y[15] = S(kSh.k33) * x * (x * x - S(3.0) * y * y);
    }
}

// --------------------------------------------------------------------------
// Cameras.
// --------------------------------------------------------------------------
struct CamD {
    int W, H;
    double fx, fy, cx, cy, znear, limx, limy;
    double R[3][3], t[3], centre[3];
};
struct CamF {
    int W, H;
    float fx, fy, cx, cy, znear, limx, limy;
    float R[9], t[3];
};

CamD cam_double(const orc_camera& c) {
    CamD d;
    d.W = c.width; d.H = c.height;
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.znear = c.znear;
    // the projected mean is clamped 30% beyond the half field of view
    d.limx = 1.3 * (0.5 * c.width / (double)c.fx);
    d.limy = 1.3 * (0.5 * c.height / (double)c.fy);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) d.R[i][j] = c.world_to_cam[4 * i + j];
        d.t[i] = c.world_to_cam[4 * i + 3];
    }
    for (int j = 0; j < 3; ++j)  // camera centre = -R^T t
        d.centre[j] = -(d.R[0][j] * d.t[0] + d.R[1][j] * d.t[1] + d.R[2][j] * d.t[2]);
    return d;
}

CamF cam_float(const orc_camera& c) {
    CamF f;
    f.W = c.width; f.H = c.height;
    f.fx = c.fx; f.fy = c.fy; f.cx = c.cx; f.cy = c.cy; f.znear = c.znear;
    f.limx = 1.3f * ((0.5f * (float)c.width) / c.fx);
    f.limy = 1.3f * ((0.5f * (float)c.height) / c.fy);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) f.R[3 * i + j] = c.world_to_cam[4 * i + j];
        f.t[i] = c.world_to_cam[4 * i + 3];
    }
    return f;
}

// --------------------------------------------------------------------------
// FP32 list decisions (visibility, depth key, tile rectangle, and the tile
// columns each row of the rectangle keeps).  Every operation is a single IEEE
// binary32 operation in the written order (the build disables contraction);
// the scale exponential and the ellipse level are binary32 roundings of
// double expressions.  The CUDA side follows the same sequence.
// --------------------------------------------------------------------------
struct GeoF {
    int vis;
    float depth;
    int x0, x1, y0, y1;  // inclusive tile rectangle
    // the ellipse {d : d^T Sigma2^-1 d <= tau} around the 2D mean (mux, muy),
    // tau = 2 ln(255 o) + kTauSlack: every pixel whose alpha reaches 1/255
    // lies inside it.  Given the offset dy from muy, its points have
    // (dx - kx dy)^2 <= pq - qq dy^2 (the conditional form of the 2D
    // Gaussian); |dy| <= ey; the rightmost point has dy = dys, the leftmost
    // dy = -dys.  ey < 0: no pixel reaches 1/255.
    float mux, muy, kx, dys, pq, qq, ey;
};

// Slack on the ellipse's level: the lists keep every tile some pixel of which
// reaches alpha >= 1/255 by a margin far above the FP32 rounding of the
// renderer's alpha (a factor e^-0.01 on the threshold).
constexpr double kTauSlack = 0.02;

// Level tau of the 1/255 ellipse: alpha = o exp(-q/2) >= 1/255 iff
// q <= 2 ln(255 o); o = sigmoid(logit), in double, rounded once to binary32.
float ellipse_level(float logit) {
    const double o = 1.0 / (1.0 + std::exp(-(double)logit));
    return (float)(2.0 * std::log(255.0 * o) + kTauSlack);
}

GeoF geom_f32(const float* X, const float* ls, const float* q, float logit, const CamF& c,
              int tiles_x, int tiles_y, int tw, int th) {
    GeoF g;
    g.vis = 0; g.depth = 0.f; g.x0 = g.x1 = g.y0 = g.y1 = 0;
    g.mux = g.muy = g.kx = g.dys = g.pq = g.qq = 0.f;
    g.ey = -1.f;
    const float* R = c.R;
    float t0 = ((R[0] * X[0] + R[1] * X[1]) + R[2] * X[2]) + c.t[0];
    float t1 = ((R[3] * X[0] + R[4] * X[1]) + R[5] * X[2]) + c.t[1];
    float t2 = ((R[6] * X[0] + R[7] * X[1]) + R[8] * X[2]) + c.t[2];
    if (!(t2 > c.znear)) return g;
    float s[3];
    for (int j = 0; j < 3; ++j) s[j] = (float)std::exp((double)ls[j]);
    float qq = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(qq > 0.f)) return g;
    float qn = std::sqrt(qq);
    float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    float r[3][3];
    r[0][0] = 1.f - 2.f * (y * y + z * z);
    r[0][1] = 2.f * (x * y - w * z);
    r[0][2] = 2.f * (x * z + w * y);
    r[1][0] = 2.f * (x * y + w * z);
    r[1][1] = 1.f - 2.f * (x * x + z * z);
    r[1][2] = 2.f * (y * z - w * x);
    r[2][0] = 2.f * (x * z - w * y);
    r[2][1] = 2.f * (y * z + w * x);
    r[2][2] = 1.f - 2.f * (x * x + y * y);
    float m[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m[i][j] = r[i][j] * s[j];
    float S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            S[i][j] = (m[i][0] * m[j][0] + m[i][1] * m[j][1]) + m[i][2] * m[j][2];
            S[j][i] = S[i][j];
        }
    float ux = t0 / t2, uy = t1 / t2;
    float cux = std::fmin(std::fmax(ux, -c.limx), c.limx);
    float cuy = std::fmin(std::fmax(uy, -c.limy), c.limy);
    float j00 = c.fx / t2;
    float j02 = -((c.fx * cux) / t2);
    float j11 = c.fy / t2;
    float j12 = -((c.fy * cuy) / t2);
    float T[2][3];
    for (int k = 0; k < 3; ++k) {
        T[0][k] = j00 * R[k] + j02 * R[6 + k];
        T[1][k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    float V[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) V[i][k] = (T[i][0] * S[0][k] + T[i][1] * S[1][k]) + T[i][2] * S[2][k];
    float a = ((V[0][0] * T[0][0] + V[0][1] * T[0][1]) + V[0][2] * T[0][2]) + 0.3f;
    float b = (V[0][0] * T[1][0] + V[0][1] * T[1][1]) + V[0][2] * T[1][2];
    float cc = ((V[1][0] * T[1][0] + V[1][1] * T[1][1]) + V[1][2] * T[1][2]) + 0.3f;
    float det = a * cc - b * b;
    if (!(det > 0.f)) return g;
    float mid = 0.5f * (a + cc);
    float disc = std::fmax(mid * mid - det, 0.1f);
    float lam = mid + std::sqrt(disc);
    float rad = std::ceil(3.0f * std::sqrt(lam));
    float mux = c.fx * ux + c.cx;
    float muy = c.fy * uy + c.cy;
    float fx0 = std::floor((mux - rad) / (float)tw);
    float fx1 = std::floor((mux + rad) / (float)tw);
    float fy0 = std::floor((muy - rad) / (float)th);
    float fy1 = std::floor((muy + rad) / (float)th);
    if (fx1 < 0.f || fx0 > (float)(tiles_x - 1) || fy1 < 0.f || fy0 > (float)(tiles_y - 1)) return g;
    g.vis = 1;
    g.depth = t2;
    g.x0 = (int)std::fmax(fx0, 0.f);
    g.x1 = (int)std::fmin(fx1, (float)(tiles_x - 1));
    g.y0 = (int)std::fmax(fy0, 0.f);
    g.y1 = (int)std::fmin(fy1, (float)(tiles_y - 1));
    g.mux = mux;
    g.muy = muy;
    const float tau = ellipse_level(logit);
    if (tau > 0.f) {
        const float sv = det / cc;  // variance of dx given dy
        g.kx = b / cc;
        g.pq = sv * tau;
        g.qq = sv / cc;
        g.ey = std::sqrt(tau * cc);
        g.dys = b * std::sqrt(tau / a);
    }
    return g;
}

// Tile columns [*sx0, *sx1] of tile row ty that the Gaussian's list covers:
// those of its rectangle holding a pixel-centre column that meets the
// ellipse inside the row's band of pixel-centre rows [yA, yB] (the band taken
// as an interval, so the test can only keep more).  The ellipse cut by the
// band is convex, so the columns it meets form one interval: from the
// leftmost point x_l(dl) to the rightmost x_r(dr), where the unconstrained
// extreme offsets -dys / dys are clamped into the band (x_r is concave in dy,
// x_l convex).  False: no tile of this row.
bool row_span(const GeoF& q, int ty, int tw, int th, int W, int H, int* sx0, int* sx1) {
    const float yA = (float)(ty * th) + 0.5f;
    const float yB = (float)std::min(ty * th + th, H) - 0.5f;
    const float lo = std::fmax(yA - q.muy, -q.ey);
    const float hi = std::fmin(yB - q.muy, q.ey);
    if (!(lo <= hi)) return false;
    const float dr = std::fmin(std::fmax(q.dys, lo), hi);
    const float dl = std::fmin(std::fmax(-q.dys, lo), hi);
    const float hr = std::sqrt(std::fmax(q.pq - q.qq * (dr * dr), 0.f));
    const float hl = std::sqrt(std::fmax(q.pq - q.qq * (dl * dl), 0.f));
    const float xr = q.mux + (q.kx * dr + hr);
    const float xl = q.mux + (q.kx * dl - hl);
    // pixel columns px whose centre px + 1/2 lies in [xl, xr]
    const float fl = std::fmax(std::ceil(xl - 0.5f), 0.f);
    const float fh = std::fmin(std::floor(xr - 0.5f), (float)(W - 1));
    if (!(fl <= fh)) return false;
    *sx0 = std::max((int)fl / tw, q.x0);
    *sx1 = std::min((int)fh / tw, q.x1);
    return *sx0 <= *sx1;
}

uint32_t float_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

// --------------------------------------------------------------------------
// Continuous preprocessing (Sec. 3, Eqs. 2-4; App. A): per (view, Gaussian),
// the 2D features the rasterizer reads.  Templated on the scalar type.
// --------------------------------------------------------------------------
template <class S>
struct Gauss {
    S X[3], ls[3], q[4], th;
    S sh[16][3];
};

template <class S>
struct Feat {
    S mu[2], con[3], o, col[3];
    int clamped[3];
};

template <class S>
void preprocess(const Gauss<S>& g, int deg, const CamD& c, Feat<S>& f) {
    S t[3];
    for (int k = 0; k < 3; ++k)
        t[k] = S(c.R[k][0]) * g.X[0] + S(c.R[k][1]) * g.X[1] + S(c.R[k][2]) * g.X[2] + S(c.t[k]);
    // Sigma = R S S^T R^T (Eq. 3) with s = exp(log-scale) and q normalised
    S s[3];
    for (int j = 0; j < 3; ++j) s[j] = exp(g.ls[j]);
    S qn = sqrt(g.q[0] * g.q[0] + g.q[1] * g.q[1] + g.q[2] * g.q[2] + g.q[3] * g.q[3]);
    S w = g.q[0] / qn, x = g.q[1] / qn, y = g.q[2] / qn, z = g.q[3] / qn;
    S R[3][3];
    R[0][0] = S(1.0) - S(2.0) * (y * y + z * z);
    R[0][1] = S(2.0) * (x * y - w * z);
    R[0][2] = S(2.0) * (x * z + w * y);
    R[1][0] = S(2.0) * (x * y + w * z);
    R[1][1] = S(1.0) - S(2.0) * (x * x + z * z);
    R[1][2] = S(2.0) * (y * z - w * x);
    R[2][0] = S(2.0) * (x * z - w * y);
    R[2][1] = S(2.0) * (y * z + w * x);
    R[2][2] = S(1.0) - S(2.0) * (x * x + y * y);
    S M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
    S Sig[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Sig[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
    // perspective projection, linearised at the mean (EWA splatting)
    S ux = t[0] / t[2], uy = t[1] / t[2];
    S cux = ux, cuy = uy;
    if (val(ux) < -c.limx) cux = S(-c.limx);
    if (val(ux) > c.limx) cux = S(c.limx);
    if (val(uy) < -c.limy) cuy = S(-c.limy);
    if (val(uy) > c.limy) cuy = S(c.limy);
    S J00 = S(c.fx) / t[2], J02 = -(S(c.fx) * cux) / t[2];
    S J11 = S(c.fy) / t[2], J12 = -(S(c.fy) * cuy) / t[2];
    S T[2][3];
    for (int k = 0; k < 3; ++k) {
        T[0][k] = J00 * S(c.R[0][k]) + J02 * S(c.R[2][k]);
        T[1][k] = J11 * S(c.R[1][k]) + J12 * S(c.R[2][k]);
    }
    S cov[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            S acc = S(0.0);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc = acc + T[i][a] * Sig[a][b] * T[j][b];
            cov[i][j] = acc;
        }
    S a = cov[0][0] + S(kDilation), b = cov[0][1], cc = cov[1][1] + S(kDilation);
    S det = a * cc - b * b;
    f.con[0] = cc / det;
    f.con[1] = -b / det;
    f.con[2] = a / det;
    f.mu[0] = S(c.fx) * ux + S(c.cx);
    f.mu[1] = S(c.fy) * uy + S(c.cy);
    f.o = S(1.0) / (S(1.0) + exp(-g.th));
    // view-dependent colour from the SH coefficients
    S d[3];
    for (int k = 0; k < 3; ++k) d[k] = g.X[k] - S(c.centre[k]);
    S dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    S Y[16];
    sh_basis<S>(deg, d[0] / dn, d[1] / dn, d[2] / dn, Y);
    int K = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        S acc = S(0.5);
        for (int k = 0; k < K; ++k) acc = acc + g.sh[k][ch] * Y[k];
        f.clamped[ch] = val(acc) < 0.0;
        f.col[ch] = f.clamped[ch] ? S(0.0) : acc;
    }
}

// --------------------------------------------------------------------------
// Alpha compositing of one pixel (Eq. 4, Alg. 2), front to back over the
// depth-sorted list of its tile; decisions on values only.
// --------------------------------------------------------------------------
inline bool near_rel(double v, double thr, double m) { return std::fabs(v - thr) <= m * thr; }

// A decision on a value within a relative margin of its threshold is "near":
// an implementation in other precision may take it the other way, and both
// outcomes are correct.  flip: bit k inverts the k-th near decision met along
// the list (the alpha clamp, the alpha skip and the termination test, in that
// order per entry), so the oracle can follow the outcome another
// implementation took; *n_near receives the number of near decisions met.
struct Decisions {
    uint32_t flip;
    int k = 0;
    explicit Decisions(uint32_t f) : flip(f) {}
    // the outcome of a test whose plain result is `plain`, near its threshold or not
    bool take(bool plain, bool near) {
        if (!near) return plain;
        const bool inv = k < 32 && ((flip >> k) & 1u);
        ++k;
        return inv ? !plain : plain;
    }
};

template <class S>
void composite(double pcx, double pcy, const int32_t* ids, int len, const Feat<S>* F,
               double ma, double mT, S C[3], int* consumed, int* flag, int* n_comp = nullptr, uint32_t flip = 0u,
               int* n_near = nullptr) {
    S T = S(1.0);
    C[0] = C[1] = C[2] = S(0.0);
    int used = len, fl = 0, nc = 0;
    Decisions dec(flip);
    for (int k = 0; k < len; ++k) {
        const Feat<S>& f = F[ids[k]];
        S dx = f.mu[0] - S(pcx), dy = f.mu[1] - S(pcy);
        S power = S(-0.5) * (f.con[0] * dx * dx + f.con[2] * dy * dy) - f.con[1] * dx * dy;
        S alpha = f.o * exp(power);
        const double av = val(alpha);
        const bool nmax = near_rel(av, kAlphaMax, ma), nmin = near_rel(av, kAlphaMin, ma);
        if (nmin) fl |= 1;
        if (nmax) fl |= 2;
        const bool clamp = dec.take(av > kAlphaMax, nmax);
        const bool skip = dec.take(av < kAlphaMin, nmin);
        if (clamp) alpha = S(kAlphaMax);
        if (skip) continue;
        S Tn = T * (S(1.0) - alpha);
        const bool nT = near_rel(val(Tn), kTMin, mT);
        if (nT) fl |= 4;
        if (dec.take(val(Tn) < kTMin, nT)) { used = k; break; }
        for (int ch = 0; ch < 3; ++ch) C[ch] = C[ch] + f.col[ch] * alpha * T;
        T = Tn;
        ++nc;
    }
    if (consumed) *consumed = used;
    if (flag) *flag = fl;
    if (n_comp) *n_comp = nc;
    if (n_near) *n_near = dec.k;
}

// Per-pixel derivatives of the three output channels with respect to the
// nine features (mu_x, mu_y, A, B, C, o, c_r, c_g, c_b) of each contributing
// Gaussian, by reverse accumulation through Eq. 4 (written separately from
// the forward-mode path).
struct Contrib {
    int id;
    double dC[3][9];
};

void pixel_feature_jacobian(double pcx, double pcy, const int32_t* ids, int len, const Feat<double>* F,
                            std::vector<Contrib>& out, double Cfinal[3], double ma, double mT, uint32_t flip) {
    struct Rec { int id; double alpha, T, g, dx, dy; bool aclamp; };
    std::vector<Rec> recs;
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    Decisions dec(flip);
    for (int k = 0; k < len; ++k) {
        const Feat<double>& f = F[ids[k]];
        double dx = f.mu[0] - pcx, dy = f.mu[1] - pcy;
        double power = -0.5 * (f.con[0] * dx * dx + f.con[2] * dy * dy) - f.con[1] * dx * dy;
        double g = std::exp(power);
        double alpha = f.o * g;
        // the same decisions, in the same order, as composite()
        const bool aclamp = dec.take(alpha > kAlphaMax, near_rel(alpha, kAlphaMax, ma));
        const bool skip = dec.take(alpha < kAlphaMin, near_rel(alpha, kAlphaMin, ma));
        if (aclamp) alpha = kAlphaMax;
        if (skip) continue;
        double Tn = T * (1.0 - alpha);
        if (dec.take(Tn < kTMin, near_rel(Tn, kTMin, mT))) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += f.col[ch] * alpha * T;
        recs.push_back(Rec{ids[k], alpha, T, g, dx, dy, aclamp});
        T = Tn;
    }
    for (int ch = 0; ch < 3; ++ch) Cfinal[ch] = C[ch];
    out.clear();
    double acc[3] = {0.0, 0.0, 0.0};  // colour accumulated up to and including n
    for (const Rec& r : recs) {
        const Feat<double>& f = F[r.id];
        Contrib c;
        c.id = r.id;
        std::memset(c.dC, 0, sizeof(c.dC));
        for (int ch = 0; ch < 3; ++ch) acc[ch] += f.col[ch] * r.alpha * r.T;
        // d alpha / d features (zero where alpha is clamped)
        double da[6] = {0, 0, 0, 0, 0, 0};
        if (!r.aclamp) {
            double dpow = f.o * r.g;  // d alpha / d power
            da[0] = dpow * (-(f.con[0] * r.dx + f.con[1] * r.dy));
            da[1] = dpow * (-(f.con[1] * r.dx + f.con[2] * r.dy));
            da[2] = dpow * (-0.5 * r.dx * r.dx);
            da[3] = dpow * (-r.dx * r.dy);
            da[4] = dpow * (-0.5 * r.dy * r.dy);
            da[5] = r.g;
        }
        for (int ch = 0; ch < 3; ++ch) {
            // later Gaussians see transmittance T_m containing (1 - alpha_n)
            double dCda = r.T * f.col[ch] - (Cfinal[ch] - acc[ch]) / (1.0 - r.alpha);
            for (int k = 0; k < 6; ++k) c.dC[ch][k] = dCda * da[k];
            c.dC[ch][6 + ch] = r.alpha * r.T;
        }
        out.push_back(c);
    }
}

// --------------------------------------------------------------------------
// Sampler: SplitMix64 (Steele, Lea, Flood 2014) and a partial Fisher-Yates
// shuffle per tile (stratified per-tile sampling, Sec. 4.4).
// --------------------------------------------------------------------------
inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
inline uint64_t sm64_next(uint64_t& state) {
    state += 0x9E3779B97F4A7C15ull;
    return sm64_mix(state);
}
uint64_t tile_seed(uint64_t seed, int64_t step, int32_t view, int32_t tile) {
    uint64_t h = sm64_mix(seed ^ 0x5851F42D4C957F2Dull);
    h = sm64_mix(h ^ (uint64_t)step);
    h = sm64_mix(h ^ (uint64_t)(uint32_t)view);
    h = sm64_mix(h ^ (uint64_t)(uint32_t)tile);
    return h;
}
void sample_tile(uint64_t seed, int64_t step, int32_t view, int32_t tile, int n, int k, uint8_t* out) {
    int a[256];
    for (int i = 0; i < n; ++i) a[i] = i;
    uint64_t st = tile_seed(seed, step, view, tile);
    for (int i = 0; i < k; ++i) {
        uint64_t r = sm64_next(st);
        int j = i + (int)(r % (uint64_t)(n - i));
        std::swap(a[i], a[j]);
        out[i] = (uint8_t)a[i];
    }
}
int samples_in_tile(const orc_config& cfg, int n_valid) {
    int k;
    if (cfg.samples_per_tile > 0) k = cfg.samples_per_tile;
    else k = (int)std::floor(cfg.sample_frac * n_valid + 0.5);
    return std::max(1, std::min(k, n_valid));
}

}  // namespace

// ==========================================================================
// Scene
// ==========================================================================
struct orc_scene {
    orc_config cfg;
    int G, deg, K, Pg;
    std::vector<double> params;
    std::vector<orc_camera> cams;
    std::vector<CamD> camd;
    std::vector<CamF> camf;
    std::vector<float> targets;  // [n_cams][H][W][3] or empty
    int W, H, tiles_x, tiles_y, T;
    // step state
    int64_t step;
    std::vector<int> views;            // camera index per slot
    std::vector<int32_t> tile_off;     // [nv*T + 1]
    std::vector<uint8_t> off;          // [S]
    std::vector<double> w;             // [S]
    std::vector<int32_t> spx, spy, sslot, stile;  // per sample
    std::vector<uint8_t> sflag;                   // per sample: an importance draw near a decision
    std::vector<uint32_t> flip;                   // per sample: near decisions taken the other way (Decisions)
    std::vector<double> ssim_s, ssim_d;           // [S][3] SSIM residual and its own-pixel derivative
    std::vector<uint8_t> ssim_flag;               // per sample: a flagged pixel inside its SSIM window
    std::vector<int64_t> ranges;       // [nv*T + 1]
    std::vector<int32_t> ids;          // [Pi]
    std::vector<GeoF> geo;             // [nv*G]
    std::vector<Feat<double>> feat;    // [nv*G]

    int64_t P() const { return (int64_t)G * Pg; }

    Gauss<double> gauss(int g) const {
        Gauss<double> r;
        for (int k = 0; k < 3; ++k) {
            r.X[k] = params[3 * g + k];
            r.ls[k] = params[3 * (int64_t)G + 3 * g + k];
        }
        for (int k = 0; k < 4; ++k) r.q[k] = params[6 * (int64_t)G + 4 * g + k];
        r.th = params[10 * (int64_t)G + g];
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) r.sh[k][ch] = params[11 * (int64_t)G + (int64_t)g * K * 3 + k * 3 + ch];
        return r;
    }
    // index of local parameter j of Gaussian g inside a P-vector
    int64_t pindex(int g, int j) const {
        if (j < 3) return 3 * (int64_t)g + j;
        if (j < 6) return 3 * (int64_t)G + 3 * (int64_t)g + (j - 3);
        if (j < 10) return 6 * (int64_t)G + 4 * (int64_t)g + (j - 6);
        if (j == 10) return 10 * (int64_t)G + g;
        return 11 * (int64_t)G + (int64_t)g * K * 3 + (j - 11);
    }
    Gauss<Dual> gauss_dual(int g, const double* v) const {
        Gauss<double> p = gauss(g);
        Gauss<Dual> r;
        for (int k = 0; k < 3; ++k) {
            r.X[k] = Dual(p.X[k], v ? v[pindex(g, k)] : 0.0);
            r.ls[k] = Dual(p.ls[k], v ? v[pindex(g, 3 + k)] : 0.0);
        }
        for (int k = 0; k < 4; ++k) r.q[k] = Dual(p.q[k], v ? v[pindex(g, 6 + k)] : 0.0);
        r.th = Dual(p.th, v ? v[pindex(g, 10)] : 0.0);
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) r.sh[k][ch] = Dual(p.sh[k][ch], v ? v[pindex(g, 11 + 3 * k + ch)] : 0.0);
        return r;
    }
    // unit tangent on local parameter j
    Gauss<Dual> gauss_unit(int g, int j) const {
        Gauss<double> p = gauss(g);
        Gauss<Dual> r;
        for (int k = 0; k < 3; ++k) {
            r.X[k] = Dual(p.X[k], j == k ? 1.0 : 0.0);
            r.ls[k] = Dual(p.ls[k], j == 3 + k ? 1.0 : 0.0);
        }
        for (int k = 0; k < 4; ++k) r.q[k] = Dual(p.q[k], j == 6 + k ? 1.0 : 0.0);
        r.th = Dual(p.th, j == 10 ? 1.0 : 0.0);
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) r.sh[k][ch] = Dual(p.sh[k][ch], j == 11 + 3 * k + ch ? 1.0 : 0.0);
        return r;
    }
    // preprocessing Jacobian a[f][j] = d feature_f / d local parameter j
    void prep_jacobian(int slot, int g, std::vector<double>& a) const {
        a.assign(9 * (size_t)Pg, 0.0);
        const CamD& c = camd[views[slot]];
        for (int j = 0; j < Pg; ++j) {
            Gauss<Dual> gd = gauss_unit(g, j);
            Feat<Dual> f;
            preprocess<Dual>(gd, deg, c, f);
            double d[9] = {f.mu[0].d, f.mu[1].d, f.con[0].d, f.con[1].d, f.con[2].d, f.o.d,
                           f.col[0].d, f.col[1].d, f.col[2].d};
            for (int k = 0; k < 9; ++k) a[(size_t)k * Pg + j] = d[k];
        }
    }
    // weight of the (sample, channel) row in J^T W J: w_i for the colour
    // residual plus ssim_weight * d^2 w_i for the SSIM residual of the same
    // pixel and channel, whose Jacobian row is d times the colour's
    double row_weight(int64_t i, int ch) const {
        if (ssim_d.empty()) return w[i];
        const double d = ssim_d[3 * i + ch];
        return w[i] * (1.0 + cfg.ssim_weight * d * d);
    }
    int nv() const { return (int)views.size(); }
    int64_t S() const { return (int64_t)off.size(); }
    const int32_t* list(int slot, int tile, int* len) const {
        int64_t b = ranges[(int64_t)slot * T + tile], e = ranges[(int64_t)slot * T + tile + 1];
        *len = (int)(e - b);
        return ids.data() + b;
    }
};

namespace {

void pixel_of(const orc_scene* s, int tile, int o, int* px, int* py) {
    int tx = tile % s->tiles_x, ty = tile / s->tiles_x;
    int vw = std::min(s->cfg.tile_w, s->W - tx * s->cfg.tile_w);
    *px = tx * s->cfg.tile_w + o % vw;
    *py = ty * s->cfg.tile_h + o / vw;
}

void compute_features(orc_scene* s) {
    int nv = s->nv();
    s->feat.assign((size_t)nv * s->G, Feat<double>());
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < (int64_t)nv * s->G; ++i) {
        int slot = (int)(i / s->G), g = (int)(i % s->G);
        if (!s->geo[i].vis) continue;
        preprocess<double>(s->gauss(g), s->deg, s->camd[s->views[slot]], s->feat[i]);
    }
}

void build_lists(orc_scene* s) {
    int nv = s->nv();
    s->geo.assign((size_t)nv * s->G, GeoF());
    std::vector<float> pf(s->params.begin(), s->params.end());
    const int G = s->G;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < (int64_t)nv * G; ++i) {
        int slot = (int)(i / G), g = (int)(i % G);
        s->geo[i] = geom_f32(&pf[3 * (size_t)g], &pf[3 * (size_t)G + 3 * g], &pf[6 * (size_t)G + 4 * g],
                             pf[10 * (size_t)G + g], s->camf[s->views[slot]], s->tiles_x, s->tiles_y, s->cfg.tile_w,
                             s->cfg.tile_h);
    }
    // per (slot, tile): sort entries by (depth bits, Gaussian index)
    std::vector<std::vector<std::pair<uint64_t, int32_t>>> bins((size_t)nv * s->T);
    for (int slot = 0; slot < nv; ++slot)
        for (int g = 0; g < G; ++g) {
            const GeoF& q = s->geo[(size_t)slot * G + g];
            if (!q.vis) continue;
            uint64_t key = ((uint64_t)float_bits(q.depth) << 32) | (uint32_t)g;
            for (int ty = q.y0; ty <= q.y1; ++ty) {
                int sx0 = q.x0, sx1 = q.x1;
                if (s->cfg.list_mode == 0 && !row_span(q, ty, s->cfg.tile_w, s->cfg.tile_h, s->W, s->H, &sx0, &sx1))
                    continue;
                for (int tx = sx0; tx <= sx1; ++tx)
                    bins[(size_t)slot * s->T + ty * s->tiles_x + tx].push_back({key, g});
            }
        }
    s->ranges.assign((size_t)nv * s->T + 1, 0);
    for (size_t b = 0; b < bins.size(); ++b) s->ranges[b + 1] = s->ranges[b] + (int64_t)bins[b].size();
    s->ids.assign((size_t)s->ranges.back(), 0);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < (int64_t)bins.size(); ++b) {
        auto& v = bins[b];
        std::sort(v.begin(), v.end());
        for (size_t k = 0; k < v.size(); ++k) s->ids[s->ranges[b] + k] = v[k].second;
    }
}

void make_samples(orc_scene* s) {
    int nv = s->nv();
    s->tile_off.assign((size_t)nv * s->T + 1, 0);
    s->off.clear(); s->w.clear(); s->spx.clear(); s->spy.clear(); s->sslot.clear(); s->stile.clear();
    uint8_t buf[256];
    for (int slot = 0; slot < nv; ++slot)
        for (int t = 0; t < s->T; ++t) {
            int tx = t % s->tiles_x, ty = t / s->tiles_x;
            int vw = std::min(s->cfg.tile_w, s->W - tx * s->cfg.tile_w);
            int vh = std::min(s->cfg.tile_h, s->H - ty * s->cfg.tile_h);
            int n = vw * vh;
            int k = samples_in_tile(s->cfg, n);
            sample_tile(s->cfg.seed, s->step, s->views[slot], t, n, k, buf);
            double wt = s->cfg.weight_mode == 1 ? (double)n / (double)k : 1.0;
            for (int i = 0; i < k; ++i) {
                int px, py;
                pixel_of(s, t, buf[i], &px, &py);
                s->off.push_back(buf[i]);
                s->w.push_back(wt);
                s->spx.push_back(px);
                s->spy.push_back(py);
                s->sslot.push_back(slot);
                s->stile.push_back(t);
            }
            s->tile_off[(size_t)slot * s->T + t + 1] = s->tile_off[(size_t)slot * s->T + t] + k;
        }
}

// Importance sampling (the q_residual and q_Gaussian distributions of the
// supplementary material, drawn per tile): every valid pixel of the tile is
// rendered; its weight is e^{|r_p|} (|r_p| the Euclidean norm of the RGB
// residual) or the number of Gaussians it composites (all zero: uniform);
// K_t pixels are drawn independently by inverse CDF with the tile's
// SplitMix64 outputs, u_i = (output i >> 11) 2^-53, pixel = the first whose
// cumulative weight exceeds u_i x total; weight total / (K_t x its weight) =
// 1 / (K_t q(p)), the Monte Carlo weight of the sampled-loss estimate.
void make_samples_importance(orc_scene* s) {
    const int nv = s->nv(), mode = s->cfg.sample_dist;
    const size_t nt = (size_t)nv * s->T;
    std::vector<std::vector<uint8_t>> offs(nt), fls(nt);
    std::vector<std::vector<double>> ws(nt);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t vt = 0; vt < (int64_t)nt; ++vt) {
        const int slot = (int)(vt / s->T), t = (int)(vt % s->T);
        const int tx = t % s->tiles_x, ty = t / s->tiles_x;
        const int vw = std::min(s->cfg.tile_w, s->W - tx * s->cfg.tile_w);
        const int vh = std::min(s->cfg.tile_h, s->H - ty * s->cfg.tile_h);
        const int n = vw * vh, k = samples_in_tile(s->cfg, n);
        const int cam = s->views[slot];
        int len;
        const int32_t* ids = s->list(slot, t, &len);
        std::vector<double> a(n), cdf(n);
        bool any_flag = false;
        for (int o = 0; o < n; ++o) {
            int px, py, fl, nc;
            pixel_of(s, t, o, &px, &py);
            double C[3];
            composite<double>(px + 0.5, py + 0.5, ids, len, s->feat.data() + (size_t)slot * s->G, s->cfg.margin_alpha,
                              s->cfg.margin_T, C, nullptr, &fl, &nc);
            any_flag = any_flag || fl != 0;
            if (mode == 1) {
                double r2 = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    const double tg = s->targets.empty() ? 0.0
                                                         : s->targets[(((size_t)cam * s->H + py) * s->W + px) * 3 + ch];
                    r2 += (C[ch] - tg) * (C[ch] - tg);
                }
                a[o] = std::exp(std::sqrt(r2));
            } else {
                a[o] = (double)nc;
            }
        }
        double run = 0.0;
        for (int o = 0; o < n; ++o) cdf[o] = (run += a[o]);
        const double total = run;
        const bool uniform = !(total > 0.0);
        uint64_t h = tile_seed(s->cfg.seed, s->step, cam, t);
        for (int i = 0; i < k; ++i) {
            const double u = (double)(sm64_next(h) >> 11) * (1.0 / 9007199254740992.0);
            int sel;
            double w;
            bool near = false;
            if (uniform) {
                sel = std::min(n - 1, (int)std::floor(u * n));
                w = (double)n / (double)k;
            } else {
                const double thr = u * total;
                sel = n - 1;
                for (int o = 0; o < n; ++o)
                    if (cdf[o] > thr) {
                        sel = o;
                        break;
                    }
                const double m = 1e-5 * total;
                near = std::fabs(cdf[sel] - thr) <= m || (sel > 0 && std::fabs(cdf[sel - 1] - thr) <= m);
                w = total / ((double)k * a[sel]);
            }
            offs[vt].push_back((uint8_t)sel);
            ws[vt].push_back(w);
            fls[vt].push_back((uint8_t)((near || any_flag) ? 1 : 0));
        }
    }
    s->off.clear(); s->w.clear(); s->spx.clear(); s->spy.clear(); s->sslot.clear(); s->stile.clear();
    s->sflag.clear();
    s->tile_off.assign(nt + 1, 0);
    for (size_t vt = 0; vt < nt; ++vt) {
        const int slot = (int)(vt / s->T), t = (int)(vt % s->T);
        for (size_t i = 0; i < offs[vt].size(); ++i) {
            int px, py;
            pixel_of(s, t, offs[vt][i], &px, &py);
            s->off.push_back(offs[vt][i]);
            s->w.push_back(ws[vt][i]);
            s->spx.push_back(px);
            s->spy.push_back(py);
            s->sslot.push_back(slot);
            s->stile.push_back(t);
            s->sflag.push_back(fls[vt][i]);
        }
        s->tile_off[vt + 1] = s->tile_off[vt] + (int32_t)offs[vt].size();
    }
}

// Dual features of every visible pair for a tangent v.
void dual_features(const orc_scene* s, const double* v, std::vector<Feat<Dual>>& fd) {
    int nv = s->nv();
    fd.assign((size_t)nv * s->G, Feat<Dual>());
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < (int64_t)nv * s->G; ++i) {
        int slot = (int)(i / s->G), g = (int)(i % s->G);
        if (!s->geo[i].vis) continue;
        preprocess<Dual>(s->gauss_dual(g, v), s->deg, s->camd[s->views[slot]], fd[i]);
    }
}

// u_i = (J v)_i at sample i (Alg. 3: dual numbers through preprocessing and
// compositing; the tangent of the composited colour).
void jvp_sample(const orc_scene* s, const std::vector<Feat<Dual>>& fd, int64_t i, double u[3]) {
    int slot = s->sslot[i], len;
    const int32_t* ids = s->list(slot, s->stile[i], &len);
    Dual C[3];
    composite<Dual>(s->spx[i] + 0.5, s->spy[i] + 0.5, ids, len, fd.data() + (size_t)slot * s->G,
                    s->cfg.margin_alpha, s->cfg.margin_T, C, nullptr, nullptr, nullptr, s->flip[i]);
    for (int ch = 0; ch < 3; ++ch) u[ch] = C[ch].d;
}

// Accumulate cot[pair][9] += sum_ch ubar_ch dC_ch/dfeat over the samples in
// [i0, i1) whose tiles are listed; returns via a callback per contribution.
template <class Fn>
void for_each_contribution(const orc_scene* s, int64_t i, Fn fn) {
    int slot = s->sslot[i], len;
    const int32_t* ids = s->list(slot, s->stile[i], &len);
    std::vector<Contrib> cs;
    double Cf[3];
    pixel_feature_jacobian(s->spx[i] + 0.5, s->spy[i] + 0.5, ids, len, s->feat.data() + (size_t)slot * s->G, cs, Cf,
                           s->cfg.margin_alpha, s->cfg.margin_T, s->flip[i]);
    for (const Contrib& c : cs) fn(slot, c);
}

// Chain 2D cotangents back to parameters: g_j += sum_f cot_f a[f][j].
void chain_back(const orc_scene* s, int slot, int g, const double* cot, double* out_local) {
    std::vector<double> a;
    s->prep_jacobian(slot, g, a);
    for (int j = 0; j < s->Pg; ++j) {
        double acc = 0.0;
        for (int f = 0; f < 9; ++f) acc += cot[f] * a[(size_t)f * s->Pg + j];
        out_local[j] += acc;
    }
}

// Samples of (slot) lying in the tiles covered by Gaussian g.
template <class Fn>
void samples_of_gaussian(const orc_scene* s, int slot, int g, Fn fn) {
    const GeoF& q = s->geo[(size_t)slot * s->G + g];
    if (!q.vis) return;
    for (int ty = q.y0; ty <= q.y1; ++ty)
        for (int tx = q.x0; tx <= q.x1; ++tx) {
            int t = ty * s->tiles_x + tx;
            int64_t b = s->tile_off[(size_t)slot * s->T + t], e = s->tile_off[(size_t)slot * s->T + t + 1];
            for (int64_t i = b; i < e; ++i) fn(i);
        }
}

// Cotangent of Gaussian g (slot) from ubar over the samples of its tiles.
void gaussian_cotangent(const orc_scene* s, int slot, int g, const double* ubar, double cot[9]) {
    for (int f = 0; f < 9; ++f) cot[f] = 0.0;
    samples_of_gaussian(s, slot, g, [&](int64_t i) {
        for_each_contribution(s, i, [&](int, const Contrib& c) {
            if (c.id != g) return;
            for (int ch = 0; ch < 3; ++ch)
                for (int f = 0; f < 9; ++f) cot[f] += ubar[3 * i + ch] * c.dC[ch][f];
        });
    });
}

// --------------------------------------------------------------------------
// Diagonal SSIM term (supplementary material, "Results with SSIM loss").
// SSIM per channel (Wang et al. 2004): local statistics under an 11 x 11
// Gaussian window, sigma 1.5, weights normalised to sum 1, pixels outside the
// image counting as 0; C1 = 0.01^2, C2 = 0.03^2 for a dynamic range of 1:
//   SSIM = (2 mx my + C1)(2 cxy + C2) / ((mx^2 + my^2 + C1)(vx + vy + C2)).
// The residual of the term is s = 1 - SSIM at every sampled pixel.  The
// diagonal approximation keeps only the dependence of s on the pixel's own
// colour X_i (Zhao et al. 2016 give dSSIM(p)/dX(q) for every q in the
// window; here q = p): with g0 the centre weight, d mx = g0, d E[X^2] =
// 2 g0 X_i, d E[XY] = g0 Y_i.
// --------------------------------------------------------------------------
constexpr int kSsimRad = 5;
constexpr double kSsimSigma = 1.5, kSsimC1 = 0.01 * 0.01, kSsimC2 = 0.03 * 0.03;

struct SsimWindow {
    double g[2 * kSsimRad + 1][2 * kSsimRad + 1];
    SsimWindow() {
        double z = 0.0;
        for (int a = -kSsimRad; a <= kSsimRad; ++a)
            for (int b = -kSsimRad; b <= kSsimRad; ++b) {
                g[a + kSsimRad][b + kSsimRad] = std::exp(-(a * a + b * b) / (2.0 * kSsimSigma * kSsimSigma));
                z += g[a + kSsimRad][b + kSsimRad];
            }
        for (auto& row : g)
            for (double& v : row) v /= z;
    }
};

void ssim_pixel(const double* X, const double* Y, int H, int W, int px, int py, double s[3], double d[3]) {
    static const SsimWindow win;
    for (int ch = 0; ch < 3; ++ch) {
        double mx = 0.0, my = 0.0, xx = 0.0, yy = 0.0, xy = 0.0;
        for (int a = -kSsimRad; a <= kSsimRad; ++a)
            for (int b = -kSsimRad; b <= kSsimRad; ++b) {
                const int y = py + a, x = px + b;
                if (y < 0 || y >= H || x < 0 || x >= W) continue;
                const double g = win.g[a + kSsimRad][b + kSsimRad];
                const double xv = X[((size_t)y * W + x) * 3 + ch], yv = Y[((size_t)y * W + x) * 3 + ch];
                mx += g * xv;
                my += g * yv;
                xx += g * xv * xv;
                yy += g * yv * yv;
                xy += g * xv * yv;
            }
        const double vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
        const double A1 = 2.0 * mx * my + kSsimC1, A2 = 2.0 * cxy + kSsimC2;
        const double B1 = mx * mx + my * my + kSsimC1, B2 = vx + vy + kSsimC2;
        const double ssim = (A1 * A2) / (B1 * B2);
        const double g0 = win.g[kSsimRad][kSsimRad];
        const double xi = X[((size_t)py * W + px) * 3 + ch], yi = Y[((size_t)py * W + px) * 3 + ch];
        const double dA1 = 2.0 * g0 * my, dA2 = 2.0 * g0 * (yi - my);
        const double dB1 = 2.0 * g0 * mx, dB2 = 2.0 * g0 * (xi - mx);
        const double dssim = (dA1 * A2 + A1 * dA2) / (B1 * B2) - ssim * (dB1 * B2 + B1 * dB2) / (B1 * B2);
        s[ch] = 1.0 - ssim;
        d[ch] = -dssim;
    }
}

// Full FP64 frames of the step's views, then s, d and the window flag of
// every sample.
void make_ssim(orc_scene* s) {
    const int64_t S = s->S();
    s->ssim_s.assign(3 * S, 0.0);
    s->ssim_d.assign(3 * S, 0.0);
    s->ssim_flag.assign(S, 0);
    const size_t npx = (size_t)s->H * s->W;
    std::vector<double> img(npx * 3), tgt(npx * 3);
    std::vector<uint8_t> fl(npx);
    for (int slot = 0; slot < s->nv(); ++slot) {
        orc_render_full(s, slot, img.data(), fl.data());
        const int cam = s->views[slot];
        for (size_t k = 0; k < npx * 3; ++k) tgt[k] = s->targets.empty() ? 0.0 : s->targets[(size_t)cam * npx * 3 + k];
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < S; ++i) {
            if (s->sslot[i] != slot) continue;
            ssim_pixel(img.data(), tgt.data(), s->H, s->W, s->spx[i], s->spy[i], &s->ssim_s[3 * i], &s->ssim_d[3 * i]);
            uint8_t f = 0;
            for (int y = std::max(0, s->spy[i] - kSsimRad); y <= std::min(s->H - 1, s->spy[i] + kSsimRad); ++y)
                for (int x = std::max(0, s->spx[i] - kSsimRad); x <= std::min(s->W - 1, s->spx[i] + kSsimRad); ++x)
                    f |= fl[(size_t)y * s->W + x];
            s->ssim_flag[i] = f;
        }
    }
}

}  // namespace

// ==========================================================================
// C API
// ==========================================================================
extern "C" {

orc_scene* orc_create(const orc_config* cfg, int32_t n_gauss, const float* params,
                      const orc_camera* cams, int32_t n_cams, const float* targets) {
    if (!cfg || n_gauss <= 0 || !params || !cams || n_cams <= 0) return nullptr;
    if (cfg->sh_degree < 0 || cfg->sh_degree > 3) return nullptr;
    if (cfg->tile_w <= 0 || cfg->tile_h <= 0 || cfg->tile_w * cfg->tile_h > 256) return nullptr;
    if (cfg->sample_dist < 0 || cfg->sample_dist > 2 || !(cfg->ssim_weight >= 0.0)) return nullptr;
    orc_scene* s = new orc_scene();
    s->cfg = *cfg;
    s->G = n_gauss;
    s->deg = cfg->sh_degree;
    s->K = (s->deg + 1) * (s->deg + 1);
    s->Pg = 11 + 3 * s->K;
    s->params.assign(params, params + s->P());
    s->cams.assign(cams, cams + n_cams);
    for (auto& c : s->cams) {
        s->camd.push_back(cam_double(c));
        s->camf.push_back(cam_float(c));
    }
    s->W = cams[0].width;
    s->H = cams[0].height;
    for (auto& c : s->cams)
        if (c.width != s->W || c.height != s->H) { delete s; return nullptr; }
    s->tiles_x = (s->W + cfg->tile_w - 1) / cfg->tile_w;
    s->tiles_y = (s->H + cfg->tile_h - 1) / cfg->tile_h;
    s->T = s->tiles_x * s->tiles_y;
    if (targets) s->targets.assign(targets, targets + (size_t)n_cams * s->W * s->H * 3);
    s->step = 0;
    return s;
}

void orc_destroy(orc_scene* s) { delete s; }

int32_t orc_set_params(orc_scene* s, const double* p) {
    std::copy(p, p + s->P(), s->params.begin());
    return 0;
}
int32_t orc_get_params(const orc_scene* s, double* p) {
    std::copy(s->params.begin(), s->params.end(), p);
    return 0;
}
int64_t orc_num_params(const orc_scene* s) { return s->P(); }

int32_t orc_begin_step(orc_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step) {
    if (n_views <= 0) return 1;
    s->views.assign(view_ids, view_ids + n_views);
    for (int v : s->views)
        if (v < 0 || v >= (int)s->cams.size()) return 1;
    s->step = lm_step;
    make_samples(s);
    build_lists(s);
    compute_features(s);
    if (s->cfg.sample_dist != 0) make_samples_importance(s);  // needs the lists and features
    else s->sflag.assign(s->off.size(), 0);
    s->flip.assign(s->off.size(), 0u);
    if (s->cfg.ssim_weight > 0.0) make_ssim(s);
    else {
        s->ssim_s.clear();
        s->ssim_d.clear();
        s->ssim_flag.clear();
    }
    return 0;
}

int64_t orc_num_samples(const orc_scene* s) { return s->S(); }

int32_t orc_get_samples(const orc_scene* s, uint8_t* off, int32_t* tile_off, double* w,
                        int32_t* px, int32_t* py, int32_t* slot) {
    for (int64_t i = 0; i < s->S(); ++i) {
        if (off) off[i] = s->off[i];
        if (w) w[i] = s->w[i];
        if (px) px[i] = s->spx[i];
        if (py) py[i] = s->spy[i];
        if (slot) slot[i] = s->sslot[i];
    }
    if (tile_off) std::copy(s->tile_off.begin(), s->tile_off.end(), tile_off);
    return 0;
}

int32_t orc_get_sample_flags(const orc_scene* s, uint8_t* flags) {
    std::copy(s->sflag.begin(), s->sflag.end(), flags);
    return 0;
}

int32_t orc_get_ssim(const orc_scene* s, double* s_out, double* d_out, uint8_t* flags) {
    const int64_t S = s->S();
    const bool on = !s->ssim_s.empty();
    for (int64_t k = 0; k < 3 * S; ++k) {
        if (s_out) s_out[k] = on ? s->ssim_s[k] : 0.0;
        if (d_out) d_out[k] = on ? s->ssim_d[k] : 0.0;
    }
    if (flags)
        for (int64_t i = 0; i < S; ++i) flags[i] = on ? s->ssim_flag[i] : 0;
    return 0;
}

int64_t orc_num_pairs(const orc_scene* s) { return (int64_t)s->ids.size(); }

int32_t orc_get_lists(const orc_scene* s, int32_t* ranges, int32_t* ids) {
    if (ranges)
        for (size_t b = 0; b + 1 < s->ranges.size(); ++b) {
            ranges[2 * b] = (int32_t)s->ranges[b];
            ranges[2 * b + 1] = (int32_t)s->ranges[b + 1];
        }
    if (ids) std::copy(s->ids.begin(), s->ids.end(), ids);
    return 0;
}

int32_t orc_get_geom(const orc_scene* s, int32_t slot, int32_t* vis, float* depth, int32_t* rect) {
    for (int g = 0; g < s->G; ++g) {
        const GeoF& q = s->geo[(size_t)slot * s->G + g];
        vis[g] = q.vis;
        depth[g] = q.depth;
        rect[4 * g + 0] = q.x0; rect[4 * g + 1] = q.x1;
        rect[4 * g + 2] = q.y0; rect[4 * g + 3] = q.y1;
    }
    return 0;
}

int32_t orc_get_features(const orc_scene* s, int32_t slot, double* feat) {
    for (int g = 0; g < s->G; ++g) {
        const Feat<double>& f = s->feat[(size_t)slot * s->G + g];
        double* o = feat + 9 * (size_t)g;
        o[0] = f.mu[0]; o[1] = f.mu[1]; o[2] = f.con[0]; o[3] = f.con[1]; o[4] = f.con[2];
        o[5] = f.o; o[6] = f.col[0]; o[7] = f.col[1]; o[8] = f.col[2];
    }
    return 0;
}

static void render_one(const orc_scene* s, int64_t i, double* rgb, uint8_t* flag, int* n_near = nullptr) {
    int slot = s->sslot[i], len, fl;
    const int32_t* ids = s->list(slot, s->stile[i], &len);
    double C[3];
    composite<double>(s->spx[i] + 0.5, s->spy[i] + 0.5, ids, len, s->feat.data() + (size_t)slot * s->G,
                      s->cfg.margin_alpha, s->cfg.margin_T, C, nullptr, &fl, nullptr, s->flip[i], n_near);
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch];
    if (flag) *flag = (uint8_t)fl;
}

int32_t orc_set_flips(orc_scene* s, const int64_t* idx, const uint32_t* masks, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        if (idx[k] < 0 || idx[k] >= s->S()) return 1;
        s->flip[idx[k]] = masks[k];
    }
    return 0;
}

int32_t orc_clear_flips(orc_scene* s) {
    std::fill(s->flip.begin(), s->flip.end(), 0u);
    return 0;
}

int32_t orc_sample_outcomes(const orc_scene* s, const double* v, const int64_t* idx, int64_t n, int32_t max_bits,
                            int32_t* n_near, double* rgb, double* u) {
    if (max_bits < 0 || max_bits > 8) return 1;
    const int64_t M = (int64_t)1 << max_bits;
    std::vector<Feat<Dual>> fd;
    dual_features(s, v, fd);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < n; ++k) {
        const int64_t i = idx[k];
        int slot = s->sslot[i], len, nn = 0;
        const int32_t* ids = s->list(slot, s->stile[i], &len);
        const double pcx = s->spx[i] + 0.5, pcy = s->spy[i] + 0.5;
        double C[3];
        composite<double>(pcx, pcy, ids, len, s->feat.data() + (size_t)slot * s->G, s->cfg.margin_alpha,
                          s->cfg.margin_T, C, nullptr, nullptr, nullptr, 0u, &nn);
        n_near[k] = nn;
        const int64_t mk = (int64_t)1 << std::min(nn, (int)max_bits);
        for (int64_t m = 0; m < M; ++m) {
            double* r = rgb + 3 * (k * M + m);
            double* d = u + 3 * (k * M + m);
            if (m >= mk) {
                for (int ch = 0; ch < 3; ++ch) r[ch] = d[ch] = std::nan("");
                continue;
            }
            composite<double>(pcx, pcy, ids, len, s->feat.data() + (size_t)slot * s->G, s->cfg.margin_alpha,
                              s->cfg.margin_T, C, nullptr, nullptr, nullptr, (uint32_t)m);
            Dual Cd[3];
            composite<Dual>(pcx, pcy, ids, len, fd.data() + (size_t)slot * s->G, s->cfg.margin_alpha,
                            s->cfg.margin_T, Cd, nullptr, nullptr, nullptr, (uint32_t)m);
            for (int ch = 0; ch < 3; ++ch) {
                r[ch] = C[ch];
                d[ch] = Cd[ch].d;
            }
        }
    }
    return 0;
}

int32_t orc_near_counts(const orc_scene* s, const int64_t* idx, int64_t n, int32_t* counts) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
        double c[3];
        int nn = 0;
        render_one(s, idx[k], c, nullptr, &nn);
        counts[k] = nn;
    }
    return 0;
}

int32_t orc_render_samples(const orc_scene* s, double* rgb, double* resid, uint8_t* flags) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < s->S(); ++i) {
        double c[3];
        render_one(s, i, c, flags ? flags + i : nullptr);
        for (int ch = 0; ch < 3; ++ch) {
            if (rgb) rgb[3 * i + ch] = c[ch];
            if (resid) {
                double tgt = 0.0;
                if (!s->targets.empty()) {
                    int cam = s->views[s->sslot[i]];
                    tgt = s->targets[(((size_t)cam * s->H + s->spy[i]) * s->W + s->spx[i]) * 3 + ch];
                }
                resid[3 * i + ch] = c[ch] - tgt;  // r_i = I_hat_i - I_i (Eq. 7)
            }
        }
    }
    return 0;
}

int32_t orc_render_samples_subset(const orc_scene* s, const int64_t* idx, int64_t n, double* rgb, uint8_t* flags) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) render_one(s, idx[k], rgb + 3 * k, flags ? flags + k : nullptr);
    return 0;
}

int32_t orc_render_full(const orc_scene* s, int32_t slot, double* img, uint8_t* flags) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < s->H; ++py)
        for (int px = 0; px < s->W; ++px) {
            int t = (py / s->cfg.tile_h) * s->tiles_x + px / s->cfg.tile_w, len, fl;
            const int32_t* ids = s->list(slot, t, &len);
            double C[3];
            composite<double>(px + 0.5, py + 0.5, ids, len, s->feat.data() + (size_t)slot * s->G,
                              s->cfg.margin_alpha, s->cfg.margin_T, C, nullptr, &fl);
            for (int ch = 0; ch < 3; ++ch) img[((size_t)py * s->W + px) * 3 + ch] = C[ch];
            if (flags) flags[(size_t)py * s->W + px] = (uint8_t)fl;
        }
    return 0;
}

// The same frame with the preprocessing and the compositing in binary32
// (Feat<float>, composite<float>: every operation rounded to float, the
// decisions taken on the float values) over the same lists: what FP32
// arithmetic alone does to a pixel, against the FP64 frame.  Not a model of
// any particular FP32 implementation's operation order.
int32_t orc_render_full_f32(const orc_scene* s, int32_t slot, double* img) {
    std::vector<Feat<float>> ff((size_t)s->G);
    for (int g = 0; g < s->G; ++g) {
        const Gauss<double> gd = s->gauss(g);
        Gauss<float> gf;
        for (int k = 0; k < 3; ++k) gf.X[k] = (float)gd.X[k], gf.ls[k] = (float)gd.ls[k];
        for (int k = 0; k < 4; ++k) gf.q[k] = (float)gd.q[k];
        gf.th = (float)gd.th;
        for (int k = 0; k < 16; ++k)
            for (int ch = 0; ch < 3; ++ch) gf.sh[k][ch] = (float)gd.sh[k][ch];
        preprocess<float>(gf, s->deg, s->camd[s->views[slot]], ff[g]);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < s->H; ++py)
        for (int px = 0; px < s->W; ++px) {
            int t = (py / s->cfg.tile_h) * s->tiles_x + px / s->cfg.tile_w, len, fl;
            const int32_t* ids = s->list(slot, t, &len);
            float C[3];
            composite<float>(px + 0.5, py + 0.5, ids, len, ff.data(), s->cfg.margin_alpha, s->cfg.margin_T, C,
                             nullptr, &fl);
            for (int ch = 0; ch < 3; ++ch) img[((size_t)py * s->W + px) * 3 + ch] = C[ch];
        }
    return 0;
}

int32_t orc_pixel_counts(const orc_scene* s, int32_t slot, int32_t* counts) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < s->H; ++py)
        for (int px = 0; px < s->W; ++px) {
            int t = (py / s->cfg.tile_h) * s->tiles_x + px / s->cfg.tile_w, len, nc;
            const int32_t* ids = s->list(slot, t, &len);
            double C[3];
            composite<double>(px + 0.5, py + 0.5, ids, len, s->feat.data() + (size_t)slot * s->G,
                              s->cfg.margin_alpha, s->cfg.margin_T, C, nullptr, nullptr, &nc);
            counts[(size_t)py * s->W + px] = nc;
        }
    return 0;
}

int32_t orc_jvp(const orc_scene* s, const double* v, double* u) {
    std::vector<Feat<Dual>> fd;
    dual_features(s, v, fd);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < s->S(); ++i) jvp_sample(s, fd, i, u + 3 * i);
    return 0;
}

int32_t orc_jvp_subset(const orc_scene* s, const double* v, const int64_t* idx, int64_t n, double* u) {
    std::vector<Feat<Dual>> fd;
    dual_features(s, v, fd);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) jvp_sample(s, fd, idx[k], u + 3 * k);
    return 0;
}

// g = J^T u: per-pixel reverse pass, then the per-(view, Gaussian) 2D
// cotangents are chained back through the preprocessing Jacobian.
int32_t orc_vjp(const orc_scene* s, const double* u, double* g) {
    const int nv = s->nv(), G = s->G;
    std::vector<double> cot((size_t)nv * G * 9, 0.0);
    for (int64_t i = 0; i < s->S(); ++i)
        for_each_contribution(s, i, [&](int slot, const Contrib& c) {
            double* dst = &cot[((size_t)slot * G + c.id) * 9];
            for (int ch = 0; ch < 3; ++ch)
                for (int f = 0; f < 9; ++f) dst[f] += u[3 * i + ch] * c.dC[ch][f];
        });
    std::fill(g, g + s->P(), 0.0);
#pragma omp parallel for schedule(dynamic, 64)
    for (int gi = 0; gi < G; ++gi) {
        std::vector<double> loc(s->Pg, 0.0);
        for (int slot = 0; slot < nv; ++slot) {
            if (!s->geo[(size_t)slot * G + gi].vis) continue;
            chain_back(s, slot, gi, &cot[((size_t)slot * G + gi) * 9], loc.data());
        }
        for (int j = 0; j < s->Pg; ++j) g[s->pindex(gi, j)] = loc[j];
    }
    return 0;
}

int32_t orc_vjp_gauss(const orc_scene* s, const double* u, const int32_t* gids, int32_t n, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n; ++k) {
        std::vector<double> loc(s->Pg, 0.0);
        for (int slot = 0; slot < s->nv(); ++slot) {
            double cot[9];
            gaussian_cotangent(s, slot, gids[k], u, cot);
            if (s->geo[(size_t)slot * s->G + gids[k]].vis) chain_back(s, slot, gids[k], cot, loc.data());
        }
        for (int j = 0; j < s->Pg; ++j) out[(size_t)k * s->Pg + j] = loc[j];
    }
    return 0;
}

// D_j = sum_i w_i J_ij^2 (w_i the row weight), accumulated row by row: each (sample, channel) row
// of J restricted to one Gaussian is dC/dfeatures times the preprocessing
// Jacobian (no Gram factorisation here).
static void diag_local(const orc_scene* s, int slot, int g, double* out_local) {
    std::vector<double> a;
    s->prep_jacobian(slot, g, a);
    samples_of_gaussian(s, slot, g, [&](int64_t i) {
        for_each_contribution(s, i, [&](int, const Contrib& c) {
            if (c.id != g) return;
            for (int ch = 0; ch < 3; ++ch)
                for (int j = 0; j < s->Pg; ++j) {
                    double Jij = 0.0;
                    for (int f = 0; f < 9; ++f) Jij += c.dC[ch][f] * a[(size_t)f * s->Pg + j];
                    out_local[j] += s->row_weight(i, ch) * Jij * Jij;
                }
        });
    });
}

// Magnitude of the same rows: sum over (sample, channel) of w (sum_f
// |dC_ch/dfeature_f a[f][j]|)^2, the scale against which a floating-point
// evaluation of each row's chain rule rounds (an FP32 evaluation of D_j has
// an error of order u sqrt(D_j M_j) by Cauchy-Schwarz, u = 2^-24).
static void diag_mag_local(const orc_scene* s, int slot, int g, double* out_local) {
    std::vector<double> a;
    s->prep_jacobian(slot, g, a);
    samples_of_gaussian(s, slot, g, [&](int64_t i) {
        for_each_contribution(s, i, [&](int, const Contrib& c) {
            if (c.id != g) return;
            for (int ch = 0; ch < 3; ++ch)
                for (int j = 0; j < s->Pg; ++j) {
                    double m = 0.0;
                    for (int f = 0; f < 9; ++f) m += std::fabs(c.dC[ch][f] * a[(size_t)f * s->Pg + j]);
                    out_local[j] += s->row_weight(i, ch) * m * m;
                }
        });
    });
}

int32_t orc_diag_magnitude(const orc_scene* s, double* M) {
    std::fill(M, M + s->P(), 0.0);
#pragma omp parallel for schedule(dynamic, 8)
    for (int g = 0; g < s->G; ++g) {
        std::vector<double> loc(s->Pg, 0.0);
        for (int slot = 0; slot < s->nv(); ++slot) diag_mag_local(s, slot, g, loc.data());
        for (int j = 0; j < s->Pg; ++j) M[s->pindex(g, j)] = loc[j];
    }
    return 0;
}

int32_t orc_diag(const orc_scene* s, double* D) {
    std::fill(D, D + s->P(), 0.0);
#pragma omp parallel for schedule(dynamic, 8)
    for (int g = 0; g < s->G; ++g) {
        std::vector<double> loc(s->Pg, 0.0);
        for (int slot = 0; slot < s->nv(); ++slot) diag_local(s, slot, g, loc.data());
        for (int j = 0; j < s->Pg; ++j) D[s->pindex(g, j)] = loc[j];
    }
    return 0;
}

int32_t orc_diag_gauss(const orc_scene* s, const int32_t* gids, int32_t n, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n; ++k) {
        std::vector<double> loc(s->Pg, 0.0);
        for (int slot = 0; slot < s->nv(); ++slot) diag_local(s, slot, gids[k], loc.data());
        for (int j = 0; j < s->Pg; ++j) out[(size_t)k * s->Pg + j] = loc[j];
    }
    return 0;
}

// A v = J^T W J v + lambda * (v or D v)   (Eq. 8; damping per the config)
int32_t orc_apply(const orc_scene* s, const double* v, const double* D, double* out) {
    std::vector<double> u((size_t)s->S() * 3);
    orc_jvp(s, v, u.data());
    for (int64_t i = 0; i < s->S(); ++i)
        for (int ch = 0; ch < 3; ++ch) u[3 * i + ch] *= s->row_weight(i, ch);
    orc_vjp(s, u.data(), out);
    for (int64_t j = 0; j < s->P(); ++j)
        out[j] += s->cfg.lambda * (s->cfg.damping_mode == 1 ? D[j] : 1.0) * v[j];
    return 0;
}

int32_t orc_apply_gauss(const orc_scene* s, const double* v, const double* D,
                        const int32_t* gids, int32_t n, double* out) {
    std::vector<double> u((size_t)s->S() * 3);
    orc_jvp(s, v, u.data());
    for (int64_t i = 0; i < s->S(); ++i)
        for (int ch = 0; ch < 3; ++ch) u[3 * i + ch] *= s->row_weight(i, ch);
    orc_vjp_gauss(s, u.data(), gids, n, out);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < s->Pg; ++j) {
            int64_t p = s->pindex(gids[k], j);
            out[(size_t)k * s->Pg + j] += s->cfg.lambda * (s->cfg.damping_mode == 1 ? D[p] : 1.0) * v[p];
        }
    return 0;
}

// b = J^T W r   (right-hand side of Eq. 8, Eq. 14 without the constant);
// with the SSIM term the stacked residual adds ssim_weight * d * s per row.
int32_t orc_rhs(const orc_scene* s, double* b) {
    std::vector<double> r((size_t)s->S() * 3);
    orc_render_samples(s, nullptr, r.data(), nullptr);
    const bool ssim = !s->ssim_s.empty();
    for (int64_t i = 0; i < s->S(); ++i)
        for (int ch = 0; ch < 3; ++ch) {
            const double e = ssim ? s->cfg.ssim_weight * s->ssim_d[3 * i + ch] * s->ssim_s[3 * i + ch] : 0.0;
            r[3 * i + ch] = s->w[i] * (r[3 * i + ch] + e);
        }
    return orc_vjp(s, r.data(), b);
}

// Jacobi preconditioner M^-1 = 1 / diag(A) (Sec. 4.2); 0 where the column is empty
// under the diagonal damping.
int32_t orc_precond(const orc_scene* s, const double* D, double* minv) {
    for (int64_t j = 0; j < s->P(); ++j) {
        double d = s->cfg.damping_mode == 1 ? (1.0 + s->cfg.lambda) * D[j] : D[j] + s->cfg.lambda;
        minv[j] = d > 0.0 ? 1.0 / d : 0.0;
    }
    return 0;
}

// Preconditioned CG of Alg. 1: x0 = 0, r0 = b, z0 = M^-1 r0, p0 = z0, then
// `iters` applications of A.
int32_t orc_cg(const orc_scene* s, const double* b, const double* D, int32_t iters, double* x, double* stats) {
    const int64_t P = s->P();
    std::vector<double> r(b, b + P), z(P), p(P), u(P), minv(P);
    orc_precond(s, D, minv.data());
    for (int64_t j = 0; j < P; ++j) { z[j] = minv[j] * r[j]; p[j] = z[j]; x[j] = 0.0; }
    double rz = 0.0;
    for (int64_t j = 0; j < P; ++j) rz += r[j] * z[j];
    if (stats) stats[0] = rz;
    for (int it = 0; it < iters; ++it) {
        orc_apply(s, p.data(), D, u.data());
        double pu = 0.0;
        for (int64_t j = 0; j < P; ++j) pu += p[j] * u[j];
        double alpha = rz / pu;
        for (int64_t j = 0; j < P; ++j) {
            x[j] += alpha * p[j];
            r[j] -= alpha * u[j];
            z[j] = minv[j] * r[j];
        }
        double rz_new = 0.0;
        for (int64_t j = 0; j < P; ++j) rz_new += r[j] * z[j];
        double beta = rz_new / rz;
        for (int64_t j = 0; j < P; ++j) p[j] = z[j] + beta * p[j];
        rz = rz_new;
        if (stats) { stats[2 + 2 * it] = alpha; stats[3 + 2 * it] = beta; }
    }
    if (stats) {
        double rr = 0.0;
        for (int64_t j = 0; j < P; ++j) rr += r[j] * r[j];
        stats[1] = std::sqrt(rr);
    }
    return 0;
}

// Step size of Sec. 4.5 / App. D: a fixed warm-up rate, then the largest
// rate that keeps every colour (SH degree-0) update within the bound, capped.
double orc_step_size(const orc_scene* s, const double* x, int64_t lm_step) {
    if (lm_step < s->cfg.warm_iters) return s->cfg.lr_warm;
    double m = 0.0;
    for (int g = 0; g < s->G; ++g)
        for (int ch = 0; ch < 3; ++ch) m = std::max(m, std::fabs(x[s->pindex(g, 11 + ch)]));
    if (m == 0.0) return s->cfg.lr_cap;
    return std::min(s->cfg.lr_cap, s->cfg.color_bound / m);
}

// One LM step (Alg. 1).  The update is beta <- beta - eta x with x solving
// A x = J^T W r (the descent reading of Eq. 8 with r = I_hat - I).
int32_t orc_lm_step(orc_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step,
                    double* x_out, double* stats) {
    if (orc_begin_step(s, view_ids, n_views, lm_step)) return 1;
    const int64_t P = s->P();
    std::vector<double> r((size_t)s->S() * 3);
    orc_render_samples(s, nullptr, r.data(), nullptr);
    double se = 0.0, sw = 0.0;
    for (int64_t i = 0; i < s->S(); ++i) {
        for (int ch = 0; ch < 3; ++ch) {
            se += s->w[i] * r[3 * i + ch] * r[3 * i + ch];
            if (!s->ssim_s.empty()) se += s->w[i] * s->cfg.ssim_weight * s->ssim_s[3 * i + ch] * s->ssim_s[3 * i + ch];
        }
        sw += 3.0 * s->w[i];
    }
    std::vector<double> b(P), D(P), x(P);
    orc_rhs(s, b.data());
    orc_diag(s, D.data());
    orc_cg(s, b.data(), D.data(), s->cfg.cg_iters, x.data(), nullptr);
    double eta = orc_step_size(s, x.data(), lm_step);
    double m = 0.0;
    for (int g = 0; g < s->G; ++g)
        for (int ch = 0; ch < 3; ++ch) m = std::max(m, std::fabs(x[s->pindex(g, 11 + ch)]));
    for (int64_t j = 0; j < P; ++j) s->params[j] -= eta * x[j];
    if (x_out) std::copy(x.begin(), x.end(), x_out);
    if (stats) { stats[0] = se / sw; stats[1] = eta; stats[2] = m; }
    return 0;
}

void orc_sh_basis(int32_t deg, double x, double y, double z, double* Y) { sh_basis<double>(deg, x, y, z, Y); }

void orc_ssim_pixel(const double* X, const double* Y, int32_t H, int32_t W, int32_t px, int32_t py, double* s,
                    double* d) {
    ssim_pixel(X, Y, H, W, px, py, s, d);
}

void orc_splitmix64(uint64_t state, int32_t n, uint64_t* out) {
    for (int i = 0; i < n; ++i) out[i] = sm64_next(state);
}

uint64_t orc_tile_seed(uint64_t seed, int64_t lm_step, int32_t view_id, int32_t tile_id) {
    return tile_seed(seed, lm_step, view_id, tile_id);
}

void orc_sample_tile(uint64_t seed, int64_t lm_step, int32_t view_id, int32_t tile_id,
                     int32_t n_valid, int32_t k, uint8_t* out) {
    sample_tile(seed, lm_step, view_id, tile_id, n_valid, k, out);
}

int32_t orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
