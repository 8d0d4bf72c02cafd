// Internal declarations shared by the CUDA translation units of liblmrs.
#pragma once

#include <cuda_runtime.h>
#include <vector>
#include <cuda_bf16.h>
#include <stdint.h>

#include "lmrs.h"

namespace lmrs {

constexpr int kWarp = 32;
constexpr int kMaxShCoeffs = 16;
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip threshold
constexpr float kAlphaMax = 0.99f;          // alpha clamp
constexpr float kTMin = 1e-4f;              // termination threshold
constexpr int kRecF4 = 6;                   // float4 per staged (view, Gaussian) record: primal, tangent
constexpr int kPrimF4 = 3;                  // float4 of a pair's primal 2D features
constexpr int kTanF4 = 3;                   // float4 of a pair's 2D feature tangent
constexpr int kCotF = 12;                   // floats per (view, Gaussian) cotangent slot (9 used)
constexpr int kDiagF = 16;                  // floats per (view, Gaussian) slot of diag(J^T W J) rows (14 used)
constexpr int kMaxPartials = 4096;          // block partials of the FP64 reductions
constexpr int kGaussF4 = 9;                  // float4 planes of the per-Gaussian cache
// float4 planes of the per-pair Jacobian cache for SH degree 0..3: screen mean
// 2x3, conic 3x10, opacity slope, clamp mask (38 floats), plus for degree >= 1
// the colour-through-direction block 3x3 (47)
__host__ __device__ constexpr int jac_f4(int deg) { return deg == 0 ? 10 : 12; }

// Camera as the kernels read it.  R, t, fx, fy, cx, cy, limx, limy, znear are
// the FP32 values the list decisions use.
struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float limx, limy;
    float znear;
    float centre[3];
    int W, H;
};

// Device scalars of the solver (FP64), one block in device memory.  The CG
// part (up to loss_num) is reset by every solve; the LM part by its users.
struct Scalars {
    double rz;       // r^T z of the current iterate
    double rz_new;
    double pAp;
    double alpha;
    double beta;
    double rz0;
    unsigned int numeric_error;
    unsigned int pad0;
    double alpha_hist[64];
    double beta_hist[64];
    // LM step
    double loss_num;  // sum w |r|^2
    double loss_den;  // sum 3 w
    unsigned long long n_eval;  // (sample, Gaussian) pairs composited before termination
    unsigned long long n_walk;  // compact-list entries over all work items (walked by the derivative kernels)
    double eta;
    unsigned int max_dc_bits;  // bits of max |x_dc| (non-negative float)
    unsigned int pad1;
    // preprocessing
    unsigned int n_list;  // tile-list entries of the step (written by the binning)
    unsigned int debug_err;  // LMRS_DEBUG builds: bit k set by a failed check k (lmrs_debug_status)
};

// Index checks of LMRS_DEBUG builds: an index outside [0, n) sets bit `bit`
// of the scene's debug word and is replaced by 0, so that the access it
// guards stays in bounds.  Release builds compile the check away.
#ifdef LMRS_DEBUG
#define LMRS_DCHECK_INDEX(c, idx, n, bit)                                                 \
    do {                                                                                  \
        if ((unsigned long long)(idx) >= (unsigned long long)(n)) {                       \
            atomicOr(&(c).sc->debug_err, 1u << (bit));                                    \
            (idx) = 0;                                                                    \
        }                                                                                 \
    } while (0)
#else
#define LMRS_DCHECK_INDEX(c, idx, n, bit) \
    do {                                  \
    } while (0)
#endif
enum { kCheckStagedId = 0, kCheckCompactWrite = 1, kCheckScatterId = 2 };

// Everything a kernel needs to know about the scene and the current step.
struct Ctx {
    int G, deg, K, Pg;
    long long P;
    int nv, W, H, tiles_x, tiles_y, T, tile_w, tile_h;
    int cache_bf16;
    int damping_mode;
    float lambda;
    const float* params;
    const CamDev* cams;     // indexed by camera id
    const int* views;       // camera id per slot
    const float* targets;   // [n_cams][H][W][3] or null
    // per (slot, Gaussian) pair, index slot * G + g
    float4* gcache;         // per Gaussian, kGaussF4 planes of G float4 (view-independent 3D state)
    float4* rec;            // per pair kPrimF4 float4: mu_x, mu_y, A, B | C, o, r, g | b, B', A', C' with
                            // (A', B', C') = -log2(e) (A / 2, B, C / 2): e^power = 2^(dx (A' dx + B' dy) + C' dy^2)
    float4* tan;            // per pair kTanF4 float4: the tangents of the 9 features of pjac
    float4* pjac;           // per (view, Gaussian) pair: jac_f4(deg) planes of nv*G float4, the Jacobian
                            // of the pair's 9 screen-space features (jac.cuh) w.r.t. its parameters
    int4* rect;             // inclusive tile rectangle, x0 > x1 when culled
    float4* ell;            // per pair 2 float4: the alpha >= 1/255 ellipse that picks each rectangle
                            // row's tile columns (row_span)
    unsigned long long* dkeys;  // (slot << 32 | depth bits, or all ones when culled), sorted in place
    unsigned int* dvals;        // Gaussian index of each depth key
    unsigned long long* cnt;  // tiles touched per depth-sorted pair (then exclusive prefix)
    unsigned long long* n_visible;  // count of visible pairs
    unsigned long long* n_entries;  // bound on the tile-list entries: band rows x rectangle width
    unsigned long long* n_rowent;   // sum over visible pairs of the rectangle rows band_meets keeps
    float* cot;             // kCotF floats: cotangents of the 9 features of pjac
    float* dslot;           // kDiagF floats: the pair's share of diag(J^T W J) (k_diag)
    // binning
    unsigned int* keys;     // slot * T + tile of each list entry
    unsigned int* ids;
    long long npairs;
    int2* ranges;           // [nv * T] begin, end
    // sampling
    const int* tile_off;    // [nv * T + 1]
    unsigned char* off;     // [S]
    const float* wtile;     // [nv * T]
    float* wsample;         // [S] per-sample weights (importance sampling), else null
    int sample_dist;
    // diagonal SSIM term (null when off): per (sample, channel) s = 1 - SSIM
    // and d = ds/dC; rows of J^T W J weigh w (1 + ssim_weight d^2)
    float* ssim_s;          // [S][3]
    float* ssim_d;          // [S][3]
    float ssim_weight;
    const float* frames;    // [nv][H][W][3] full renders of the step's views (SSIM windows)
    long long S;
    const int2* work;       // (slot * T + tile, first sample in tile) per warp item
    int nwork;
    int* item_cost;         // [nwork] list entries a work item traverses (from the forward render)
    // compact lists (written by the forward render): the entries a work item's
    // pixels need; chunk q of tile vt at max_items * begin(vt) + q * len(vt)
    unsigned int* cids;     // [max_items * npairs]
    int* clen;              // [nv * T * max_items]
    int max_items;          // largest number of 32-sample chunks in a tile
    // per-sample caches
    float* resid;           // [S][3]
    float* cacheC;          // [S][3] FP32 (or BF16 in cacheCh)
    float* cacheT;          // [S]
    __nv_bfloat16* cacheCh; // [S][3]
    __nv_bfloat16* cacheTh; // [S]
    int* cacheN;            // [S] list position where compositing stopped
    Scalars* sc;
    double* partials;
    unsigned int* counter;
};

// ---- batches of scenes ----------------------------------------------------
constexpr int kMaxBatchIters = 64;  // CG iterations a batch step can run
constexpr int kBatchBlock = 128;    // block size of the batched kernels
constexpr int kVecChunk = 2048;     // vector entries per chunk

// Per-scene vectors, solver history and step-size settings of a batch.
struct BatchVec {
    float *b, *x, *r, *z, *p, *Ap, *minv, *D, *params;
    double* rz;   // [kMaxBatchIters + 1]: r_i^T z_i
    double* pAp;  // [kMaxBatchIters]: p_i^T A p_i
    long long P;
    long long lm_step;
    double lr_warm, lr_cap, color_bound;
    int warm_iters;
};

// Segment tables of a batch: chunks (scene, begin, end) that never cross a
// scene, one chunk per block iteration; counts live in device memory so a
// captured graph replays with new contents.
struct BatchTables {
    const Ctx* ctxs;
    const BatchVec* vecs;
    const int4* gchunks;  // Gaussians, <= kBatchBlock per chunk
    const int4* vchunks;  // P-vector entries, <= kVecChunk
    const int4* wchunks;  // raster work items, <= kBatchBlock / 32
    const int* counts;    // [3]: number of g, v, w chunks
};

// ---- launch count (every kernel launch goes through note_launch) --------
void note_launch();

// ---- preprocess.cu --------------------------------------------------------
void set_sh_constants();
void launch_sample(const Ctx& c, long long lm_step, unsigned long long seed, cudaStream_t st);
// per-Gaussian view-independent cache (scale, rotation, 3D covariance,
// opacity); valid until the parameters change
void launch_prep_gauss(const Ctx& c, cudaStream_t st);
void launch_prep_fwd(const Ctx& c, cudaStream_t st);
// tangent features of v (P floats) for every visible pair; clears the
// pairs' cotangent slots
void launch_prep_jvp(const Ctx& c, const float* v, cudaStream_t st);
// the same for the PCG direction p <- z + beta p (beta from the device
// scalars), formed and written back to p in the same pass
void launch_prep_jvp_direction(const Ctx& c, const float* z, float* p, cudaStream_t st);
// g = J^T u chained from the cotangent slots (+ lambda damping of v if v).
// With dot, pAp = v^T g in FP64 and alpha = rz / pAp on the device.
void launch_prep_vjp(const Ctx& c, float* g, const float* v, const float* D, bool dot, cudaStream_t st);
void launch_prep_diag(const Ctx& c, float* D, cudaStream_t st);

// ---- binning.cu -----------------------------------------------------------
// Exclusive prefix sum of n 64-bit counts in place; returns the total via a
// device word (total_dev) the caller reads.
void scan_u64(unsigned long long* data, long long n, unsigned long long* total_dev, void* tmp, size_t tmp_bytes,
              cudaStream_t st);
size_t scan_u64_tmp_bytes(long long n);
// tile counts of the depth-sorted pairs into cnt (then scanned in place)
void launch_sorted_counts(const Ctx& c, cudaStream_t st);
// one (slot * T + tile, Gaussian) entry per overlapped tile, in depth order
void launch_emit(const Ctx& c, cudaStream_t st);
size_t radix_tmp_bytes(long long n);
// Two-level stable binning of the depth-sorted pairs into the tile lists
// (c.ids, c.ranges), for views whose tile rows and columns fit the shared
// counters (bin_rows_fit): bin_rows places every visible pair into the lists
// of the tile rows it spans (rl, one entry per (pair, row): the Gaussian
// index and the pair's tile columns packed in 64 bits; counts per
// (slot, row, chunk) in mat, bin_row_mat_elems of them, scanned in place,
// 32-bit total in *rtotal); bin_tiles places the row lists' pairs into the
// tiles (counts per (tile, segment of its row list) in cnt,
// bin_tile_count_elems of them, scanned into the runs' starts, total in
// *etotal) and writes the ranges.  tmp: scan scratch of
// bin_scan_tmp_bytes(max(mat elements, tile-count elements)).
bool bin_rows_fit(const Ctx& c);
size_t bin_row_mat_elems(const Ctx& c);
size_t bin_tile_count_elems(const Ctx& c);
size_t bin_scan_tmp_bytes(long long n);
void bin_rows(const Ctx& c, unsigned* mat, unsigned long long* rl, unsigned* rtotal, void* tmp, cudaStream_t st);
void bin_tiles(const Ctx& c, const unsigned* mat, const unsigned* rtotal, const unsigned long long* rl, unsigned* cnt,
               unsigned* etotal, void* tmp, cudaStream_t st);
// Stable LSD radix sort of (keys, vals) on the low `bits` key bits.
// Result ends in keys/vals (the alternate buffers are scratch).
void radix_sort(unsigned long long* keys, unsigned int* vals, unsigned long long* keys_alt, unsigned int* vals_alt,
                long long n, int bits, void* tmp, size_t tmp_bytes, cudaStream_t st);
void radix_sort32(unsigned int* keys, unsigned int* vals, unsigned int* keys_alt, unsigned int* vals_alt, long long n,
                  int bits, void* tmp, size_t tmp_bytes, cudaStream_t st);
void launch_ranges(const Ctx& c, cudaStream_t st);

// ---- raster.cu ------------------------------------------------------------
// Forward render of the sampled pixels: residuals and caches; loss sums.
void launch_raster_fwd_samples(const Ctx& c, cudaStream_t st);
// Full frames of every slot into images [nv][H][W][3].
void launch_raster_full(const Ctx& c, float* images, cudaStream_t st);
void launch_ssim(const Ctx& c, cudaStream_t st);
void launch_frame_sqerr(const Ctx& c, const float* frames, double* out, cudaStream_t st);
// host-side view draws (view_sampler.cu)
void uniform_views(int n_cams, int n_views, uint64_t seed, int64_t step, std::vector<int32_t>& out);
void launch_raster_jvp(const Ctx& c, float* u, cudaStream_t st);
// Back-scatter of the per-sample cotangent (u, or w * residual when u is
// null) into the cotangent slots; needs the caches.
void launch_raster_vjp(const Ctx& c, const float* u, cudaStream_t st);
// Fused J^T W J: JVP pass then VJP pass per warp item.
void launch_raster_jtj(const Ctx& c, cudaStream_t st);
// Per-pair rows of diag(J^T W J) into c.dslot (cleared by the caller).
void launch_raster_diag(const Ctx& c, cudaStream_t st);
// k_diag that also back-scatters the right-hand side's cotangents into c.cot
void launch_raster_diag_rhs(const Ctx& c, cudaStream_t st);
// Longest-first order of the work items by the traversal lengths the forward
// render recorded: sorted[k] = work[order[k]].  Scratch: keys/vals and their
// alternates (nwork each) and radix_tmp_bytes(nwork).
void launch_order_work(const Ctx& c, unsigned long long* keys, unsigned int* vals, unsigned long long* keys_alt,
                       unsigned int* vals_alt, void* tmp, size_t tmp_bytes, int2* sorted, cudaStream_t st);

// ---- cg.cu ----------------------------------------------------------------
void launch_precond(const Ctx& c, const float* D, float* minv, cudaStream_t st);
void launch_cg_init(const Ctx& c, const float* b, const float* minv, float* x, float* r, float* z, float* p,
                    cudaStream_t st);
void launch_cg_update(const Ctx& c, int iter, const float* p, const float* Ap, const float* minv, float* x, float* r,
                      float* z, cudaStream_t st);
void launch_max_dc(const Ctx& c, const float* x, cudaStream_t st);
void launch_lm_update(const Ctx& c, long long lm_step, double lr_warm, double lr_cap, double color_bound,
                      int warm_iters, const float* x, float* params, cudaStream_t st);
void launch_zero_scalars(const Ctx& c, cudaStream_t st);

// ---- batched CG (all scenes of a batch in one launch per phase) ----------
// grid: blocks of a batched launch (grid-stride over the chunks)
void launch_b_precond_init(const BatchTables& t, int grid, cudaStream_t st);
void launch_b_direction(const BatchTables& t, int iter, int grid, cudaStream_t st);
void launch_b_prep_jvp(const BatchTables& t, int deg, int grid, cudaStream_t st);
void launch_b_jtj(const BatchTables& t, int grid, cudaStream_t st);
void launch_b_prep_vjp(const BatchTables& t, int deg, int iter, int grid, cudaStream_t st);
void launch_b_update(const BatchTables& t, int iter, int grid, cudaStream_t st);
void launch_b_lm_update(const BatchTables& t, int iters, int grid, cudaStream_t st);
// All of the above in one persistent cooperative launch (grid barriers between
// the phases, each waiting at most timeout_s); bar: grid_bar_bytes() of device
// memory, zeroed by the launcher.  grid_bar_error: the error word of a host
// copy of those bytes (1: a barrier's wait ran out).
size_t grid_bar_bytes();
cudaError_t launch_b_pcg(const BatchTables& t, int deg, int iters, void* bar, double timeout_s, cudaStream_t st);
int grid_bar_error(const void* bar_host_copy);

// ---- the per-tile SplitMix64 stream of the pixel sampler --------------------
// Tile columns [x0, x1] that the list of a pair covers in tile row ty of its
// rectangle rc.  The ellipse {d : d^T Sigma2^-1 d <= tau} around the 2D mean,
// tau = 2 ln(255 o) + 0.02, holds every pixel where alpha reaches 1/255 (by a
// factor e^-0.01 on the threshold, far above FP32 rounding), so a tile it
// misses changes no pixel.  e0 = (mux, muy, kx, dys), e1 = (pq, qq, ey, -):
// given the offset dy from muy the ellipse holds dx with (dx - kx dy)^2 <=
// pq - qq dy^2, |dy| <= ey (< 0: empty), and its rightmost / leftmost points
// lie at dy = dys / -dys.  Its cut by the row's band of pixel-centre rows
// [yA, yB] (taken as an interval) is convex, so the pixel-centre columns it
// meets run from x_l(dl) to x_r(dr), the extreme offsets clamped into the
// band (x_r is concave in dy, x_l convex).  Every operation is rounded on
// its own, in a fixed order, so the lists are reproducible bit for bit.
__device__ __forceinline__ bool row_span(float4 e0, float4 e1, int ty, int4 rc, int tw, int th, int W, int H,
                                         int& x0, int& x1) {
    const float yA = __fadd_rn((float)(ty * th), 0.5f);
    const float yB = __fsub_rn((float)min(ty * th + th, H), 0.5f);
    const float lo = fmaxf(__fsub_rn(yA, e0.y), -e1.z);
    const float hi = fminf(__fsub_rn(yB, e0.y), e1.z);
    if (!(lo <= hi)) return false;  // the band misses the ellipse's rows (band_meets)
    const float dr = fminf(fmaxf(e0.w, lo), hi);
    const float dl = fminf(fmaxf(-e0.w, lo), hi);
    const float hr = __fsqrt_rn(fmaxf(__fsub_rn(e1.x, __fmul_rn(e1.y, __fmul_rn(dr, dr))), 0.f));
    const float hl = __fsqrt_rn(fmaxf(__fsub_rn(e1.x, __fmul_rn(e1.y, __fmul_rn(dl, dl))), 0.f));
    const float xr = __fadd_rn(e0.x, __fadd_rn(__fmul_rn(e0.z, dr), hr));
    const float xl = __fadd_rn(e0.x, __fsub_rn(__fmul_rn(e0.z, dl), hl));
    // pixel columns px whose centre px + 1/2 lies in [xl, xr]
    const float fl = fmaxf(ceilf(__fsub_rn(xl, 0.5f)), 0.f);
    const float fh = fminf(floorf(__fsub_rn(xr, 0.5f)), (float)(W - 1));
    if (!(fl <= fh)) return false;
    // their tile columns (a shift for power-of-two tile widths)
    const int il = (int)fl, ih = (int)fh;
    const bool pow2 = (tw & (tw - 1)) == 0;
    const int sh = __ffs(tw) - 1;
    x0 = max(pow2 ? il >> sh : il / tw, rc.x);
    x1 = min(pow2 ? ih >> sh : ih / tw, rc.y);
    return x0 <= x1;
}

// The first test of row_span alone: whether tile row ty's band meets the
// ellipse's rows |dy| <= ey.  Monotone in ty from both ends, so the rows that
// pass are contiguous; row_span can still find no tile in one of them (no
// pixel-centre column inside, or outside the rectangle's columns).
__device__ __forceinline__ bool band_meets(float4 e0, float4 e1, int ty, int th, int H) {
    const float yA = __fadd_rn((float)(ty * th), 0.5f);
    const float yB = __fsub_rn((float)min(ty * th + th, H), 0.5f);
    return fmaxf(__fsub_rn(yA, e0.y), -e1.z) <= fminf(__fsub_rn(yB, e0.y), e1.z);
}

__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// state of (seed, LM step, camera, tile); output i is sm64_mix(state + (i+1) gamma)
__device__ __forceinline__ unsigned long long tile_stream(unsigned long long seed, long long lm_step, int cam,
                                                          int tile) {
    unsigned long long h = sm64_mix(seed ^ 0x5851F42D4C957F2Dull);
    h = sm64_mix(h ^ (unsigned long long)lm_step);
    h = sm64_mix(h ^ (unsigned long long)(unsigned int)cam);
    return sm64_mix(h ^ (unsigned long long)(unsigned int)tile);
}
constexpr unsigned long long kSm64Gamma = 0x9E3779B97F4A7C15ull;

void launch_importance(const Ctx& c, long long lm_step, unsigned long long seed, cudaStream_t st);

// ---- device memory from the library's stream-ordered pool -----------------
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);
void pool_trim();

}  // namespace lmrs

namespace lmrs {
// Optional per-launch CUDA-event timing of the scene being driven by the
// calling thread (set by the ABI entry points while timing is enabled).
struct LaunchTimer;
LaunchTimer* active_timer();
int timer_start(LaunchTimer* t, const char* name, cudaStream_t st);
void timer_stop(LaunchTimer* t, int rec, cudaStream_t st);
}  // namespace lmrs

#define LMRS_LAUNCH(kernel, grid, block, smem, stream, ...)                     \
    do {                                                                        \
        ::lmrs::note_launch();                                                  \
        ::lmrs::LaunchTimer* t_ = ::lmrs::active_timer();                       \
        const int r_ = t_ ? ::lmrs::timer_start(t_, #kernel, (stream)) : -1;    \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);            \
        if (t_) ::lmrs::timer_stop(t_, r_, (stream));                           \
    } while (0)

// The same for a kernel given as a function pointer with an explicit name
// (template kernels whose argument lists contain commas).
#define LMRS_LAUNCH_AS(name, kptr, grid, block, smem, stream, ...)              \
    do {                                                                        \
        ::lmrs::note_launch();                                                  \
        ::lmrs::LaunchTimer* t_ = ::lmrs::active_timer();                       \
        const int r_ = t_ ? ::lmrs::timer_start(t_, (name), (stream)) : -1;     \
        (kptr)<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);            \
        if (t_) ::lmrs::timer_stop(t_, r_, (stream));                           \
    } while (0)
