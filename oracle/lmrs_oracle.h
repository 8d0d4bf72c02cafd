/*
 * FP64 CPU oracle for the matrix-free Levenberg-Marquardt / residual-sampling
 * hot path (Sec. 4, Alg. 1-3 of "Matrix-free Second-order Optimization of
 * Gaussian Splats with Residual Sampling").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this library: only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library; both are written from the paper
 * and from the conventions listed below.
 *
 * Conventions (readings of the paper; see the design notes of the project):
 *   parameters: group-major SoA, [means Gx3 | log-scales Gx3 | quats Gx4
 *     (w,x,y,z) | opacity logits G | SH Gx(d+1)^2x3]; s = exp(log-scale),
 *     q normalised, o = sigmoid(logit), colour = SH(dir) + 0.5 clamped at 0.
 *   decisions that choose integers (visibility, depth key, tile rectangle,
 *     the tile columns kept per row of the rectangle) are taken in FP32 with
 *     a fixed operation order; everything else is FP64.
 *   a Gaussian's tile list entries are the tiles of its rectangle some
 *     pixel-centre column of which meets the ellipse where alpha reaches
 *     1/255 (level 2 ln(255 o) + 0.02) within the tile row's band: a tile it
 *     leaves out has alpha < 1/255 at every pixel, so no pixel changes.
 *   per-pixel skip / clamp / termination tests are taken in FP64 and a pixel
 *     whose test lies within a relative margin of its threshold is flagged.
 */
#ifndef LMRS_ORACLE_H
#define LMRS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float world_to_cam[12];   /* row-major 3x4 [R | t] */
    float znear;
} orc_camera;

typedef struct {
    int32_t sh_degree;        /* 0..3 */
    int32_t tile_w, tile_h;   /* tile_w * tile_h <= 256 */
    double  sample_frac;      /* K_t = clamp(floor(frac * n_valid + 0.5), 1, n_valid) */
    int32_t samples_per_tile; /* > 0 overrides sample_frac: K_t = min(n_valid, this) */
    int32_t weight_mode;      /* 0: w = 1; 1: w = n_valid / K_t */
    double  lambda;
    int32_t damping_mode;     /* 0: lambda * I; 1: lambda * diag(J^T W J) */
    int32_t cg_iters;
    double  lr_warm, lr_cap, color_bound;
    int32_t warm_iters;
    uint64_t seed;
    double  margin_alpha;     /* relative margin that flags an alpha test */
    double  margin_T;         /* relative margin that flags a termination test */
    int32_t sample_dist;      /* 0 uniform without replacement; 1 q_residual; 2 q_Gaussian (i.i.d. per tile) */
    double  ssim_weight;      /* weight of the diagonal SSIM residual term (0: MSE only) */
    int32_t list_mode;        /* 0: per tile row, the tiles the alpha >= 1/255 ellipse reaches;
                                 1: every tile of the 3-sigma rectangle (the 3DGS lists, Sec. 3) */
} orc_config;

typedef struct orc_scene orc_scene;

orc_scene* orc_create(const orc_config* cfg, int32_t n_gauss, const float* params,
                      const orc_camera* cams, int32_t n_cams, const float* targets);
void    orc_destroy(orc_scene* s);
/* Replace the parameters (FP64; list decisions use their FP32 rounding). */
int32_t orc_set_params(orc_scene* s, const double* params);
int32_t orc_get_params(const orc_scene* s, double* params);
int64_t orc_num_params(const orc_scene* s);

/* Pixel sampling for (views, lm_step) plus FP32 binning and FP64 features. */
int32_t orc_begin_step(orc_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step);

int64_t orc_num_samples(const orc_scene* s);
int32_t orc_get_samples(const orc_scene* s, uint8_t* off, int32_t* tile_off, double* w,
                        int32_t* px, int32_t* py, int32_t* slot);
/* Per sample: 1 when an importance draw may legitimately go another way in
 * a different precision (its threshold within a relative margin of a bin
 * edge of the tile's cumulative weights, or a flagged pixel in its tile). */
int32_t orc_get_sample_flags(const orc_scene* s, uint8_t* flags);
/* SSIM term of the step (ssim_weight > 0): per sample and channel the
 * residual s = 1 - SSIM and its derivative d = ds/dX at the sample's own
 * pixel (S x 3 each), and per sample 1 when its 11 x 11 window holds a
 * full-frame pixel flagged near a compositing decision.  Zeros when off. */
int32_t orc_get_ssim(const orc_scene* s, double* s_out, double* d_out, uint8_t* flags);
int64_t orc_num_pairs(const orc_scene* s);
int32_t orc_get_lists(const orc_scene* s, int32_t* ranges, int32_t* ids);
int32_t orc_get_geom(const orc_scene* s, int32_t slot, int32_t* vis, float* depth, int32_t* rect);
int32_t orc_get_features(const orc_scene* s, int32_t slot, double* feat);

/* Per-sample outcomes of near decisions (reset by orc_begin_step).  A test on
 * a value within a relative margin of its threshold (margin_alpha for the
 * alpha skip at 1/255 and the clamp at 0.99, margin_T for the termination at
 * 1e-4) is "near": an FP32 evaluation may take it either way.  Bit k of a
 * sample's mask inverts the k-th near decision met along its list (per
 * entry: clamp, skip, termination), in every sample-level computation
 * (render, J v, J^T u, diag, right-hand side, operator).  orc_near_counts
 * gives the number of near decisions each sample meets under its mask. */
int32_t orc_set_flips(orc_scene* s, const int64_t* idx, const uint32_t* masks, int64_t n);
int32_t orc_clear_flips(orc_scene* s);
int32_t orc_near_counts(const orc_scene* s, const int64_t* idx, int64_t n, int32_t* counts);
/* Every outcome of the near decisions of samples idx[0..n): n_near[k] as in
 * orc_near_counts (masks ignored); for m < 2^min(n_near[k], max_bits) the
 * colour (rgb) and J v (u, tangent v) of sample idx[k] with mask m at
 * [(k 2^max_bits + m) 3 + ch], NaN for the other m.  max_bits <= 8. */
int32_t orc_sample_outcomes(const orc_scene* s, const double* v, const int64_t* idx, int64_t n, int32_t max_bits,
                            int32_t* n_near, double* rgb, double* u);

int32_t orc_render_samples(const orc_scene* s, double* rgb, double* resid, uint8_t* flags);
int32_t orc_render_samples_subset(const orc_scene* s, const int64_t* idx, int64_t n,
                                  double* rgb, uint8_t* flags);
int32_t orc_render_full(const orc_scene* s, int32_t slot, double* img, uint8_t* flags);
/* Number of Gaussians each pixel of the view composites (alpha >= 1/255
 * before termination), H x W. */
int32_t orc_pixel_counts(const orc_scene* s, int32_t slot, int32_t* counts);
/* The view's full frame (H x W x 3) with the preprocessing and compositing
 * evaluated in binary32 over the same lists (test infrastructure: the FP32
 * rounding error of a pixel against the FP64 frame, as a function of how
 * many Gaussians it composites). */
int32_t orc_render_full_f32(const orc_scene* s, int32_t slot, double* img);

int32_t orc_jvp(const orc_scene* s, const double* v, double* u);
int32_t orc_jvp_subset(const orc_scene* s, const double* v, const int64_t* idx, int64_t n, double* u);
int32_t orc_vjp(const orc_scene* s, const double* u, double* g);
int32_t orc_vjp_gauss(const orc_scene* s, const double* u, const int32_t* gids, int32_t n, double* out);
int32_t orc_diag(const orc_scene* s, double* D);
/* Per entry j: sum over the rows (sample, channel) of w (sum_f |dC/df a_fj|)^2,
 * the magnitude of the terms of D_j's chain rule. */
int32_t orc_diag_magnitude(const orc_scene* s, double* M);
int32_t orc_diag_gauss(const orc_scene* s, const int32_t* gids, int32_t n, double* out);
int32_t orc_apply(const orc_scene* s, const double* v, const double* D, double* out);
int32_t orc_apply_gauss(const orc_scene* s, const double* v, const double* D,
                        const int32_t* gids, int32_t n, double* out);
int32_t orc_rhs(const orc_scene* s, double* b);
int32_t orc_precond(const orc_scene* s, const double* D, double* minv);
/* stats: [0] r^T z initial, [1] final |r|, [2..] alpha_i, beta_i pairs */
int32_t orc_cg(const orc_scene* s, const double* b, const double* D, int32_t iters,
               double* x, double* stats);
double  orc_step_size(const orc_scene* s, const double* x, int64_t lm_step);
/* One LM step (Alg. 1): stats [0] sampled MSE before, [1] eta, [2] max|x_dc| */
int32_t orc_lm_step(orc_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step,
                    double* x_out, double* stats);

/* Pieces exposed for the pin tests. */
void    orc_sh_basis(int32_t deg, double x, double y, double z, double* Y);
void    orc_splitmix64(uint64_t state, int32_t n, uint64_t* out);
uint64_t orc_tile_seed(uint64_t seed, int64_t lm_step, int32_t view_id, int32_t tile_id);
void    orc_sample_tile(uint64_t seed, int64_t lm_step, int32_t view_id, int32_t tile_id,
                        int32_t n_valid, int32_t k, uint8_t* out);
int32_t orc_num_threads(void);
/* SSIM of the three channels of images X and Y (H x W x 3) at pixel (px, py):
 * s = 1 - SSIM and d = ds/dX(px, py), every other pixel held fixed. */
void    orc_ssim_pixel(const double* X, const double* Y, int32_t H, int32_t W, int32_t px, int32_t py,
                       double* s, double* d);

#ifdef __cplusplus
}
#endif
#endif
