/*
 * lmrs.h -- C ABI of the GB300 (sm_103a) matrix-free Levenberg-Marquardt
 * hot path for 3D Gaussian splatting with residual sampling
 * ("Matrix-free Second-order Optimization of Gaussian Splats with Residual
 * Sampling", Sec. 4 and App. A).
 *
 * The library computes, on one GPU, the pieces of one LM step (Alg. 1):
 * per-tile pixel sampling (Sec. 4.4), projection and tile binning with a
 * radix sort on (tile, depth) (Sec. 3), the alpha-composited render and its
 * residuals (Eq. 4, Eq. 7), the Jacobian-vector product J v by forward mode
 * (Alg. 3), the back-scatter J^T u, diag(J^T W J), the damped operator
 * (J^T W J + lambda D) v of the normal equation (Eq. 8), the preconditioned
 * CG solve (Alg. 1) and the parameter update with the step-size rule of
 * Sec. 4.5 / App. D.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Parameter vectors ("P-vectors": parameters, v, J^T u, D, x, b) hold P =
 *   G * P_g floats, P_g = 11 + 3 (d+1)^2 for SH degree d, group-major:
 *     [ means G x 3 | log-scales G x 3 | quaternions G x 4 (w,x,y,z) |
 *       opacity logits G | SH coefficients G x (d+1)^2 x 3 ]
 *   scale = exp(log-scale), rotation from the normalised quaternion, opacity
 *   = sigmoid(logit), colour = sum_k sh_k Y_k(view direction) + 0.5,
 *   clamped at 0 (real SH basis without Condon-Shortley phase).
 * - Sampled-pixel vectors (residuals, J v, the u of J^T u) hold S x 3
 *   floats, one RGB triple per sampled pixel, ordered by view slot, then
 *   tile (row-major), then the sample order inside the tile.
 * - Pointers named *_dev are device pointers on the scene's device.  Entry
 *   points documented as "host or device" accept either (CUDA unified
 *   addressing decides).  The library never frees caller memory.
 * - Every call is asynchronous on the scene's stream unless it returns data
 *   to host memory or takes a non-NULL stats pointer; those synchronise the
 *   stream before returning.
 * - Errors are returned as lmrs_status; nothing is thrown across the ABI.
 *   After LMRS_ERR_CUDA the scene should be destroyed; after any other error
 *   the scene stays usable.  lmrs_last_error() describes the last failure.
 * - A scene is not thread-safe: one host thread at a time.
 */
#ifndef LMRS_H
#define LMRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lmrs_scene lmrs_scene;

typedef enum {
    LMRS_OK = 0,
    LMRS_ERR_INVALID_ARG = 1,      /* bad pointer, size, view id or config value */
    LMRS_ERR_OOM = 2,              /* a device allocation failed */
    LMRS_ERR_CUDA = 3,             /* a CUDA call or kernel launch failed */
    LMRS_ERR_NOT_PREPROCESSED = 4, /* a prerequisite call (preprocess, render, diag) is missing */
    LMRS_ERR_NUMERIC = 5,          /* non-finite or non-positive CG curvature */
    LMRS_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up */
    LMRS_ERR_BUDGET = 7            /* a size limit of the library was exceeded */
} lmrs_status;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  Pixel (x, y)
 * covers [x, x+1) x [y, y+1) with its centre at (x + 0.5, y + 0.5); a point
 * t in camera space projects to (fx t_x / t_z + cx, fy t_y / t_z + cy). */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float world_to_cam[12]; /* row-major 3x4 [R | t] */
    float znear;            /* Gaussians with camera-space depth <= znear are culled */
} lmrs_camera;

typedef struct {
    int32_t sh_degree;        /* 0..3 */
    int32_t tile_w, tile_h;   /* tile shape in pixels, tile_w * tile_h <= 256 (16 x 16 in the paper, Sec. 4.4) */
    double  sample_frac;      /* K_t = clamp(floor(frac * n_valid + 0.5), 1, n_valid) samples per tile */
    int32_t samples_per_tile; /* > 0 overrides sample_frac: K_t = min(n_valid, samples_per_tile) */
    int32_t weight_mode;      /* 0: w = 1; 1: w = n_valid / K_t (the 1/q weight of Eq. 13 per tile) */
    double  lambda;           /* damping of Eq. 8 */
    int32_t damping_mode;     /* 0: + lambda * I (Eq. 8); 1: + lambda * diag(J^T W J) */
    int32_t cg_iters;         /* PCG iterations per LM step (Alg. 1), each one operator application */
    double  lr_warm;          /* step size of the first warm_iters LM steps (App. D: 0.05 for 10) */
    double  lr_cap;           /* upper bound of the step size (App. D: 0.2) */
    double  color_bound;      /* largest SH degree-0 change per step (Sec. 4.5: 1) */
    int32_t warm_iters;
    int32_t cache_bf16;       /* 1: per-sample render caches (final colour, transmittance) in BF16 */
    uint64_t seed;            /* key of the per-tile pixel sampler */
    int32_t sample_dist;      /* residual sampling distribution within each tile (supplementary material):
                                 0 uniform without replacement (the paper's choice);
                                 1 q_residual, 2 q_Gaussian: K_t i.i.d. draws with probability proportional
                                 to e^{|r_p|} (|r_p| the Euclidean norm of the pixel's RGB residual) or to
                                 the number of Gaussians the pixel composites (uniform when a tile has none),
                                 weight 1 / (K_t q(p)) per sample (weight_mode is then not used).  Modes 1
                                 and 2 render every pixel of the step's views in lmrs_preprocess. */
    double  ssim_weight;      /* weight of the diagonal SSIM term (supplementary material, "Results with SSIM
                                 loss": 0.2 beside the MSE term's 1); 0 turns it off.  Per sampled pixel and
                                 channel the residual s = 1 - SSIM (Wang et al. 2004: 11 x 11 Gaussian window,
                                 sigma 1.5, pixels outside the image count as 0, C1 = 0.01^2, C2 = 0.03^2) is
                                 added to the objective as ssim_weight * w * s^2, with the Jacobian of s kept
                                 only through the pixel's own colour, d = ds/dC (the diagonal approximation):
                                 J^T W J gains ssim_weight * w * d^2 per (sample, channel) row and J^T W r
                                 gains ssim_weight * w * d * s.  lmrs_render then renders every pixel of the
                                 step's views.  lmrs_jvp and lmrs_vjp stay the colour Jacobian's products. */
} lmrs_config;

typedef struct {
    double rz0;        /* r_0^T z_0 */
    double rz_final;   /* r_n^T z_n */
    double res_norm;   /* |r_n| */
    double alpha[64];  /* per-iteration alpha (first 64 iterations) */
    double beta[64];
    int32_t iters;
} lmrs_cg_stats;

typedef struct {
    double loss;          /* sum_i w_i |r_i|^2 / (3 sum_i w_i) over the sampled pixels, before the update */
    double eta;           /* step size used */
    double max_dc;        /* max |x| over the SH degree-0 entries of the solution */
    double rz0, rz_final; /* PCG diagnostics */
    int64_t n_samples;    /* S */
    int64_t n_pairs;      /* (view, tile, Gaussian) entries in the sorted tile lists */
} lmrs_step_stats;

/* Fills *cfg with the defaults: SH degree 0, 16x16 tiles, sample_frac 1,
 * weight_mode 0, lambda 0.1, damping_mode 1, 8 CG iterations, lr_warm 0.05,
 * lr_cap 0.2, color_bound 1, warm_iters 10, FP32 caches, seed 0. */
lmrs_status lmrs_config_default(lmrs_config* cfg);

/* Creates a scene on the current CUDA device.
 *   params     : P floats (host or device), copied.
 *   cams_host  : n_cams cameras in host memory, copied; all of one size.
 *   targets_dev: n_cams x height x width x 3 floats (device), borrowed: must
 *                outlive the scene; may be NULL (then residuals are renders).
 *   cuda_stream: cudaStream_t used for every launch (NULL = legacy stream).
 * The scene owns every internal device buffer (parameters, CG vectors,
 * per-pair records, sort buffers, per-sample caches). */
lmrs_status lmrs_scene_create(const lmrs_config* cfg, int64_t n_gauss, const float* params,
                              const lmrs_camera* cams_host, int32_t n_cams,
                              const float* targets_dev, void* cuda_stream, lmrs_scene** out);
lmrs_status lmrs_scene_destroy(lmrs_scene* scene);

/* Copies P floats in or out of the scene's parameters (host or device
 * pointer).  set_params invalidates a previous preprocess. */
lmrs_status lmrs_set_params(lmrs_scene* scene, const float* src);
lmrs_status lmrs_get_params(lmrs_scene* scene, float* dst);

/* Per-step setup of one LM step for the views view_ids_host[0..n_views)
 * (camera indices, host memory): per-tile pixel sampling keyed by
 * (seed, lm_step, camera index, tile) (Sec. 4.4), projection of every
 * Gaussian into every view, tile binning and the radix sort by (tile,
 * depth, Gaussian index).  Synchronises once (to size the sort). */
lmrs_status lmrs_preprocess(lmrs_scene* scene, const int32_t* view_ids_host, int32_t n_views,
                            int64_t lm_step);

/* Alpha-composited render (Eq. 4, Alg. 2) of the preprocessed views.
 *   images_dev   : n_views x height x width x 3 floats or NULL; full frames.
 *   residuals_dev: S x 3 floats or NULL; r = render - target at the sampled
 *                  pixels (Eq. 7).
 * Always fills the per-sample caches (final colour, final transmittance,
 * list position of the termination) used by vjp, rhs, diag and lm_step.
 * Requires lmrs_preprocess. */
lmrs_status lmrs_render(lmrs_scene* scene, float* images_dev, float* residuals_dev);

/* u = J v at the sampled pixels: forward mode through preprocessing and
 * compositing (Alg. 3).  v_dev: P floats; u_dev: S x 3 floats.
 * Requires lmrs_preprocess. */
lmrs_status lmrs_jvp(lmrs_scene* scene, const float* v_dev, float* u_dev);

/* g = J^T u (no weights): reverse mode, compositing then preprocessing
 * (App. A).  u_dev: S x 3 floats; g_dev: P floats, overwritten.
 * Requires lmrs_render. */
lmrs_status lmrs_vjp(lmrs_scene* scene, const float* u_dev, float* g_dev);

/* b = J^T W r, the right-hand side of Eq. 8 (Eq. 14 up to its constant),
 * from the cached residuals.  b_dev: P floats.  Requires lmrs_render. */
lmrs_status lmrs_rhs(lmrs_scene* scene, float* b_dev);

/* D = diag(J^T W J) (App. A, "Diag kernel"), also kept by the scene for the
 * damping and the Jacobi preconditioner.  d_dev: P floats or NULL.
 * Requires lmrs_render. */
lmrs_status lmrs_jtj_diag(lmrs_scene* scene, float* d_dev);

/* out = (J^T W J + lambda * (I or D)) v, the operator of Eq. 8 (Alg. 1,
 * line "u = ..."), fused JVP + VJP rasterisation.  v, out: P floats (host or
 * device; host pointers are staged through the scene and the call
 * synchronises).  Requires lmrs_preprocess, and lmrs_jtj_diag when
 * damping_mode = 1. */
lmrs_status lmrs_jtjv(lmrs_scene* scene, const float* v, float* out);

/* Preconditioned CG of Alg. 1 on A x = b with the Jacobi preconditioner
 * 1 / diag(A) (Sec. 4.2): x_0 = 0, exactly `iters` operator applications,
 * FP64 inner products and scalars on the device.  b_dev, x_dev: P floats.
 * st may be NULL.  Requires lmrs_jtj_diag. */
lmrs_status lmrs_cg_solve(lmrs_scene* scene, const float* b_dev, float* x_dev, int32_t iters,
                          lmrs_cg_stats* st);

/* Step size of Sec. 4.5 / App. D for a solution x (device, P floats):
 * lr_warm while lm_step < warm_iters, else min(lr_cap, color_bound /
 * max |x_dc|) (lr_cap when that maximum is 0); returned in *eta_host. */
lmrs_status lmrs_step_size(lmrs_scene* scene, const float* x_dev, int64_t lm_step, double* eta_host);

/* The step size of lmrs_step_size without a scene and without allocating
 * any device memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc, for example code whose device
 * memory is owned by another allocator (a framework's caching pool that has
 * reserved the free memory, so a driver allocation can fail or force a
 * device-wide synchronisation) and latency-critical loops in which an
 * allocation or free would stall.
 *   x_dev      : solution, G * (11 + 3 (sh_degree+1)^2) floats (device), read.
 *   n_gauss    : G, at most 8,388,608 (4096 blocks of 2048 Gaussians);
 *                larger G returns LMRS_ERR_BUDGET before any device work.
 *   lm_step, lr_warm, lr_cap, color_bound, warm_iters: as in lmrs_config.
 *   cuda_stream: stream of the launch (NULL = legacy stream).
 *   *eta_host  : the step size (host); the call synchronises the stream.
 * Scratch: a 16,512-byte static device array that every GPU loading the
 * library holds until the process exits.  The first call on a device looks
 * up its address (cudaGetSymbolAddress) with that device current.  All
 * calls on a device share the
 * array, so calls that overlap on the GPU race; each call clears the words
 * that must start at zero.  Errors: LMRS_ERR_INVALID_ARG for null pointers,
 * n_gauss <= 0 or sh_degree outside 0..3; LMRS_ERR_CUDA if a CUDA call fails. */
lmrs_status lmrs_step_size_noalloc(const float* x_dev, int64_t n_gauss, int32_t sh_degree, int64_t lm_step,
                                   double lr_warm, double lr_cap, double color_bound, int32_t warm_iters,
                                   void* cuda_stream, double* eta_host);

/* One LM step (Alg. 1): preprocess, render, b = J^T W r, D, PCG with
 * cfg.cg_iters iterations, step size, and the update beta <- beta - eta x
 * (the descent reading of Eq. 8 with r = render - target).  st may be NULL
 * (then nothing synchronises).  The solution x stays readable through
 * lmrs_get_solution.  When the solve meets a non-finite r^T z or p^T A p, or
 * p^T A p <= 0 (non-finite parameters or targets, for example), the update
 * is skipped on the device (the parameters stay as they were, eta = 0) and,
 * with st given, the call returns LMRS_ERR_NUMERIC; the scene stays usable. */
lmrs_status lmrs_lm_step(lmrs_scene* scene, const int32_t* view_ids_host, int32_t n_views,
                         int64_t lm_step, lmrs_step_stats* st);
lmrs_status lmrs_get_solution(lmrs_scene* scene, float* x_dst);

/* ---- Batches: many small fits stepping together ------------------------
 * A batch groups scenes (same SH degree, same cg_iters <= 64) whose LM steps
 * run together.  The paper steps one scene at a time; this is the batched
 * form of Alg. 1.  Per LM step:
 *   1. each scene's per-step setup (sampling, binning, render, J^T W r,
 *      diag) runs on its own stream, n_threads scenes at a time on host
 *      threads (give the scenes distinct streams for overlap);
 *   2. the PCG iterations of all scenes run over segment tables, with
 *      per-scene FP64 scalars, phase by phase (direction, preprocess-JVP,
 *      fused raster, preprocess-VJP + p^T A p, vector update): by default
 *      in one persistent cooperative launch with grid barriers between the
 *      phases, else as one launch per phase, the whole loop a CUDA graph
 *      captured at the first step and replayed (re-captured when the
 *      tables outgrow their buffers) -- see lmrs_batch_set_persistent;
 *   3. the per-scene step sizes and updates run as two more phases.
 * Each scene's result equals its own lmrs_lm_step up to the summation
 * order of the inner products.  The scenes stay owned by the caller, must
 * outlive the batch and must not be used by other calls during a step.
 * cuda_stream: stream of the batched launches; NULL makes the batch create
 * its own (graph capture needs a non-legacy stream). */
typedef struct lmrs_batch lmrs_batch;
lmrs_status lmrs_batch_create(lmrs_scene* const* scenes, int32_t n_scenes, int32_t n_threads, void* cuda_stream,
                              lmrs_batch** out);
lmrs_status lmrs_batch_destroy(lmrs_batch* batch);
/* One LM step of every scene.  view_ids: the views of scene 0, then of
 * scene 1, ... (camera indices of each scene, host); n_views[i], lm_steps[i]
 * per scene (host).  stats: n_scenes entries or NULL (then nothing
 * synchronises).  Scene errors are returned as the first failing status. */
lmrs_status lmrs_batch_lm_step(lmrs_batch* batch, const int32_t* view_ids, const int32_t* n_views,
                               const int64_t* lm_steps, lmrs_step_stats* stats);
const char* lmrs_batch_last_error(const lmrs_batch* batch);
/* Outcome of the last lmrs_batch_lm_step for scene i: LMRS_OK (stepped),
 * the scene's own error (its setup failed; LMRS_ERR_NUMERIC when its CG hit
 * a non-finite or non-positive p^T A p, detected only when stats were
 * requested; that scene's parameters are left unchanged), or
 * LMRS_ERR_NOT_PREPROCESSED (not stepped because another scene failed
 * before the batched loop). */
lmrs_status lmrs_batch_scene_status(const lmrs_batch* batch, int32_t i);
/* The launch form of step 2 and 3 above: 1 (the default), one persistent
 * cooperative launch that runs every phase of every PCG iteration and the
 * updates for all scenes, a grid-wide barrier between phases; 0, the CUDA
 * graph of per-phase launches.  Each barrier's wait is bounded (2 s by
 * %globaltimer); a barrier that cannot complete ends the launch, and
 * lmrs_batch_lm_step with stats then returns LMRS_ERR_TIMEOUT.  Where the
 * device refuses a cooperative launch of the grid (too large, or not
 * supported) the batch switches to the graph form for good.  Both forms
 * give the same result up to the summation order of the atomics.
 * Errors: LMRS_ERR_INVALID_ARG for a null batch or on outside {0, 1}. */
lmrs_status lmrs_batch_set_persistent(lmrs_batch* batch, int32_t on);
/* Self-test of that grid barrier, for the host side of failure detection:
 * one cooperative launch whose barrier expects `missing` more blocks than it
 * has.  missing = 0 passes (LMRS_OK); missing > 0 can never complete, so
 * every block's wait runs out after timeout_s (<= 10) and the call returns
 * LMRS_ERR_TIMEOUT with the device still usable.  Synchronises cuda_stream
 * (NULL = legacy stream).  The paper has no counterpart. */
lmrs_status lmrs_grid_barrier_selftest(int32_t missing, double timeout_s, void* cuda_stream);

/* ---- View sampling (Sec. 4.3) and the fit loop ----------------------------
 * Uniform views of step k: n_views camera indices drawn without replacement
 * (partial Fisher-Yates driven by SplitMix64 keyed by (seed, k)), sorted;
 * all cameras when n_views <= 0 or >= n_cams.  views: n_cams entries. */
lmrs_status lmrs_uniform_views(int32_t n_cams, int32_t n_views, uint64_t seed, int64_t step, int32_t* views);

/* K-means view sampler (Sec. 4.3): camera features [position, viewing
 * direction], positions centred on their mean and scaled by the largest
 * distance from it, the direction being the camera's +z axis in world
 * space; Lloyd's algorithm with k-means++ initialisation (SplitMix64 keyed
 * by seed), ties to the lower cluster index, at most 100 iterations;
 * n_clusters = views per step (capped at n_cams).  Host only. */
typedef struct lmrs_view_sampler lmrs_view_sampler;
lmrs_status lmrs_view_sampler_create(const lmrs_camera* cams_host, int32_t n_cams, int32_t n_clusters, uint64_t seed,
                                     lmrs_view_sampler** out);
lmrs_status lmrs_view_sampler_destroy(lmrs_view_sampler* sampler);
/* labels[n_cams] (or NULL), the cluster count and the Lloyd iterations run. */
lmrs_status lmrs_view_sampler_labels(const lmrs_view_sampler* sampler, int32_t* labels, int32_t* n_clusters,
                                     int32_t* iterations);
/* One camera drawn uniformly from every cluster for step `step` (SplitMix64
 * keyed by (seed, step, cluster)), sorted; views: n_clusters entries;
 * *n_views receives the count (fewer only if a cluster came out empty). */
lmrs_status lmrs_view_sampler_draw(const lmrs_view_sampler* sampler, int64_t step, int32_t* views, int32_t* n_views);

/* Full-frame MSE of the current parameters against the targets over every
 * camera (Eq. 7 without sampling; PSNR = -10 log10(mse) for colours in
 * [0, 1]).  Renders the cameras 8 at a time; leaves the scene preprocessed
 * for the last of them. */
lmrs_status lmrs_eval_mse(lmrs_scene* scene, double* mse);

/* An LM-RS fit (Alg. 1 repeated) with the schedules of Sec. 5: views per
 * step and PCG iterations switch from *_first to *_later at switch_step
 * (16 -> 32 views and 5 -> 8 iterations at step 50 in the paper's
 * real-world runs), views drawn uniformly (view_mode 0) or by the K-means
 * sampler with as many clusters as views (view_mode 1, Sec. 4.3), step k
 * using LM step index k.  records: n_steps entries. */
typedef struct {
    int32_t n_steps;
    int32_t views_first, views_later;
    int32_t cg_first, cg_later;
    int32_t switch_step;
    int32_t view_mode;    /* 0 uniform, 1 K-means */
    int32_t eval_every;   /* full-frame MSE every eval_every steps and after the last; 0: never */
    uint64_t seed;        /* view draws */
} lmrs_fit_config;

typedef struct {
    int32_t step, n_views, cg_iters;
    double loss;      /* sampled loss of the step (before its update) */
    double eta;
    double mse_full;  /* after the step when evaluated, else -1 */
    double psnr;      /* -10 log10(mse_full), else -1 */
    double ms;        /* host wall time of the step (it synchronises) */
} lmrs_fit_record;

lmrs_status lmrs_fit(lmrs_scene* scene, const lmrs_fit_config* cfg, lmrs_fit_record* records);

/* ---- Serving: a queue of fit jobs on one device --------------------------
 * The paper fits one scene at a time; the server keeps many fits resident
 * and steps them together with the batched LM step above.
 *   - lmrs_server_submit copies a job (parameters, cameras, targets: host
 *     memory) and queues it; it does not wait for the device.
 *   - a scheduler thread admits queued jobs while fewer than max_active
 *     jobs are resident and the device bytes of the resident jobs (for
 *     each, the larger of its admission estimate and what it holds) plus
 *     the next job's estimate (lmrs_footprint_bytes) stay within
 *     budget_bytes.  The next job is the oldest (policy 0, FIFO) or the one
 *     with the least estimated work, Gaussians x views per step x max_steps,
 *     oldest first among equals (policy 1).  An admitted job's parameters,
 *     CG vectors, raster caches and targets stay on the device until it
 *     finishes.
 *   - every scheduler iteration runs one LM step of each resident job: the
 *     jobs with fewer than solo_min_samples sampled pixels per step in one
 *     batch per group of equal SH degree and cg_iters (lmrs_batch_lm_step),
 *     the others each with lmrs_lm_step on its own stream from a host thread
 *     (up to setup_threads at a time), so their kernels overlap on the
 *     device; then it retires the
 *     jobs that reached target_loss or have run max_steps steps; the freed
 *     memory admits the next jobs (continuous batching).  A job reaches its
 *     target when its sampled loss (Eq. 11 at the step's samples, before the
 *     update) is <= target_loss (stop_full_frame 0), or, with
 *     stop_full_frame 1, when the full-frame MSE of its updated parameters
 *     over every camera (lmrs_eval_mse) is <= target_loss; that is evaluated
 *     after the steps whose sampled loss is <= full_frame_gate x
 *     target_loss.
 *   - the views of step k: lmrs_uniform_views(n_cams, views_per_step,
 *     cfg.seed, k).  A job's steps therefore do not depend on the other jobs: its
 *     result alone and in any mix agree up to the summation order.
 * Jobs stay owned by the server; their records are kept until forgotten. */
typedef struct lmrs_server lmrs_server;
typedef struct {
    int64_t budget_bytes;   /* device bytes the resident jobs may hold */
    int32_t max_active;     /* resident jobs at most (1..1024) */
    int32_t setup_threads;  /* host threads for the per-scene step setup (>= 1) */
    double tiles_per_pair;  /* footprint model: tile entries per visible (view, Gaussian) pair; <= 0: 10 */
    int32_t policy;         /* admission order: 0 FIFO, 1 least estimated work first */
    int32_t stop_full_frame;  /* 1: the target is the full-frame MSE (see above) */
    double full_frame_gate;   /* sampled loss / target_loss at or below which the full frames are checked; <= 0: 1.25 */
    int64_t solo_min_samples; /* sampled pixels per step from which a job steps on its own stream; <= 0: 131072 */
} lmrs_server_config;

typedef enum { LMRS_JOB_QUEUED = 0, LMRS_JOB_RUNNING = 1, LMRS_JOB_DONE = 2, LMRS_JOB_FAILED = 3 } lmrs_job_state;

typedef struct {
    int32_t state;           /* lmrs_job_state */
    int32_t status;          /* lmrs_status of a failed job, else LMRS_OK */
    int32_t converged;       /* 1: target_loss reached; 0: stopped at max_steps (or not finished) */
    int32_t steps;           /* LM steps run so far */
    double loss;             /* sampled loss of the last step */
    double full_mse;         /* full-frame MSE at the last check (stop_full_frame), -1 if none */
    double t_submit;         /* seconds since the server was created */
    double t_admit;          /* -1 while queued */
    double t_done;           /* -1 until finished */
    int64_t footprint_est;   /* the admission estimate (bytes) */
    int64_t footprint_peak;  /* device bytes the job held at most */
} lmrs_job_info;

typedef struct {
    int32_t queued, active;
    int64_t finished;        /* jobs done or failed */
    int64_t bytes_in_use;    /* device bytes held by the resident jobs */
    int64_t bytes_peak;
    int64_t iterations;      /* scheduler iterations (batched steps) run */
} lmrs_server_stats;

/* Starts the scheduler thread on the current device. */
lmrs_status lmrs_server_create(const lmrs_server_config* cfg, lmrs_server** out);
/* Queues a fit: cfg as for lmrs_scene_create; params_host[P],
 * cams_host[n_cams], targets_host[n_cams][H][W][3] are copied.  Invalid
 * configurations are rejected here; a job whose estimate alone exceeds the
 * budget is rejected with LMRS_ERR_BUDGET. */
lmrs_status lmrs_server_submit(lmrs_server* srv, const lmrs_config* cfg, int64_t n_gauss, const float* params_host,
                               const lmrs_camera* cams_host, int32_t n_cams, const float* targets_host,
                               int32_t views_per_step, double target_loss, int32_t max_steps, int64_t* job_id);
lmrs_status lmrs_server_poll(lmrs_server* srv, int64_t job_id, lmrs_job_info* info);
/* Waits until the job is done or failed; LMRS_ERR_TIMEOUT after timeout_s
 * seconds (info then holds the current state). */
lmrs_status lmrs_server_wait(lmrs_server* srv, int64_t job_id, double timeout_s, lmrs_job_info* info);
/* Final parameters of a done job (P floats, host). */
lmrs_status lmrs_server_result(lmrs_server* srv, int64_t job_id, float* params_host);
/* Drops the record of a finished job. */
lmrs_status lmrs_server_forget(lmrs_server* srv, int64_t job_id);
lmrs_status lmrs_server_get_stats(lmrs_server* srv, lmrs_server_stats* out);
/* Stops the scheduler after its current iteration and waits for it;
 * unfinished jobs end as failed with LMRS_ERR_TIMEOUT. */
lmrs_status lmrs_server_destroy(lmrs_server* srv);

/* Footprint model of the admission test: device bytes of a scene during an
 * LM step with views_per_step views (all when <= 0): 9 P-vectors, the
 * per-Gaussian cache, 290 B per (view, Gaussian) pair plus its Jacobian
 * cache (10 planes of 16 B for SH degree 0, 12 otherwise), the tile entries
 * (tiles_per_pair per pair: ids, the binning's row lists and the compact
 * lists), 41 B per sample (+4 with importance sampling, +24 with the SSIM
 * term), the per-tile tables, the targets, and 25% headroom on the per-step
 * parts.  It is an estimate, not a bound: a scene whose Gaussians cover more
 * tiles than tiles_per_pair holds more, and the server then counts what the
 * job holds. */
int64_t lmrs_footprint_bytes(const lmrs_config* cfg, int64_t n_gauss, int32_t n_cams, int32_t width, int32_t height,
                             int32_t views_per_step, double tiles_per_pair);
/* (sample, Gaussian) pairs composited before termination by the last
 * lmrs_render (alpha >= 1/255 and T still >= 1e-4, Eq. 4): the evaluations
 * each J v and J^T u application repeats.  -1 before a render. */
int64_t lmrs_num_evaluations(lmrs_scene* scene);
/* List entries the derivative kernels walk per application: the sum over
 * work items (up to 32 samples of one tile) of their compact lists, the
 * entries at which some sample of the item has alpha >= 1/255 before it
 * stops, from the last lmrs_render.  -1 before a render. */
int64_t lmrs_num_walked_entries(lmrs_scene* scene);
/* Device bytes the scene holds now. */
int64_t lmrs_scene_device_bytes(const lmrs_scene* scene);

/* Tile-shape autotuner.  The tile shape groups pixels for the per-tile
 * residual sampling (Sec. 4.4) and for the tile lists of every raster pass;
 * the fastest shape depends on the scene.  For each candidate shape
 * (shapes[2i], shapes[2i+1]) = (tile_w, tile_h), tile_w * tile_h <= 256,
 * the tuner builds a private copy of the scene with that shape (cfg
 * otherwise unchanged, except that a fixed samples_per_tile is scaled by
 * the tile area so the sampled fraction stays the same) and times `reps`
 * full LM steps (after one untimed step), each from params_dev, with CUDA
 * events on cuda_stream (NULL: a private stream).  The candidates are
 * different but equally valid samplings of the same objective.
 *   params_dev / targets_dev: as lmrs_scene_create (device, borrowed);
 *   view_ids_host[n_views]: the views of each timed step;
 *   best: index of the shape with the lowest median step time;
 *   ms_per_step[n_shapes]: the medians, or NULL.
 * Returns LMRS_ERR_INVALID_ARG for a bad shape or argument (best = -1);
 * scene-creation and step errors are passed through. */
lmrs_status lmrs_autotune_tile(const lmrs_config* cfg, int64_t n_gauss, const float* params_dev,
                               const lmrs_camera* cams_host, int32_t n_cams, const float* targets_dev,
                               const int32_t* view_ids_host, int32_t n_views, const int32_t* shapes,
                               int32_t n_shapes, int32_t reps, void* cuda_stream, int32_t* best,
                               float* ms_per_step);

/* Introspection (host memory; synchronising).  Sample layout: off[S] is the
 * offset of each sample inside the valid part of its tile (row-major over
 * min(tile_w, remaining width) columns), tile_off[n_views*T + 1] the prefix
 * over tiles.  Tile lists: ranges[n_views*T][2] = [begin, end) into ids[];
 * a Gaussian's list covers the tiles of its 3-sigma rectangle where its
 * alpha can reach 1/255 at a pixel (the ellipse q <= 2 ln(255 o) + 0.02 met
 * by a pixel-centre column within the tile row), so a tile left out changes
 * no pixel.  lmrs_num_pairs is the number of list entries (ids[]); it waits
 * for the preprocessing on the scene's stream; -1 before preprocessing or
 * when that read fails. */
int64_t lmrs_num_params(const lmrs_scene* scene);
int64_t lmrs_num_samples(const lmrs_scene* scene);
int64_t lmrs_num_pairs(const lmrs_scene* scene);
int64_t lmrs_num_visible(const lmrs_scene* scene); /* visible (view, Gaussian) pairs */
lmrs_status lmrs_get_samples(lmrs_scene* scene, uint8_t* off_host, int32_t* tile_off_host);
lmrs_status lmrs_get_tile_lists(lmrs_scene* scene, int32_t* ranges_host, int32_t* ids_host);
/* Per-sample weights w_i (host, S floats): the tile weight of weight_mode for
 * sample_dist 0, 1 / (K_t q(p_i)) otherwise. */
lmrs_status lmrs_get_sample_weights(lmrs_scene* scene, float* w_host);
/* The SSIM term of the last lmrs_render (host, S x 3 floats each, NULL to
 * skip): s = 1 - SSIM and d = ds/dC at each sample's own pixel.
 * LMRS_ERR_INVALID_ARG when ssim_weight is 0. */
lmrs_status lmrs_get_ssim(lmrs_scene* scene, float* s_host, float* d_host);

/* Per-kernel device time, measured with CUDA events recorded on the scene's
 * stream around every launch while timing is enabled (off by default). */
typedef struct {
    char name[64];     /* kernel name */
    int64_t launches;
    double total_ms;   /* sum of the launches' event-to-event times */
} lmrs_kernel_time;

lmrs_status lmrs_set_timing(lmrs_scene* scene, int32_t enable);
/* Synchronises, aggregates the launches timed since the previous call by
 * kernel name into out[0..min(max_entries, n)) and sets *n_entries = n. */
lmrs_status lmrs_get_timing(lmrs_scene* scene, lmrs_kernel_time* out, int32_t max_entries, int32_t* n_entries);

/* Waits for the scene's stream. */
lmrs_status lmrs_synchronize(lmrs_scene* scene);

const char* lmrs_status_str(lmrs_status s);
const char* lmrs_last_error(const lmrs_scene* scene);

/* Number of kernels this library has launched in the process so far. */
int64_t lmrs_launch_count(void);

/* ---- Bounds-checked builds ----------------------------------------------
 * The paper has no counterpart: these stand in for a memory checker on GPUs
 * where none can be run.  A library built with LMRS_DEBUG defined (build.py
 * build(debug=True), into _build_debug/) checks the indexes the rasterisers
 * take from the lists before each access: a Gaussian id of a staged list
 * entry (< G), a compact-list write (< the tile list's length) and the id of
 * every back-scattered entry.  A failed check sets its bit in the scene's
 * debug word and the access uses index 0 instead, so it stays in bounds.
 * Release builds compile the checks away.
 *   lmrs_debug_build: 1 in an LMRS_DEBUG build, else 0.
 *   lmrs_debug_status: the scene's debug word (host, *bits_host; bit 0 a
 *     staged id, bit 1 a compact-list write, bit 2 a back-scattered id),
 *     then cleared; waits for the scene's stream.  Always 0 in release
 *     builds.  LMRS_ERR_INVALID_ARG for a null argument. */
int32_t lmrs_debug_build(void);
lmrs_status lmrs_debug_status(lmrs_scene* scene, uint32_t* bits_host);

/* ---- Peak rates of the current device ------------------------------------
 * Measured by microbenchmarks of this library (the paper has no
 * counterpart: they are the denominators of the raster kernels' roofline,
 * App. A's Jv / J^T v kernels being FP32-, exponential- and atomic-bound).
 * Each kernel runs once untimed and once timed with CUDA events on
 * cuda_stream (NULL = legacy stream):
 *   fp32_tflops / fp64_tflops : fused multiply-adds (2 FLOP each), 8
 *                               independent chains per thread, 64 warps per SM;
 *   ex2_gops                  : 2^x on the special-function unit
 *                               (ex2.approx, as __expf issues it);
 *   atomic_scattered_gops     : float atomic adds, every lane a different
 *                               64-byte slot of a 64 MB buffer (L2-resident);
 *   red_v4_scattered_gops     : the same with 4-wide vector adds (ops, each
 *                               adding 4 floats);
 *   atomic_same_address_gops  : the 32 lanes of a warp on one address.
 * sm_count and sm_clock_max_mhz are the device attributes.  The call
 * allocates and frees a 64 MB scratch buffer and two small output arrays
 * with cudaMalloc, takes a few tens of milliseconds and synchronises.
 * Errors: LMRS_ERR_INVALID_ARG (out NULL), LMRS_ERR_OOM, LMRS_ERR_CUDA. */
typedef struct {
    int32_t sm_count;
    double sm_clock_max_mhz;
    double fp32_tflops, fp64_tflops, ex2_gops;
    double atomic_scattered_gops, red_v4_scattered_gops, atomic_same_address_gops;
} lmrs_peaks;
lmrs_status lmrs_measure_peaks(void* cuda_stream, lmrs_peaks* out);

#ifdef __cplusplus
}
#endif
#endif /* LMRS_H */
