// Tile-shape autotuner (host code over the public C-ABI).
//
// The tile shape sets how pixels are grouped for the per-tile residual
// sampling (Sec. 4.4) and for the tile lists every raster pass walks: a
// wide tile trades a longer per-tile list (more Gaussians overlap its
// perimeter) against fewer tiles per view.  Which shape is fastest depends
// on the Gaussian footprints of the scene, so it is measured: each
// candidate runs full LM steps on a private copy of the scene, timed with
// CUDA events on a private stream, and the shape with the lowest median time
// wins.  The caller's scene is not touched.
#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "lmrs.h"

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Median LM-step time (ms) of one configuration, every rep starting from
// the same parameters.
lmrs_status time_shape(const lmrs_config& cfg, int64_t n_gauss, const float* params, const lmrs_camera* cams,
                       int32_t n_cams, const float* targets, const int32_t* views, int32_t n_views, int32_t reps,
                       int64_t lm_step, cudaStream_t st, float* ms_out) {
    lmrs_scene* s = nullptr;
    lmrs_status rc = lmrs_scene_create(&cfg, n_gauss, params, cams, n_cams, targets, st, &s);
    if (rc != LMRS_OK) return rc;
    EventPair ev;
    std::vector<float> t;
    if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) rc = LMRS_ERR_CUDA;
    // one untimed step first (buffer growth happens there)
    for (int r = -1; rc == LMRS_OK && r < reps; ++r) {
        rc = lmrs_set_params(s, params);
        if (rc != LMRS_OK) break;
        if (cudaEventRecord(ev.a, st) != cudaSuccess) rc = LMRS_ERR_CUDA;
        if (rc == LMRS_OK) rc = lmrs_lm_step(s, views, n_views, lm_step, nullptr);
        if (rc == LMRS_OK && cudaEventRecord(ev.b, st) != cudaSuccess) rc = LMRS_ERR_CUDA;
        if (rc == LMRS_OK && cudaEventSynchronize(ev.b) != cudaSuccess) rc = LMRS_ERR_CUDA;
        float ms = 0.f;
        if (rc == LMRS_OK && cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) rc = LMRS_ERR_CUDA;
        if (rc == LMRS_OK && r >= 0) t.push_back(ms);
    }
    lmrs_scene_destroy(s);
    if (rc != LMRS_OK) {
        cudaGetLastError();
        return rc;
    }
    std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
    *ms_out = t[t.size() / 2];
    return LMRS_OK;
}

}  // namespace

extern "C" lmrs_status lmrs_autotune_tile(const lmrs_config* cfg, int64_t n_gauss, const float* params_dev,
                                          const lmrs_camera* cams_host, int32_t n_cams, const float* targets_dev,
                                          const int32_t* view_ids_host, int32_t n_views, const int32_t* shapes,
                                          int32_t n_shapes, int32_t reps, void* cuda_stream, int32_t* best,
                                          float* ms_per_step) {
    if (!cfg || !params_dev || !cams_host || !targets_dev || !view_ids_host || !shapes || !best || n_shapes <= 0 ||
        n_views <= 0 || reps <= 0)
        return LMRS_ERR_INVALID_ARG;
    *best = -1;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    bool own = false;
    if (!st) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LMRS_ERR_CUDA;
        own = true;
    }
    const double area0 = (double)cfg->tile_w * cfg->tile_h;
    float best_ms = 0.f;
    lmrs_status rc = LMRS_OK;
    for (int i = 0; i < n_shapes && rc == LMRS_OK; ++i) {
        lmrs_config c = *cfg;
        c.tile_w = shapes[2 * i];
        c.tile_h = shapes[2 * i + 1];
        if (c.tile_w <= 0 || c.tile_h <= 0 || c.tile_w * c.tile_h > 256) {
            rc = LMRS_ERR_INVALID_ARG;
            break;
        }
        // a fixed per-tile sample count keeps the same fraction of pixels
        if (cfg->samples_per_tile > 0)
            c.samples_per_tile = std::max(1, (int)(cfg->samples_per_tile * (c.tile_w * c.tile_h) / area0 + 0.5));
        float ms = 0.f;
        rc = time_shape(c, n_gauss, params_dev, cams_host, n_cams, targets_dev, view_ids_host, n_views, reps,
                        (int64_t)cfg->warm_iters, st, &ms);
        if (rc != LMRS_OK) break;
        if (ms_per_step) ms_per_step[i] = ms;
        if (*best < 0 || ms < best_ms) {
            *best = i;
            best_ms = ms;
        }
    }
    if (own) cudaStreamDestroy(st);
    if (rc != LMRS_OK) *best = -1;
    return rc;
}
