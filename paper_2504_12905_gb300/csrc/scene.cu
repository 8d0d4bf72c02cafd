// C-ABI of liblmrs (include/lmrs.h): scene state, buffer management and the
// orchestration of the kernels of one LM step (Alg. 1).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace lmrs {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Per-launch CUDA events on the launching stream, resolved when read.
struct LaunchTimer {
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) {
            e = pool.back();
            pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    }
    ~LaunchTimer() {
        for (auto& r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};
static thread_local LaunchTimer* t_active = nullptr;
LaunchTimer* active_timer() { return t_active; }
int timer_start(LaunchTimer* t, const char* name, cudaStream_t st) {
    LaunchTimer::Rec r{name, t->get(), t->get()};
    cudaEventRecord(r.a, st);
    t->recs.push_back(r);
    return (int)t->recs.size() - 1;
}
void timer_stop(LaunchTimer* t, int i, cudaStream_t st) { cudaEventRecord(t->recs[i].b, st); }
}  // namespace lmrs

using namespace lmrs;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

}  // namespace

struct lmrs_scene {
    lmrs_config cfg;
    int G = 0, deg = 0, K = 0, Pg = 0;
    long long P = 0;
    int n_cams = 0, W = 0, H = 0, tiles_x = 0, tiles_y = 0, T = 0;
    std::vector<lmrs_camera> cams_h;  // host copy (view sampling)
    cudaStream_t st = nullptr;
    std::string err;
    const float* targets = nullptr;
    // device state
    DevBuf params, cams, views, gcache, pjac;
    DevBuf rec, tan, rect, ell, dkeys, dvals, dkeys_alt, dvals_alt, dtmp, cnt, cot, dslot;
    DevBuf keys, ids, keys_alt, ids_alt, ranges, scan_tmp, radix_tmp, total;
    DevBuf tile_off, off, wtile, wsample, work;
    DevBuf item_cost, work_sorted, okeys, ovals, okeys_alt, ovals_alt, otmp;
    DevBuf cids, clen, binmat, bintmp, rowl, tcnt;
    int max_items = 1;
    DevBuf resid, cacheC, cacheT, cacheCh, cacheTh, cacheN;
    DevBuf x, r, z, p, Ap, minv, D, b, stage_a, stage_b;
    DevBuf sc, partials, counter, frames, sqerr;
    DevBuf ssim_s, ssim_d, sframes;  // the SSIM term: per-sample values, full frames of the step's views
    // host state of the current step
    std::vector<int> views_h;
    int nv = 0;
    long long step = 0, S = 0, npairs = 0, nvisible = 0;
    int nwork = 0;
    int layout_nv = -1;
    std::vector<int> tile_off_h;
    bool preprocessed = false, rendered = false, have_D = false;
    bool ordered = false;  // work items in longest-first order (after a render)
    bool timing = false;
    LaunchTimer timer;

    // every device buffer the scene owns
    std::vector<DevBuf*> bufs() {
        return {&params, &cams, &views, &gcache, &pjac, &rec, &tan, &rect, &ell, &dkeys, &dvals, &dkeys_alt, &dvals_alt, &dtmp, &cnt,
                &cot, &dslot, &keys, &ids, &keys_alt, &ids_alt, &ranges, &scan_tmp, &radix_tmp, &total, &tile_off,
                &off, &wtile, &wsample, &work, &item_cost, &work_sorted, &okeys, &ovals, &okeys_alt, &ovals_alt, &otmp,
                &cids, &clen, &binmat, &bintmp, &rowl, &tcnt, &resid, &cacheC, &cacheT, &cacheCh, &cacheTh, &cacheN, &x, &r, &z, &p, &Ap,
                &minv, &D, &b, &stage_a, &stage_b, &sc, &partials, &counter, &frames, &sqerr, &ssim_s, &ssim_d, &sframes};
    }

    Ctx ctx() const {
        Ctx c;
        std::memset(&c, 0, sizeof(c));
        c.G = G; c.deg = deg; c.K = K; c.Pg = Pg; c.P = P;
        c.nv = nv; c.W = W; c.H = H; c.tiles_x = tiles_x; c.tiles_y = tiles_y; c.T = T;
        c.tile_w = cfg.tile_w; c.tile_h = cfg.tile_h;
        c.cache_bf16 = cfg.cache_bf16;
        c.damping_mode = cfg.damping_mode;
        c.lambda = (float)cfg.lambda;
        c.params = params.as<float>();
        c.cams = cams.as<CamDev>();
        c.views = views.as<int>();
        c.targets = targets;
        c.gcache = gcache.as<float4>();
        c.rec = rec.as<float4>();
        c.tan = tan.as<float4>();
        c.pjac = pjac.as<float4>();
        c.rect = rect.as<int4>();
        c.ell = ell.as<float4>();
        c.dkeys = dkeys.as<unsigned long long>();
        c.dvals = dvals.as<unsigned int>();
        c.cnt = cnt.as<unsigned long long>();
        c.n_entries = total.as<unsigned long long>();
        c.n_visible = total.as<unsigned long long>() + 1;
        c.n_rowent = total.as<unsigned long long>() + 2;
        c.cot = cot.as<float>();
        c.dslot = dslot.as<float>();
        c.keys = keys.as<unsigned int>();
        c.ids = ids.as<unsigned int>();
        c.npairs = npairs;
        c.ranges = ranges.as<int2>();
        c.tile_off = tile_off.as<int>();
        c.off = off.as<unsigned char>();
        c.wtile = wtile.as<float>();
        c.wsample = cfg.sample_dist != 0 ? wsample.as<float>() : nullptr;
        c.sample_dist = cfg.sample_dist;
        const bool ssim = cfg.ssim_weight > 0.0;
        c.ssim_s = ssim ? ssim_s.as<float>() : nullptr;
        c.ssim_d = ssim ? ssim_d.as<float>() : nullptr;
        c.ssim_weight = (float)cfg.ssim_weight;
        c.frames = sframes.as<float>();
        c.S = S;
        c.work = ordered ? work_sorted.as<int2>() : work.as<int2>();
        c.item_cost = item_cost.as<int>();
        c.cids = cids.as<unsigned int>();
        c.clen = clen.as<int>();
        c.max_items = max_items;
        c.nwork = nwork;
        c.resid = resid.as<float>();
        c.cacheC = cacheC.as<float>();
        c.cacheT = cacheT.as<float>();
        c.cacheCh = cacheCh.as<__nv_bfloat16>();
        c.cacheTh = cacheTh.as<__nv_bfloat16>();
        c.cacheN = cacheN.as<int>();
        c.sc = sc.as<Scalars>();
        c.partials = partials.as<double>();
        c.counter = counter.as<unsigned int>();
        return c;
    }
};

namespace {

const char* kStatusStr[] = {"LMRS_OK", "LMRS_ERR_INVALID_ARG", "LMRS_ERR_OOM", "LMRS_ERR_CUDA",
                            "LMRS_ERR_NOT_PREPROCESSED", "LMRS_ERR_NUMERIC", "LMRS_ERR_TIMEOUT", "LMRS_ERR_BUDGET"};

lmrs_status fail(lmrs_scene* s, lmrs_status code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

lmrs_status cuda_fail(lmrs_scene* s, cudaError_t e, const char* what) {
    return fail(s, e == cudaErrorMemoryAllocation ? LMRS_ERR_OOM : LMRS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(s, call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
    } while (0)

#define CHECK_LAUNCH(s)                                               \
    do {                                                              \
        cudaError_t e_ = cudaGetLastError();                          \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, "kernel launch"); \
    } while (0)

#define TRY(expr)                        \
    do {                                 \
        lmrs_status st_ = (expr);        \
        if (st_ != LMRS_OK) return st_;  \
    } while (0)

// Routes the launches of one ABI call to the scene's timer when enabled.
struct TimerScope {
    LaunchTimer* prev;
    explicit TimerScope(lmrs_scene* s) : prev(t_active) { t_active = (s && s->timing) ? &s->timer : nullptr; }
    ~TimerScope() { t_active = prev; }
};

// Device memory comes from one stream-ordered pool per device owned by the
// library: allocations and frees are ordered on the owner's stream (no
// device-wide synchronisation, so scenes on different streams keep
// running concurrently when a buffer grows), freed blocks stay in the pool
// for reuse, and the pool never adds hidden cross-stream dependencies.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t lib_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        int no = 0;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// Grows b to at least `bytes` on stream st (contents are not kept).  A
// buffer that has to grow again gets 25% headroom: per-step sizes (pairs,
// samples) drift as the parameters move.
cudaError_t ensure_on(DevBuf& b, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return cudaSuccess;
    const size_t want = b.cap ? bytes + bytes / 4 : bytes;
    if (b.p) {
        cudaError_t e = cudaFreeAsync(b.p, st);
        b.p = nullptr;
        b.cap = 0;
        if (e != cudaSuccess) return e;
    }
    cudaMemPool_t pool = nullptr;
    cudaError_t e = lib_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&b.p, want, pool, st);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.cap = want;
    return cudaSuccess;
}

lmrs_status ensure(lmrs_scene* s, DevBuf& b, size_t bytes) {
    const cudaError_t e = ensure_on(b, bytes, s->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(s, e, "device allocation");
    }
    return LMRS_OK;
}

void release(DevBuf& b, cudaStream_t st) {
    if (b.p) cudaFreeAsync(b.p, st);
    b.p = nullptr;
    b.cap = 0;
}

// Returns the pool's unused blocks to the device (after scenes or batches
// are destroyed).
void trim_pool() {
    cudaMemPool_t pool = nullptr;
    if (lib_pool(&pool) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
}

}  // namespace

namespace lmrs {
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = lib_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
    return e;
}
void pool_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}
void pool_trim() { trim_pool(); }
}  // namespace lmrs

namespace {

bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

CamDev make_cam(const lmrs_camera& c) {
    CamDev d;
    std::memset(&d, 0, sizeof(d));
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) d.R[3 * i + j] = c.world_to_cam[4 * i + j];
        d.t[i] = c.world_to_cam[4 * i + 3];
    }
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.znear = c.znear;
    // FP32 list decisions: the clamp limits in this exact operation order
    d.limx = 1.3f * ((0.5f * (float)c.width) / c.fx);
    d.limy = 1.3f * ((0.5f * (float)c.height) / c.fy);
    for (int j = 0; j < 3; ++j) {
        double v = 0.0;
        for (int k = 0; k < 3; ++k) v -= (double)c.world_to_cam[4 * k + j] * (double)c.world_to_cam[4 * k + 3];
        d.centre[j] = (float)v;  // camera centre -R^T t
    }
    d.W = c.width;
    d.H = c.height;
    return d;
}

int samples_in_tile(const lmrs_config& cfg, int n_valid) {
    int k = cfg.samples_per_tile > 0 ? cfg.samples_per_tile : (int)std::floor(cfg.sample_frac * n_valid + 0.5);
    return std::max(1, std::min(k, n_valid));
}

// Sample layout for nv slots (depends on the image size and config only).
lmrs_status build_layout(lmrs_scene* s) {
    if (s->layout_nv == s->nv) return LMRS_OK;
    const int nT = s->nv * s->T;
    s->max_items = 1;
    std::vector<int> toff(nT + 1, 0);
    std::vector<float> w(nT);
    std::vector<int2> work;
    for (int slot = 0; slot < s->nv; ++slot)
        for (int t = 0; t < s->T; ++t) {
            const int tx = t % s->tiles_x, ty = t / s->tiles_x;
            const int vw = std::min(s->cfg.tile_w, s->W - tx * s->cfg.tile_w);
            const int vh = std::min(s->cfg.tile_h, s->H - ty * s->cfg.tile_h);
            const int n = vw * vh;
            const int k = samples_in_tile(s->cfg, n);
            const int vt = slot * s->T + t;
            toff[vt + 1] = toff[vt] + k;
            w[vt] = s->cfg.weight_mode == 1 ? (float)((double)n / (double)k) : 1.f;
            for (int j = 0; j < k; j += 32) work.push_back(make_int2(vt, j));
            s->max_items = std::max(s->max_items, (k + 31) / 32);
        }
    s->S = toff[nT];
    s->nwork = (int)work.size();
    TRY(ensure(s, s->tile_off, sizeof(int) * (nT + 1)));
    TRY(ensure(s, s->wtile, sizeof(float) * nT));
    TRY(ensure(s, s->work, sizeof(int2) * std::max<size_t>(work.size(), 1)));
    TRY(ensure(s, s->off, (size_t)s->S));
    if (s->cfg.sample_dist != 0) TRY(ensure(s, s->wsample, sizeof(float) * (size_t)s->S));
    if (s->cfg.ssim_weight > 0.0) {
        TRY(ensure(s, s->ssim_s, sizeof(float) * 3 * s->S));
        TRY(ensure(s, s->ssim_d, sizeof(float) * 3 * s->S));
    }
    TRY(ensure(s, s->resid, sizeof(float) * 3 * s->S));
    TRY(ensure(s, s->cacheC, sizeof(float) * 3 * s->S));
    TRY(ensure(s, s->cacheT, sizeof(float) * s->S));
    TRY(ensure(s, s->cacheCh, sizeof(__nv_bfloat16) * 3 * s->S));
    TRY(ensure(s, s->cacheTh, sizeof(__nv_bfloat16) * s->S));
    TRY(ensure(s, s->cacheN, sizeof(int) * s->S));
    const size_t nw = std::max<size_t>(work.size(), 1);
    TRY(ensure(s, s->item_cost, sizeof(int) * nw));
    TRY(ensure(s, s->work_sorted, sizeof(int2) * nw));
    TRY(ensure(s, s->okeys, sizeof(unsigned long long) * nw));
    TRY(ensure(s, s->okeys_alt, sizeof(unsigned long long) * nw));
    TRY(ensure(s, s->ovals, sizeof(unsigned int) * nw));
    TRY(ensure(s, s->ovals_alt, sizeof(unsigned int) * nw));
    TRY(ensure(s, s->otmp, radix_tmp_bytes((long long)nw)));
    TRY(ensure(s, s->clen, sizeof(int) * (size_t)nT * s->max_items));
    // pageable sources: the copies are staged before the calls return
    CK(s, cudaMemcpyAsync(s->tile_off.p, toff.data(), sizeof(int) * (nT + 1), cudaMemcpyHostToDevice, s->st));
    CK(s, cudaMemcpyAsync(s->wtile.p, w.data(), sizeof(float) * nT, cudaMemcpyHostToDevice, s->st));
    if (!work.empty())
        CK(s, cudaMemcpyAsync(s->work.p, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    s->tile_off_h = toff;
    s->layout_nv = s->nv;
    return LMRS_OK;
}

lmrs_status check_scene(lmrs_scene* s) { return s ? LMRS_OK : LMRS_ERR_INVALID_ARG; }

lmrs_status need_pre(lmrs_scene* s) {
    if (!s->preprocessed) return fail(s, LMRS_ERR_NOT_PREPROCESSED, "lmrs_preprocess has not been called");
    return LMRS_OK;
}
lmrs_status need_render(lmrs_scene* s) {
    TRY(need_pre(s));
    if (!s->rendered) return fail(s, LMRS_ERR_NOT_PREPROCESSED, "lmrs_render has not been called");
    return LMRS_OK;
}

lmrs_status do_jtj_diag(lmrs_scene* s) {
    const size_t pairs = (size_t)s->nv * s->G;
    TRY(ensure(s, s->dslot, sizeof(float) * kDiagF * pairs));
    CK(s, cudaMemsetAsync(s->dslot.p, 0, sizeof(float) * kDiagF * pairs, s->st));
    Ctx c = s->ctx();
    launch_raster_diag(c, s->st);
    launch_prep_diag(c, s->D.as<float>(), s->st);
    CHECK_LAUNCH(s);
    s->have_D = true;
    return LMRS_OK;
}

// Right-hand side J^T W r -> b and diag(J^T W J) -> D of an LM step in one
// walk of the compact lists (k_diag<rhs>), then their parameter-level
// kernels: the same results as lmrs_rhs followed by do_jtj_diag.
lmrs_status do_rhs_diag(lmrs_scene* s, float* b) {
    TRY(need_render(s));
    const size_t pairs = (size_t)s->nv * s->G;
    TRY(ensure(s, s->dslot, sizeof(float) * kDiagF * pairs));
    CK(s, cudaMemsetAsync(s->dslot.p, 0, sizeof(float) * kDiagF * pairs, s->st));
    CK(s, cudaMemsetAsync(s->cot.p, 0, sizeof(float) * kCotF * pairs, s->st));
    Ctx c = s->ctx();
    launch_raster_diag_rhs(c, s->st);
    launch_prep_diag(c, s->D.as<float>(), s->st);
    launch_prep_vjp(c, b, nullptr, nullptr, false, s->st);
    CHECK_LAUNCH(s);
    s->have_D = true;
    return LMRS_OK;
}

// (J^T W J + lambda damp) v -> out, device pointers.
lmrs_status do_jtjv(lmrs_scene* s, const float* v, float* out) {
    Ctx c = s->ctx();
    launch_prep_jvp(c, v, s->st);
    launch_raster_jtj(c, s->st);
    launch_prep_vjp(c, out, v, s->D.as<float>(), false, s->st);
    CHECK_LAUNCH(s);
    return LMRS_OK;
}

lmrs_status do_cg(lmrs_scene* s, const float* b, float* x, int iters) {
    Ctx c = s->ctx();
    float* r = s->r.as<float>();
    float* z = s->z.as<float>();
    float* p = s->p.as<float>();
    float* Ap = s->Ap.as<float>();
    float* minv = s->minv.as<float>();
    const float* D = s->D.as<float>();
    launch_zero_scalars(c, s->st);
    launch_precond(c, D, minv, s->st);
    launch_cg_init(c, b, minv, x, r, z, p, s->st);
    for (int it = 0; it < iters; ++it) {
        launch_prep_jvp_direction(c, z, p, s->st);       // p = z + beta p, tangent features of p
        launch_raster_jtj(c, s->st);                     // J^T W J p into the cotangent slots
        launch_prep_vjp(c, Ap, p, D, true, s->st);       // Ap (+ damping), p^T A p, alpha
        launch_cg_update(c, it, p, Ap, minv, x, r, z, s->st);  // x, r, z, beta
    }
    CHECK_LAUNCH(s);
    return LMRS_OK;
}

lmrs_status lm_step_iters(lmrs_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step, int iters,
                          lmrs_step_stats* st);

// Tile-list entries of the preprocessed step: known on the host after the
// emission path, read from the scalars (one small copy) after the binning
// path; -1 when the copy fails.
long long pairs_exact(lmrs_scene* s) {
    if (s->npairs < 0) {
        unsigned int n = 0u;
        if (cudaMemcpyAsync(&n, &s->sc.as<Scalars>()->n_list, sizeof(n), cudaMemcpyDeviceToHost, s->st) !=
                cudaSuccess ||
            cudaStreamSynchronize(s->st) != cudaSuccess)
            return -1;
        s->npairs = (long long)n;
    }
    return s->npairs;
}

lmrs_status read_scalars(lmrs_scene* s, Scalars* h) {
    CK(s, cudaMemcpyAsync(h, s->sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

}  // namespace

extern "C" {

lmrs_status lmrs_config_default(lmrs_config* cfg) {
    if (!cfg) return LMRS_ERR_INVALID_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->sh_degree = 0;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->sample_frac = 1.0;
    cfg->samples_per_tile = 0;
    cfg->weight_mode = 0;
    cfg->lambda = 0.1;
    cfg->damping_mode = 1;
    cfg->cg_iters = 8;
    cfg->lr_warm = 0.05;
    cfg->lr_cap = 0.2;
    cfg->color_bound = 1.0;
    cfg->warm_iters = 10;
    cfg->cache_bf16 = 0;
    cfg->seed = 0;
    return LMRS_OK;
}

lmrs_status lmrs_scene_create(const lmrs_config* cfg, int64_t n_gauss, const float* params,
                              const lmrs_camera* cams_host, int32_t n_cams, const float* targets_dev,
                              void* cuda_stream, lmrs_scene** out) {
    if (!out) return LMRS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || !params || !cams_host || n_cams <= 0 || n_gauss <= 0 || n_gauss > (1ll << 30))
        return LMRS_ERR_INVALID_ARG;
    if (cfg->sh_degree < 0 || cfg->sh_degree > 3 || cfg->tile_w <= 0 || cfg->tile_h <= 0 ||
        cfg->tile_w * cfg->tile_h > 256 || !(cfg->sample_frac > 0.0) || cfg->cg_iters < 0 ||
        (cfg->damping_mode != 0 && cfg->damping_mode != 1) || (cfg->weight_mode != 0 && cfg->weight_mode != 1) ||
        !(cfg->lambda >= 0.0) || cfg->sample_dist < 0 || cfg->sample_dist > 2 ||
        !(cfg->ssim_weight >= 0.0 && cfg->ssim_weight < 1e30))
        return LMRS_ERR_INVALID_ARG;
    for (int i = 0; i < n_cams; ++i)
        if (cams_host[i].width != cams_host[0].width || cams_host[i].height != cams_host[0].height ||
            cams_host[i].width <= 0 || cams_host[i].height <= 0 || !(cams_host[i].fx > 0.f) || !(cams_host[i].fy > 0.f))
            return LMRS_ERR_INVALID_ARG;
    lmrs_scene* s = new lmrs_scene();
    s->cfg = *cfg;
    s->G = (int)n_gauss;
    s->deg = cfg->sh_degree;
    s->K = (s->deg + 1) * (s->deg + 1);
    s->Pg = 11 + 3 * s->K;
    s->P = (long long)s->G * s->Pg;
    s->n_cams = n_cams;
    s->W = cams_host[0].width;
    s->H = cams_host[0].height;
    s->tiles_x = (s->W + cfg->tile_w - 1) / cfg->tile_w;
    s->tiles_y = (s->H + cfg->tile_h - 1) / cfg->tile_h;
    s->T = s->tiles_x * s->tiles_y;
    s->st = static_cast<cudaStream_t>(cuda_stream);
    s->targets = targets_dev;
    set_sh_constants();
    lmrs_status rc = LMRS_OK;
    auto take = [&](DevBuf& b, size_t bytes) {
        if (rc == LMRS_OK) rc = ensure(s, b, bytes);
    };
    const size_t pv = sizeof(float) * (size_t)s->P;
    take(s->params, pv);
    for (DevBuf* b : {&s->x, &s->r, &s->z, &s->p, &s->Ap, &s->minv, &s->D, &s->b}) take(*b, pv);
    take(s->cams, sizeof(CamDev) * n_cams);
    take(s->gcache, sizeof(float4) * kGaussF4 * (size_t)s->G);
    take(s->sc, sizeof(Scalars));
    take(s->partials, sizeof(double) * kMaxPartials);
    take(s->counter, sizeof(unsigned int) * 4);
    take(s->total, sizeof(unsigned long long) * 4);
    if (rc != LMRS_OK) {
        lmrs_scene_destroy(s);
        return rc;
    }
    s->cams_h.assign(cams_host, cams_host + n_cams);
    std::vector<CamDev> cd(n_cams);
    for (int i = 0; i < n_cams; ++i) cd[i] = make_cam(cams_host[i]);
    // the stream-ordered allocations are complete before the synchronous
    // copies below (which keep the legacy-stream ordering with the caller)
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess) e = cudaMemcpy(s->cams.p, cd.data(), sizeof(CamDev) * n_cams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->params.p, params, pv, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemset(s->counter.p, 0, sizeof(unsigned int) * 4);
    if (e == cudaSuccess) e = cudaMemset(s->sc.p, 0, sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMemset(s->D.p, 0, pv);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lmrs_scene_destroy(s);
        return e == cudaErrorMemoryAllocation ? LMRS_ERR_OOM : LMRS_ERR_CUDA;
    }
    *out = s;
    return LMRS_OK;
}

lmrs_status lmrs_scene_destroy(lmrs_scene* s) {
    if (!s) return LMRS_ERR_INVALID_ARG;
    if (s->st) cudaStreamSynchronize(s->st);
    for (DevBuf* b : s->bufs())
        release(*b, s->st);
    cudaStreamSynchronize(s->st);
    trim_pool();
    delete s;
    return LMRS_OK;
}

lmrs_status lmrs_set_params(lmrs_scene* s, const float* src) {
    TRY(check_scene(s));
    if (!src) return fail(s, LMRS_ERR_INVALID_ARG, "null source");
    CK(s, cudaMemcpyAsync(s->params.p, src, sizeof(float) * s->P, cudaMemcpyDefault, s->st));
    s->preprocessed = s->rendered = s->have_D = s->ordered = false;
    return LMRS_OK;
}

lmrs_status lmrs_get_params(lmrs_scene* s, float* dst) {
    TRY(check_scene(s));
    if (!dst) return fail(s, LMRS_ERR_INVALID_ARG, "null destination");
    CK(s, cudaMemcpyAsync(dst, s->params.p, sizeof(float) * s->P, cudaMemcpyDefault, s->st));
    if (!is_device_ptr(dst)) CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

lmrs_status lmrs_get_solution(lmrs_scene* s, float* dst) {
    TRY(check_scene(s));
    if (!dst) return fail(s, LMRS_ERR_INVALID_ARG, "null destination");
    CK(s, cudaMemcpyAsync(dst, s->x.p, sizeof(float) * s->P, cudaMemcpyDefault, s->st));
    if (!is_device_ptr(dst)) CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

lmrs_status lmrs_preprocess(lmrs_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!view_ids || n_views <= 0) return fail(s, LMRS_ERR_INVALID_ARG, "no views");
    for (int i = 0; i < n_views; ++i)
        if (view_ids[i] < 0 || view_ids[i] >= s->n_cams) return fail(s, LMRS_ERR_INVALID_ARG, "view id out of range");
    if ((long long)n_views * s->T >= (1ll << 31) || (long long)n_views * s->G >= (1ll << 31))
        return fail(s, LMRS_ERR_BUDGET, "too many (view, tile) or (view, Gaussian) pairs");
    s->preprocessed = s->rendered = s->have_D = s->ordered = false;
    s->views_h.assign(view_ids, view_ids + n_views);
    s->nv = n_views;
    s->step = lm_step;
    const size_t pairs = (size_t)s->nv * s->G;
    TRY(ensure(s, s->views, sizeof(int) * n_views));
    TRY(ensure(s, s->rec, sizeof(float4) * kPrimF4 * pairs));
    TRY(ensure(s, s->tan, sizeof(float4) * kTanF4 * pairs));
    // blocked by 32 pairs, each view's Gaussians padded to a multiple of 32
    TRY(ensure(s, s->pjac, sizeof(float4) * jac_f4(s->deg) * (size_t)s->nv * (size_t)((s->G + 31) & ~31)));
    TRY(ensure(s, s->rect, sizeof(int4) * pairs));
    TRY(ensure(s, s->ell, 2 * sizeof(float4) * pairs));
    TRY(ensure(s, s->dkeys, sizeof(unsigned long long) * pairs));
    TRY(ensure(s, s->dkeys_alt, sizeof(unsigned long long) * pairs));
    TRY(ensure(s, s->dvals, sizeof(unsigned int) * pairs));
    TRY(ensure(s, s->dvals_alt, sizeof(unsigned int) * pairs));
    TRY(ensure(s, s->dtmp, radix_tmp_bytes((long long)pairs)));
    TRY(ensure(s, s->cot, sizeof(float) * kCotF * pairs));
    TRY(ensure(s, s->ranges, sizeof(int2) * (size_t)s->nv * s->T));
    TRY(build_layout(s));
    CK(s, cudaMemcpyAsync(s->views.p, s->views_h.data(), sizeof(int) * n_views, cudaMemcpyHostToDevice, s->st));
    Ctx c = s->ctx();
    // tile lists: two-level (rows, tiles) binning, or entry emission + tile
    // sort for views whose tile rows or columns exceed the shared counters
    const bool rows = bin_rows_fit(c);
    if (!rows) {
        TRY(ensure(s, s->cnt, sizeof(unsigned long long) * pairs));
        TRY(ensure(s, s->scan_tmp, scan_u64_tmp_bytes((long long)pairs)));
        c = s->ctx();
    }
    // total[0]: tile-list entries, [1]: visible pairs, [2]: row-list entries
    // (all from the projection), [3]: the two 32-bit scan totals
    CK(s, cudaMemsetAsync(s->total.p, 0, 4 * sizeof(unsigned long long), s->st));
    if (s->cfg.sample_dist == 0) launch_sample(c, lm_step, s->cfg.seed, s->st);  // importance draws follow the binning
    launch_prep_gauss(c, s->st);
    launch_prep_fwd(c, s->st);
    // (slot, depth, index) order of the pairs
    int sbits = 0;
    while ((1 << sbits) < s->nv) ++sbits;
    radix_sort(c.dkeys, c.dvals, s->dkeys_alt.as<unsigned long long>(), s->dvals_alt.as<unsigned int>(),
               (long long)pairs, 32 + sbits, s->dtmp.p, s->dtmp.cap, s->st);
    if (!rows) {
        launch_sorted_counts(c, s->st);
        scan_u64(c.cnt, (long long)pairs, s->total.as<unsigned long long>(), s->scan_tmp.p, s->scan_tmp.cap, s->st);
    }
    CHECK_LAUNCH(s);
    unsigned long long tot[3] = {0ull, 0ull, 0ull};
    CK(s, cudaMemcpyAsync(tot, s->total.p, sizeof(tot), cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    // the emission path counted the entries exactly; the binning path has a
    // bound here and writes the exact number to the scalars (pairs_exact)
    const unsigned long long total = tot[0];
    s->nvisible = (long long)tot[1];
    if (total >= (1ull << 31)) return fail(s, LMRS_ERR_BUDGET, "more than 2^31 (view, tile, Gaussian) pairs");
    s->npairs = rows ? -1 : (long long)total;
    const size_t np = std::max<size_t>((size_t)total, 1);
    TRY(ensure(s, s->ids, sizeof(unsigned int) * np));
    TRY(ensure(s, s->cids, sizeof(unsigned int) * np * (size_t)s->max_items));
    if (rows) {
        const size_t nmat = bin_row_mat_elems(c), nvt = bin_tile_count_elems(c);
        TRY(ensure(s, s->binmat, sizeof(unsigned) * nmat));
        TRY(ensure(s, s->tcnt, sizeof(unsigned) * nvt));
        TRY(ensure(s, s->rowl, sizeof(unsigned long long) * std::max<size_t>((size_t)tot[2], 1)));
        TRY(ensure(s, s->bintmp, bin_scan_tmp_bytes((long long)std::max(nmat, nvt))));
        c = s->ctx();
        unsigned* total32 = reinterpret_cast<unsigned*>(s->total.as<unsigned long long>() + 3);
        bin_rows(c, s->binmat.as<unsigned>(), s->rowl.as<unsigned long long>(), total32, s->bintmp.p, s->st);
        bin_tiles(c, s->binmat.as<unsigned>(), total32, s->rowl.as<unsigned long long>(), s->tcnt.as<unsigned>(),
                  total32 + 1, s->bintmp.p, s->st);
    } else {
        TRY(ensure(s, s->keys, sizeof(unsigned int) * np));
        TRY(ensure(s, s->keys_alt, sizeof(unsigned int) * np));
        TRY(ensure(s, s->ids_alt, sizeof(unsigned int) * np));
        TRY(ensure(s, s->radix_tmp, radix_tmp_bytes((long long)np)));
        c = s->ctx();
        // entries in depth order, then a stable sort on the (slot, tile) bits
        launch_emit(c, s->st);
        int vbits = 0;
        while ((1ll << vbits) < (long long)s->nv * s->T) ++vbits;
        radix_sort32(c.keys, c.ids, s->keys_alt.as<unsigned int>(), s->ids_alt.as<unsigned int>(), s->npairs, vbits,
                     s->radix_tmp.p, s->radix_tmp.cap, s->st);
        CK(s, cudaMemsetAsync(s->ranges.p, 0, sizeof(int2) * (size_t)s->nv * s->T, s->st));
        launch_ranges(c, s->st);
    }
    if (s->cfg.sample_dist != 0) launch_importance(c, lm_step, s->cfg.seed, s->st);
    CHECK_LAUNCH(s);
    s->preprocessed = true;
    return LMRS_OK;
}

}  // extern "C"

namespace {

// The forward render of a step; with_ssim adds the SSIM term of the samples
// (full frames of the step's views, then k_ssim).
lmrs_status do_render(lmrs_scene* s, float* images_dev, float* residuals_dev, bool with_ssim) {
    TimerScope ts_(s);
    TRY(need_pre(s));
    s->ordered = false;  // the forward render indexes the work items in their natural order
    const bool ssim = with_ssim && s->cfg.ssim_weight > 0.0;
    const size_t frames = (size_t)s->nv * s->H * s->W * 3;
    if (ssim) TRY(ensure(s, s->sframes, sizeof(float) * frames));
    Ctx c = s->ctx();
    CK(s, cudaMemsetAsync(&c.sc->loss_num, 0, offsetof(Scalars, eta) - offsetof(Scalars, loss_num), s->st));
    launch_raster_fwd_samples(c, s->st);
    if (ssim) {
        launch_raster_full(c, s->sframes.as<float>(), s->st);
        launch_ssim(c, s->st);
        if (images_dev)
            CK(s, cudaMemcpyAsync(images_dev, s->sframes.p, sizeof(float) * frames, cudaMemcpyDeviceToDevice, s->st));
    } else if (images_dev) {
        launch_raster_full(c, images_dev, s->st);
    }
    launch_order_work(c, s->okeys.as<unsigned long long>(), s->ovals.as<unsigned int>(),
                      s->okeys_alt.as<unsigned long long>(), s->ovals_alt.as<unsigned int>(), s->otmp.p, s->otmp.cap,
                      s->work_sorted.as<int2>(), s->st);
    CHECK_LAUNCH(s);
    s->ordered = true;
    if (residuals_dev)
        CK(s, cudaMemcpyAsync(residuals_dev, s->resid.p, sizeof(float) * 3 * s->S, cudaMemcpyDeviceToDevice, s->st));
    s->rendered = true;
    return LMRS_OK;
}

}  // namespace

extern "C" {

lmrs_status lmrs_render(lmrs_scene* s, float* images_dev, float* residuals_dev) {
    TRY(check_scene(s));
    return do_render(s, images_dev, residuals_dev, true);
}

lmrs_status lmrs_jvp(lmrs_scene* s, const float* v, float* u) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!v || !u) return fail(s, LMRS_ERR_INVALID_ARG, "null vector");
    TRY(need_pre(s));
    Ctx c = s->ctx();
    launch_prep_jvp(c, v, s->st);
    launch_raster_jvp(c, u, s->st);
    CHECK_LAUNCH(s);
    return LMRS_OK;
}

lmrs_status lmrs_vjp(lmrs_scene* s, const float* u, float* g) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!u || !g) return fail(s, LMRS_ERR_INVALID_ARG, "null vector");
    TRY(need_render(s));
    Ctx c = s->ctx();
    CK(s, cudaMemsetAsync(s->cot.p, 0, sizeof(float) * kCotF * (size_t)s->nv * s->G, s->st));
    launch_raster_vjp(c, u, s->st);
    launch_prep_vjp(c, g, nullptr, nullptr, false, s->st);
    CHECK_LAUNCH(s);
    return LMRS_OK;
}

lmrs_status lmrs_rhs(lmrs_scene* s, float* b) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!b) return fail(s, LMRS_ERR_INVALID_ARG, "null vector");
    TRY(need_render(s));
    Ctx c = s->ctx();
    CK(s, cudaMemsetAsync(s->cot.p, 0, sizeof(float) * kCotF * (size_t)s->nv * s->G, s->st));
    launch_raster_vjp(c, nullptr, s->st);
    launch_prep_vjp(c, b, nullptr, nullptr, false, s->st);
    CHECK_LAUNCH(s);
    return LMRS_OK;
}

lmrs_status lmrs_jtj_diag(lmrs_scene* s, float* d) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    TRY(need_render(s));
    TRY(do_jtj_diag(s));
    if (d) CK(s, cudaMemcpyAsync(d, s->D.p, sizeof(float) * s->P, cudaMemcpyDeviceToDevice, s->st));
    return LMRS_OK;
}

lmrs_status lmrs_jtjv(lmrs_scene* s, const float* v, float* out) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!v || !out) return fail(s, LMRS_ERR_INVALID_ARG, "null vector");
    TRY(need_pre(s));
    if (s->cfg.damping_mode == 1 && !s->have_D)
        return fail(s, LMRS_ERR_NOT_PREPROCESSED, "diagonal damping needs lmrs_jtj_diag first");
    const size_t pv = sizeof(float) * s->P;
    const bool vdev = is_device_ptr(v), odev = is_device_ptr(out);
    const float* vin = v;
    float* o = out;
    if (!vdev) {
        TRY(ensure(s, s->stage_a, pv));
        CK(s, cudaMemcpyAsync(s->stage_a.p, v, pv, cudaMemcpyHostToDevice, s->st));
        vin = s->stage_a.as<float>();
    }
    if (!odev) {
        TRY(ensure(s, s->stage_b, pv));
        o = s->stage_b.as<float>();
    }
    TRY(do_jtjv(s, vin, o));
    if (!odev) {
        CK(s, cudaMemcpyAsync(out, o, pv, cudaMemcpyDeviceToHost, s->st));
        CK(s, cudaStreamSynchronize(s->st));
    }
    return LMRS_OK;
}

lmrs_status lmrs_cg_solve(lmrs_scene* s, const float* b, float* x, int32_t iters, lmrs_cg_stats* st) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!b || !x || iters < 0) return fail(s, LMRS_ERR_INVALID_ARG, "bad CG arguments");
    TRY(need_pre(s));
    if (!s->have_D) return fail(s, LMRS_ERR_NOT_PREPROCESSED, "CG needs lmrs_jtj_diag (preconditioner) first");
    TRY(do_cg(s, b, x, iters));
    if (st) {
        Scalars h;
        TRY(read_scalars(s, &h));
        std::memset(st, 0, sizeof(*st));
        st->rz0 = h.rz0;
        st->rz_final = h.rz;
        st->iters = iters;
        for (int i = 0; i < std::min(iters, 64); ++i) {
            st->alpha[i] = h.alpha_hist[i];
            st->beta[i] = h.beta_hist[i];
        }
        if (h.numeric_error) return fail(s, LMRS_ERR_NUMERIC, "non-finite or non-positive CG curvature");
    }
    return LMRS_OK;
}

lmrs_status lmrs_step_size(lmrs_scene* s, const float* x, int64_t lm_step, double* eta) {
    TRY(check_scene(s));
    TimerScope ts_(s);
    if (!x || !eta) return fail(s, LMRS_ERR_INVALID_ARG, "null argument");
    Ctx c = s->ctx();
    CK(s, cudaMemsetAsync(&c.sc->max_dc_bits, 0, sizeof(unsigned int), s->st));
    launch_max_dc(c, x, s->st);
    CHECK_LAUNCH(s);
    Scalars h;
    TRY(read_scalars(s, &h));
    float m;
    std::memcpy(&m, &h.max_dc_bits, sizeof(m));
    if (lm_step < s->cfg.warm_iters) *eta = s->cfg.lr_warm;
    else if (m == 0.f) *eta = s->cfg.lr_cap;
    else *eta = std::fmin(s->cfg.lr_cap, s->cfg.color_bound / (double)m);
    return LMRS_OK;
}

lmrs_status lmrs_lm_step(lmrs_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step,
                         lmrs_step_stats* st) {
    TRY(check_scene(s));
    return lm_step_iters(s, view_ids, n_views, lm_step, s->cfg.cg_iters, st);
}

}  // extern "C"

namespace {

// A named range on the host timeline of a profiler (NVTX; without a tool
// attached the calls return at once), closed when it goes out of scope.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// One LM step (Alg. 1) with `iters` PCG iterations.
lmrs_status lm_step_iters(lmrs_scene* s, const int32_t* view_ids, int32_t n_views, int64_t lm_step, int iters,
                          lmrs_step_stats* st) {
    TimerScope ts_(s);
    NvtxRange step_("lmrs_lm_step");
    {
        NvtxRange r_("preprocess");
        TRY(lmrs_preprocess(s, view_ids, n_views, lm_step));
    }
    {
        NvtxRange r_("render");
        TRY(lmrs_render(s, nullptr, nullptr));
    }
    {
        NvtxRange r_("rhs_diag");
        TRY(do_rhs_diag(s, s->b.as<float>()));
    }
    {
        NvtxRange r_("pcg");
        TRY(do_cg(s, s->b.as<float>(), s->x.as<float>(), iters));
    }
    NvtxRange u_("update");
    Ctx c = s->ctx();
    CK(s, cudaMemsetAsync(&c.sc->max_dc_bits, 0, sizeof(unsigned int), s->st));
    launch_max_dc(c, s->x.as<float>(), s->st);
    launch_lm_update(c, lm_step, s->cfg.lr_warm, s->cfg.lr_cap, s->cfg.color_bound, s->cfg.warm_iters,
                     s->x.as<float>(), s->params.as<float>(), s->st);
    CHECK_LAUNCH(s);
    // the parameters changed: the per-step state no longer describes them
    s->preprocessed = s->rendered = s->have_D = s->ordered = false;
    if (st) {
        Scalars h;
        TRY(read_scalars(s, &h));
        float m;
        std::memcpy(&m, &h.max_dc_bits, sizeof(m));
        st->loss = h.loss_den > 0.0 ? h.loss_num / h.loss_den : 0.0;
        st->eta = h.eta;
        st->max_dc = m;
        st->rz0 = h.rz0;
        st->rz_final = h.rz;
        st->n_samples = s->S;
        st->n_pairs = s->npairs >= 0 ? s->npairs : (int64_t)h.n_list;
        if (h.numeric_error) return fail(s, LMRS_ERR_NUMERIC, "non-finite or non-positive CG curvature");
    }
    return LMRS_OK;
}

}  // namespace

extern "C" {

lmrs_status lmrs_eval_mse(lmrs_scene* s, double* mse) {
    TRY(check_scene(s));
    if (!mse) return fail(s, LMRS_ERR_INVALID_ARG, "null output");
    if (!s->targets) return fail(s, LMRS_ERR_INVALID_ARG, "the scene has no targets");
    constexpr int kChunk = 8;
    const size_t frame = (size_t)s->H * s->W * 3;
    TRY(ensure(s, s->frames, sizeof(float) * frame * std::min(kChunk, s->n_cams)));
    TRY(ensure(s, s->sqerr, sizeof(double)));
    CK(s, cudaMemsetAsync(s->sqerr.p, 0, sizeof(double), s->st));
    std::vector<int32_t> views;
    for (int c0 = 0; c0 < s->n_cams; c0 += kChunk) {
        views.clear();
        for (int v = c0; v < std::min(s->n_cams, c0 + kChunk); ++v) views.push_back(v);
        TRY(lmrs_preprocess(s, views.data(), (int32_t)views.size(), 0));
        TRY(do_render(s, s->frames.as<float>(), nullptr, false));
        TimerScope ts_(s);
        launch_frame_sqerr(s->ctx(), s->frames.as<float>(), s->sqerr.as<double>(), s->st);
        CHECK_LAUNCH(s);
    }
    double sum = 0.0;
    CK(s, cudaMemcpyAsync(&sum, s->sqerr.p, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    *mse = sum / ((double)s->n_cams * (double)frame);
    return LMRS_OK;
}

lmrs_status lmrs_fit(lmrs_scene* s, const lmrs_fit_config* f, lmrs_fit_record* rec) {
    TRY(check_scene(s));
    if (!f || !rec || f->n_steps <= 0 || f->views_first <= 0 || f->views_later <= 0 || f->cg_first < 0 ||
        f->cg_later < 0 || (f->view_mode != 0 && f->view_mode != 1))
        return fail(s, LMRS_ERR_INVALID_ARG, "bad fit configuration");
    if (f->eval_every > 0 && !s->targets) return fail(s, LMRS_ERR_INVALID_ARG, "evaluation needs targets");
    lmrs_view_sampler* smp = nullptr;
    int smp_k = -1;
    std::vector<int32_t> views(s->n_cams);
    lmrs_status rc = LMRS_OK;
    for (int k = 0; k < f->n_steps && rc == LMRS_OK; ++k) {
        const bool early = k < f->switch_step;
        const int nvk = std::min(s->n_cams, early ? f->views_first : f->views_later);
        const int iters = early ? f->cg_first : f->cg_later;
        int32_t nv = nvk;
        if (f->view_mode == 1) {
            if (smp_k != nvk) {
                if (smp) lmrs_view_sampler_destroy(smp);
                smp = nullptr;
                rc = lmrs_view_sampler_create(s->cams_h.data(), s->n_cams, nvk, f->seed, &smp);
                if (rc != LMRS_OK) break;
                smp_k = nvk;
            }
            lmrs_view_sampler_draw(smp, k, views.data(), &nv);
        } else {
            lmrs_uniform_views(s->n_cams, nvk, f->seed, k, views.data());
        }
        const auto t0 = std::chrono::steady_clock::now();
        lmrs_step_stats st;
        rc = lm_step_iters(s, views.data(), nv, k, iters, &st);
        const auto t1 = std::chrono::steady_clock::now();
        if (rc != LMRS_OK) break;
        lmrs_fit_record& r = rec[k];
        r.step = k;
        r.n_views = nv;
        r.cg_iters = iters;
        r.loss = st.loss;
        r.eta = st.eta;
        r.ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        r.mse_full = -1.0;
        r.psnr = -1.0;
        if (f->eval_every > 0 && ((k + 1) % f->eval_every == 0 || k + 1 == f->n_steps)) {
            double m = 0.0;
            rc = lmrs_eval_mse(s, &m);
            r.mse_full = m;
            r.psnr = m > 0.0 ? -10.0 * std::log10(m) : INFINITY;
        }
    }
    if (smp) lmrs_view_sampler_destroy(smp);
    return rc;
}

lmrs_status lmrs_set_timing(lmrs_scene* s, int32_t enable) {
    TRY(check_scene(s));
    s->timing = enable != 0;
    return LMRS_OK;
}

lmrs_status lmrs_get_timing(lmrs_scene* s, lmrs_kernel_time* out, int32_t max_entries, int32_t* n_entries) {
    TRY(check_scene(s));
    if (!n_entries || (max_entries > 0 && !out)) return fail(s, LMRS_ERR_INVALID_ARG, "null output");
    CK(s, cudaStreamSynchronize(s->st));
    std::vector<lmrs_kernel_time> agg;
    for (auto& r : s->timer.recs) {
        float ms = 0.f;
        CK(s, cudaEventElapsedTime(&ms, r.a, r.b));
        lmrs_kernel_time* k = nullptr;
        for (auto& e : agg)
            if (std::strncmp(e.name, r.name, sizeof(e.name) - 1) == 0) k = &e;
        if (!k) {
            lmrs_kernel_time e;
            std::memset(&e, 0, sizeof(e));
            std::strncpy(e.name, r.name, sizeof(e.name) - 1);
            agg.push_back(e);
            k = &agg.back();
        }
        k->launches += 1;
        k->total_ms += ms;
        s->timer.pool.push_back(r.a);
        s->timer.pool.push_back(r.b);
    }
    s->timer.recs.clear();
    *n_entries = (int32_t)agg.size();
    for (int i = 0; i < (int)agg.size() && i < max_entries; ++i) out[i] = agg[i];
    return LMRS_OK;
}

int64_t lmrs_num_params(const lmrs_scene* s) { return s ? s->P : -1; }
int64_t lmrs_num_samples(const lmrs_scene* s) { return s && s->layout_nv >= 0 ? s->S : -1; }
int64_t lmrs_num_pairs(const lmrs_scene* s) {
    return s && s->preprocessed ? pairs_exact(const_cast<lmrs_scene*>(s)) : -1;
}
int64_t lmrs_num_visible(const lmrs_scene* s) { return s && s->preprocessed ? s->nvisible : -1; }

lmrs_status lmrs_get_samples(lmrs_scene* s, uint8_t* off, int32_t* tile_off) {
    TRY(check_scene(s));
    TRY(need_pre(s));
    if (off) CK(s, cudaMemcpyAsync(off, s->off.p, (size_t)s->S, cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    if (tile_off) std::copy(s->tile_off_h.begin(), s->tile_off_h.end(), tile_off);
    return LMRS_OK;
}

lmrs_status lmrs_get_tile_lists(lmrs_scene* s, int32_t* ranges, int32_t* ids) {
    TRY(check_scene(s));
    TRY(need_pre(s));
    if (ranges)
        CK(s, cudaMemcpyAsync(ranges, s->ranges.p, sizeof(int2) * (size_t)s->nv * s->T, cudaMemcpyDeviceToHost, s->st));
    const long long n = pairs_exact(s);
    if (n < 0) return fail(s, LMRS_ERR_CUDA, "reading the tile-list size");
    if (ids && n > 0) CK(s, cudaMemcpyAsync(ids, s->ids.p, sizeof(unsigned int) * n, cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

lmrs_status lmrs_synchronize(lmrs_scene* s) {
    TRY(check_scene(s));
    CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

const char* lmrs_status_str(lmrs_status st) {
    const int i = (int)st;
    return (i >= 0 && i < (int)(sizeof(kStatusStr) / sizeof(kStatusStr[0]))) ? kStatusStr[i] : "LMRS_ERR_UNKNOWN";
}

const char* lmrs_last_error(const lmrs_scene* s) { return s ? s->err.c_str() : "null scene"; }

int64_t lmrs_launch_count(void) { return lmrs::g_launches.load(std::memory_order_relaxed); }

int32_t lmrs_debug_build(void) {
#ifdef LMRS_DEBUG
    return 1;
#else
    return 0;
#endif
}

lmrs_status lmrs_debug_status(lmrs_scene* s, uint32_t* bits) {
    TRY(check_scene(s));
    if (!bits) return fail(s, LMRS_ERR_INVALID_ARG, "null argument");
    unsigned int* w = &s->sc.as<Scalars>()->debug_err;
    CK(s, cudaMemcpyAsync(bits, w, sizeof(unsigned int), cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaMemsetAsync(w, 0, sizeof(unsigned int), s->st));
    CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

int64_t lmrs_footprint_bytes(const lmrs_config* cfg, int64_t n_gauss, int32_t n_cams, int32_t width, int32_t height,
                             int32_t views_per_step, double tiles_per_pair) {
    if (!cfg || n_gauss <= 0 || n_cams <= 0 || width <= 0 || height <= 0 || cfg->tile_w <= 0 || cfg->tile_h <= 0 ||
        cfg->sh_degree < 0 || cfg->sh_degree > 3)
        return 0;
    const double nv = (views_per_step <= 0 || views_per_step > n_cams) ? n_cams : views_per_step;
    const double tpp = tiles_per_pair > 0.0 ? tiles_per_pair : 10.0;
    const double G = (double)n_gauss;
    const double P = G * (11 + 3 * (cfg->sh_degree + 1) * (cfg->sh_degree + 1));
    const int tx = (width + cfg->tile_w - 1) / cfg->tile_w, ty = (height + cfg->tile_h - 1) / cfg->tile_h;
    double S_view = 0.0, items_view = 0.0;
    int max_items = 1;
    for (int t = 0; t < tx * ty; ++t) {
        const int vw = std::min(cfg->tile_w, width - (t % tx) * cfg->tile_w);
        const int vh = std::min(cfg->tile_h, height - (t / tx) * cfg->tile_h);
        const int k = samples_in_tile(*cfg, vw * vh);
        S_view += k;
        items_view += (k + 31) / 32;
        max_items = std::max(max_items, (k + 31) / 32);
    }
    const double pairs = nv * G, entries = tpp * pairs, S = nv * S_view, items = nv * items_view;
    // rec 96, Jacobian cache, rect 16, row-span ellipse 32, depth keys/values
    // and their alternates 24, counts 8, cotangent slots 48, diagonal slots 64;
    // scan and sort scratch ~2
    const double per_pair = 96 + 16.0 * jac_f4(cfg->sh_degree) + 16 + 32 + 24 + 8 + 48 + 4.0 * kDiagF + 2;
    // ids and the binning's row lists 8 (the emission path: keys, ids and their
    // alternates 16, the bound taken), compact lists 4 per work item of a tile
    const double per_entry = 16 + 4.0 * max_items + 1;
    // offset 1, residual 12, FP32 and BF16 caches 12 + 4 + 6 + 2, stop index 4,
    // importance weight 4, SSIM values 24
    const double per_sample = 41 + (cfg->sample_dist != 0 ? 4 : 0) + (cfg->ssim_weight > 0.0 ? 24 : 0);
    // tile offset, weight, range 16; the binning's counts per (tile, row-list
    // segment) 32 (8 segments); compact lengths 4 per item; work items and
    // their ordering buffers 36
    const double per_view_tile = 48 + 4.0 * max_items;
    const double per_item = 36;
    const double fixed = 9 * 4 * P + 4.0 * kGaussF4 * 4 * G + (double)sizeof(CamDev) * n_cams +
                         sizeof(double) * kMaxPartials + 65536;
    const double var = pairs * per_pair + entries * per_entry + S * per_sample + nv * tx * ty * per_view_tile +
                       items * per_item;
    const double targets = (double)n_cams * height * width * 3 * sizeof(float);
    // full frames of the step's views for the SSIM windows
    const double frames = cfg->ssim_weight > 0.0 ? nv * height * width * 3 * sizeof(float) : 0.0;
    return (int64_t)(fixed + targets + frames + 1.25 * var);
}

lmrs_status lmrs_get_ssim(lmrs_scene* s, float* s_host, float* d_host) {
    TRY(check_scene(s));
    if (!(s->cfg.ssim_weight > 0.0)) return fail(s, LMRS_ERR_INVALID_ARG, "the SSIM term is off");
    TRY(need_render(s));
    if (s_host) CK(s, cudaMemcpyAsync(s_host, s->ssim_s.p, sizeof(float) * 3 * s->S, cudaMemcpyDeviceToHost, s->st));
    if (d_host) CK(s, cudaMemcpyAsync(d_host, s->ssim_d.p, sizeof(float) * 3 * s->S, cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    return LMRS_OK;
}

lmrs_status lmrs_get_sample_weights(lmrs_scene* s, float* w) {
    TRY(check_scene(s));
    TRY(need_pre(s));
    if (!w) return fail(s, LMRS_ERR_INVALID_ARG, "null output");
    if (s->cfg.sample_dist != 0) {
        CK(s, cudaMemcpyAsync(w, s->wsample.p, sizeof(float) * s->S, cudaMemcpyDeviceToHost, s->st));
        CK(s, cudaStreamSynchronize(s->st));
        return LMRS_OK;
    }
    std::vector<float> wt((size_t)s->nv * s->T);
    CK(s, cudaMemcpyAsync(wt.data(), s->wtile.p, sizeof(float) * wt.size(), cudaMemcpyDeviceToHost, s->st));
    CK(s, cudaStreamSynchronize(s->st));
    for (size_t vt = 0; vt < wt.size(); ++vt)
        for (int i = s->tile_off_h[vt]; i < s->tile_off_h[vt + 1]; ++i) w[i] = wt[vt];
    return LMRS_OK;
}

int64_t lmrs_num_evaluations(lmrs_scene* s) {
    if (check_scene(s) != LMRS_OK || !s->rendered) return -1;
    unsigned long long n = 0;
    if (cudaMemcpyAsync(&n, &s->ctx().sc->n_eval, sizeof(n), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int64_t)n;
}

int64_t lmrs_num_walked_entries(lmrs_scene* s) {
    if (check_scene(s) != LMRS_OK || !s->rendered) return -1;
    unsigned long long n = 0;
    if (cudaMemcpyAsync(&n, &s->ctx().sc->n_walk, sizeof(n), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int64_t)n;
}

int64_t lmrs_scene_device_bytes(const lmrs_scene* s) {
    if (!s) return 0;
    int64_t n = 0;
    for (DevBuf* b : const_cast<lmrs_scene*>(s)->bufs()) n += (int64_t)b->cap;
    return n;
}

}  // extern "C"

// ===========================================================================
// Batches
// ===========================================================================
struct lmrs_batch {
    std::vector<lmrs_scene*> scenes;
    int n = 0, deg = 0, iters = 0, nthreads = 1;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    // device tables
    DevBuf ctxs, vecs, gch, vch, wch, counts, hist;
    // host copies (kept alive while the asynchronous uploads are staged)
    std::vector<Ctx> hctx;
    std::vector<BatchVec> hvec;
    std::vector<int4> hg, hv, hw;
    int hcounts[3] = {0, 0, 0};
    // the captured CG loop
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
    void* graph_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> ev_scene;
    cudaEvent_t ev_batch = nullptr;
    std::vector<lmrs_status> scene_rc;  // per scene, of the last step
    // the launch form: one persistent cooperative launch of every phase (the
    // default), or the graph of per-phase launches
    bool persistent = true;
    DevBuf bar;  // its grid barrier's words
};

namespace {

constexpr int kBatchGrid = 1216;  // blocks of the batched launches (8 per SM), grid-stride over chunks
constexpr double kBarrierTimeoutS = 2.0;  // a grid barrier of the persistent PCG waits at most this long

lmrs_status bfail(lmrs_batch* b, lmrs_status code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

void add_chunks(std::vector<int4>& out, int scene, long long n, int step) {
    for (long long b0 = 0; b0 < n; b0 += step) out.push_back(make_int4(scene, (int)b0, (int)std::min(n, b0 + step), 0));
}

// Per-step setup of scene i: everything of its LM step before the PCG loop.
lmrs_status scene_setup(lmrs_scene* s, const int32_t* views, int nv, long long step) {
    TRY(lmrs_preprocess(s, views, nv, step));
    TRY(lmrs_render(s, nullptr, nullptr));
    TimerScope ts_(s);
    TRY(do_rhs_diag(s, s->b.as<float>()));
    return LMRS_OK;
}

lmrs_status batch_tables(lmrs_batch* B, const int64_t* steps) {
    B->hctx.resize(B->n);
    B->hvec.resize(B->n);
    B->hg.clear();
    B->hv.clear();
    B->hw.clear();
    double* hist = B->hist.as<double>();
    for (int i = 0; i < B->n; ++i) {
        lmrs_scene* s = B->scenes[i];
        if (s->P >= (1ll << 31)) return bfail(B, LMRS_ERR_BUDGET, "scene too large for a batch");
        B->hctx[i] = s->ctx();
        BatchVec& v = B->hvec[i];
        v.b = s->b.as<float>();
        v.x = s->x.as<float>();
        v.r = s->r.as<float>();
        v.z = s->z.as<float>();
        v.p = s->p.as<float>();
        v.Ap = s->Ap.as<float>();
        v.minv = s->minv.as<float>();
        v.D = s->D.as<float>();
        v.params = s->params.as<float>();
        v.rz = hist + (size_t)i * 2 * (kMaxBatchIters + 1);
        v.pAp = v.rz + kMaxBatchIters + 1;
        v.P = s->P;
        v.lm_step = steps[i];
        v.lr_warm = s->cfg.lr_warm;
        v.lr_cap = s->cfg.lr_cap;
        v.color_bound = s->cfg.color_bound;
        v.warm_iters = s->cfg.warm_iters;
        add_chunks(B->hg, i, s->G, kBatchBlock);
        add_chunks(B->hv, i, s->P, kVecChunk);
        add_chunks(B->hw, i, s->nwork, kBatchBlock / kWarp);
    }
    B->hcounts[0] = (int)B->hg.size();
    B->hcounts[1] = (int)B->hv.size();
    B->hcounts[2] = (int)B->hw.size();
    cudaError_t ea = ensure_on(B->gch, sizeof(int4) * B->hg.size(), B->st);
    if (ea == cudaSuccess) ea = ensure_on(B->vch, sizeof(int4) * B->hv.size(), B->st);
    if (ea == cudaSuccess) ea = ensure_on(B->wch, sizeof(int4) * std::max<size_t>(B->hw.size(), 1), B->st);
    if (ea != cudaSuccess) {
        cudaGetLastError();
        return bfail(B, ea == cudaErrorMemoryAllocation ? LMRS_ERR_OOM : LMRS_ERR_CUDA, "batch tables");
    }
    auto up = [&](DevBuf& d, const void* h, size_t bytes) {
        return bytes ? cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, B->st) : cudaSuccess;
    };
    cudaError_t e = up(B->ctxs, B->hctx.data(), sizeof(Ctx) * B->n);
    if (e == cudaSuccess) e = up(B->vecs, B->hvec.data(), sizeof(BatchVec) * B->n);
    if (e == cudaSuccess) e = up(B->gch, B->hg.data(), sizeof(int4) * B->hg.size());
    if (e == cudaSuccess) e = up(B->vch, B->hv.data(), sizeof(int4) * B->hv.size());
    if (e == cudaSuccess) e = up(B->wch, B->hw.data(), sizeof(int4) * B->hw.size());
    if (e == cudaSuccess) e = up(B->counts, B->hcounts, sizeof(B->hcounts));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(B->hist.p, 0, sizeof(double) * (size_t)B->n * 2 * (kMaxBatchIters + 1), B->st);
    if (e != cudaSuccess) return bfail(B, LMRS_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    return LMRS_OK;
}

BatchTables batch_view(const lmrs_batch* B) {
    BatchTables t;
    t.ctxs = B->ctxs.as<Ctx>();
    t.vecs = B->vecs.as<BatchVec>();
    t.gchunks = B->gch.as<int4>();
    t.vchunks = B->vch.as<int4>();
    t.wchunks = B->wch.as<int4>();
    t.counts = B->counts.as<int>();
    return t;
}

// Capture the PCG loop and the updates of all scenes as one graph (again
// whenever a table buffer moved).
lmrs_status batch_graph(lmrs_batch* B) {
    void* key[5] = {B->ctxs.p, B->vecs.p, B->gch.p, B->vch.p, B->wch.p};
    if (B->exec && std::equal(key, key + 5, B->graph_key)) return LMRS_OK;
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    LaunchTimer* saved = t_active;
    t_active = nullptr;  // no event records inside the captured graph
    const long long before = lmrs_launch_count();
    cudaError_t e = cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const BatchTables t = batch_view(B);
        launch_b_precond_init(t, kBatchGrid, B->st);
        for (int it = 0; it < B->iters; ++it) {
            launch_b_direction(t, it, kBatchGrid, B->st);
            launch_b_prep_jvp(t, B->deg, kBatchGrid, B->st);
            launch_b_jtj(t, kBatchGrid, B->st);
            launch_b_prep_vjp(t, B->deg, it, kBatchGrid, B->st);
            launch_b_update(t, it, kBatchGrid, B->st);
        }
        launch_b_lm_update(t, B->iters, kBatchGrid, B->st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(B->st, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    t_active = saved;
    // captured launches run at every replay, not now
    B->graph_kernels = lmrs_launch_count() - before;
    g_launches.fetch_sub(B->graph_kernels, std::memory_order_relaxed);
    if (e != cudaSuccess) {
        cudaGetLastError();
        B->exec = nullptr;
        return bfail(B, LMRS_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    std::copy(key, key + 5, B->graph_key);
    return LMRS_OK;
}

}  // namespace

extern "C" {

lmrs_status lmrs_batch_create(lmrs_scene* const* scenes, int32_t n_scenes, int32_t n_threads, void* cuda_stream,
                              lmrs_batch** out) {
    if (!out) return LMRS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!scenes || n_scenes <= 0) return LMRS_ERR_INVALID_ARG;
    for (int i = 0; i < n_scenes; ++i) {
        if (!scenes[i]) return LMRS_ERR_INVALID_ARG;
        if (scenes[i]->deg != scenes[0]->deg || scenes[i]->cfg.cg_iters != scenes[0]->cfg.cg_iters)
            return LMRS_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (scenes[j] == scenes[i]) return LMRS_ERR_INVALID_ARG;
    }
    if (scenes[0]->cfg.cg_iters > kMaxBatchIters) return LMRS_ERR_BUDGET;
    lmrs_batch* B = new lmrs_batch();
    B->scenes.assign(scenes, scenes + n_scenes);
    B->n = n_scenes;
    B->deg = scenes[0]->deg;
    B->iters = scenes[0]->cfg.cg_iters;
    B->nthreads = std::max(1, std::min<int>(n_threads, n_scenes));
    lmrs_status rc = LMRS_OK;
    if (cuda_stream) {
        B->st = static_cast<cudaStream_t>(cuda_stream);
    } else if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess) {
        rc = LMRS_ERR_CUDA;
    } else {
        B->own_stream = true;
    }
    if (rc == LMRS_OK && ensure_on(B->ctxs, sizeof(Ctx) * n_scenes, B->st) != cudaSuccess) rc = LMRS_ERR_OOM;
    if (rc == LMRS_OK && ensure_on(B->vecs, sizeof(BatchVec) * n_scenes, B->st) != cudaSuccess) rc = LMRS_ERR_OOM;
    if (rc == LMRS_OK && ensure_on(B->counts, sizeof(int) * 3, B->st) != cudaSuccess) rc = LMRS_ERR_OOM;
    if (rc == LMRS_OK && ensure_on(B->hist, sizeof(double) * n_scenes * 2 * (kMaxBatchIters + 1), B->st) != cudaSuccess) rc = LMRS_ERR_OOM;
    B->ev_scene.assign(n_scenes, nullptr);
    for (int i = 0; rc == LMRS_OK && i < n_scenes; ++i)
        if (cudaEventCreateWithFlags(&B->ev_scene[i], cudaEventDisableTiming) != cudaSuccess) rc = LMRS_ERR_CUDA;
    if (rc == LMRS_OK && cudaEventCreateWithFlags(&B->ev_batch, cudaEventDisableTiming) != cudaSuccess)
        rc = LMRS_ERR_CUDA;
    if (rc != LMRS_OK) {
        cudaGetLastError();
        lmrs_batch_destroy(B);
        return rc;
    }
    *out = B;
    return LMRS_OK;
}

lmrs_status lmrs_batch_destroy(lmrs_batch* B) {
    if (!B) return LMRS_ERR_INVALID_ARG;
    if (B->st) cudaStreamSynchronize(B->st);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    for (auto e : B->ev_scene)
        if (e) cudaEventDestroy(e);
    if (B->ev_batch) cudaEventDestroy(B->ev_batch);
    for (DevBuf* d : {&B->ctxs, &B->vecs, &B->gch, &B->vch, &B->wch, &B->counts, &B->hist, &B->bar})
        release(*d, B->st);
    if (B->st) cudaStreamSynchronize(B->st);
    if (B->own_stream) cudaStreamDestroy(B->st);
    trim_pool();
    delete B;
    return LMRS_OK;
}

lmrs_status lmrs_batch_lm_step(lmrs_batch* B, const int32_t* view_ids, const int32_t* n_views, const int64_t* lm_steps,
                               lmrs_step_stats* stats) {
    if (!B) return LMRS_ERR_INVALID_ARG;
    if (!view_ids || !n_views || !lm_steps) return bfail(B, LMRS_ERR_INVALID_ARG, "null argument");
    NvtxRange step_("lmrs_batch_lm_step");
    B->scene_rc.assign(B->n, LMRS_ERR_NOT_PREPROCESSED);  // "not stepped" until the graph ran
    std::vector<long long> voff(B->n + 1, 0);
    for (int i = 0; i < B->n; ++i) {
        if (n_views[i] <= 0) return bfail(B, LMRS_ERR_INVALID_ARG, "scene without views");
        voff[i + 1] = voff[i] + n_views[i];
    }
    // 1. per-scene setup, n threads at a time, each scene on its own stream
    std::vector<lmrs_status> rc(B->n, LMRS_OK);
    auto work = [&](int w) {
        for (int i = w; i < B->n; i += B->nthreads) {
            lmrs_scene* s = B->scenes[i];
            rc[i] = scene_setup(s, view_ids + voff[i], n_views[i], lm_steps[i]);
            if (rc[i] == LMRS_OK && cudaEventRecord(B->ev_scene[i], s->st) != cudaSuccess) rc[i] = LMRS_ERR_CUDA;
        }
    };
    if (B->nthreads == 1) {
        work(0);
    } else {
        std::vector<std::thread> pool;
        for (int w = 0; w < B->nthreads; ++w) pool.emplace_back(work, w);
        for (auto& th : pool) th.join();
    }
    lmrs_status first = LMRS_OK;
    int first_i = -1;
    for (int i = 0; i < B->n; ++i)
        if (rc[i] != LMRS_OK) {
            B->scene_rc[i] = rc[i];
            if (first_i < 0) {
                first = rc[i];
                first_i = i;
            }
        }
    if (first_i >= 0) return bfail(B, first, "scene " + std::to_string(first_i) + ": " + B->scenes[first_i]->err);
    // 2. tables, then the batched PCG loop and updates (one graph)
    for (int i = 0; i < B->n; ++i)
        if (cudaStreamWaitEvent(B->st, B->ev_scene[i], 0) != cudaSuccess)
            return bfail(B, LMRS_ERR_CUDA, "stream wait");
    TRY(batch_tables(B, lm_steps));
    if (B->persistent) {
        if (ensure_on(B->bar, grid_bar_bytes(), B->st) != cudaSuccess) return bfail(B, LMRS_ERR_OOM, "barrier words");
        const cudaError_t e = launch_b_pcg(batch_view(B), B->deg, B->iters, B->bar.p, kBarrierTimeoutS, B->st);
        if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
            // the device cannot hold the whole grid at once: from here on the
            // batch uses the graph of per-phase launches
            cudaGetLastError();
            B->persistent = false;
        } else if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(B, LMRS_ERR_CUDA, std::string("persistent PCG launch: ") + cudaGetErrorString(e));
        }
    }
    if (!B->persistent) {
        TRY(batch_graph(B));
        cudaError_t e = cudaGraphLaunch(B->exec, B->st);
        if (e != cudaSuccess) return bfail(B, LMRS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        g_launches.fetch_add(B->graph_kernels, std::memory_order_relaxed);
    }
    // 3. the scenes' next work waits for the batch
    if (cudaEventRecord(B->ev_batch, B->st) != cudaSuccess) return bfail(B, LMRS_ERR_CUDA, "event record");
    for (lmrs_scene* s : B->scenes) {
        if (cudaStreamWaitEvent(s->st, B->ev_batch, 0) != cudaSuccess) return bfail(B, LMRS_ERR_CUDA, "stream wait");
        s->preprocessed = s->rendered = s->have_D = s->ordered = false;
    }
    std::fill(B->scene_rc.begin(), B->scene_rc.end(), LMRS_OK);
    if (!stats) return LMRS_OK;
    if (cudaStreamSynchronize(B->st) != cudaSuccess) return bfail(B, LMRS_ERR_CUDA, "synchronise");
    if (B->persistent) {
        unsigned char hb[64] = {};
        if (cudaMemcpy(hb, B->bar.p, grid_bar_bytes(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bfail(B, LMRS_ERR_CUDA, "read barrier words");
        if (grid_bar_error(hb)) {
            for (auto& r : B->scene_rc) r = LMRS_ERR_TIMEOUT;
            return bfail(B, LMRS_ERR_TIMEOUT, "a grid barrier of the persistent PCG timed out");
        }
    }
    std::vector<double> hist((size_t)B->n * 2 * (kMaxBatchIters + 1));
    if (cudaMemcpy(hist.data(), B->hist.p, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return bfail(B, LMRS_ERR_CUDA, "read history");
    lmrs_status out = LMRS_OK;
    for (int i = 0; i < B->n; ++i) {
        lmrs_scene* s = B->scenes[i];
        Scalars h;
        if (cudaMemcpy(&h, s->sc.p, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bfail(B, LMRS_ERR_CUDA, "read scalars");
        float m;
        std::memcpy(&m, &h.max_dc_bits, sizeof(m));
        const double* rz = hist.data() + (size_t)i * 2 * (kMaxBatchIters + 1);
        stats[i].loss = h.loss_den > 0.0 ? h.loss_num / h.loss_den : 0.0;
        stats[i].eta = h.eta;
        stats[i].max_dc = m;
        stats[i].rz0 = rz[0];
        stats[i].rz_final = rz[B->iters];
        stats[i].n_samples = s->S;
        stats[i].n_pairs = s->npairs >= 0 ? s->npairs : (int64_t)h.n_list;
        if (h.numeric_error) {
            B->scene_rc[i] = LMRS_ERR_NUMERIC;
            if (out == LMRS_OK) out = bfail(B, LMRS_ERR_NUMERIC, "scene " + std::to_string(i));
        }
    }
    return out;
}

const char* lmrs_batch_last_error(const lmrs_batch* B) { return B ? B->err.c_str() : "null batch"; }

lmrs_status lmrs_batch_set_persistent(lmrs_batch* B, int32_t on) {
    if (!B || (on != 0 && on != 1)) return LMRS_ERR_INVALID_ARG;
    B->persistent = on == 1;
    return LMRS_OK;
}

lmrs_status lmrs_batch_scene_status(const lmrs_batch* B, int32_t i) {
    if (!B || i < 0 || i >= B->n) return LMRS_ERR_INVALID_ARG;
    return i < (int)B->scene_rc.size() ? B->scene_rc[i] : LMRS_ERR_NOT_PREPROCESSED;
}

}  // extern "C"
