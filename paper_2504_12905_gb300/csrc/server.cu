// Fit-job server: FIFO admission against a device-memory budget and
// continuous batching of the resident jobs' LM steps (Alg. 1, one step of
// every resident job per scheduler iteration through lmrs_batch_lm_step).
// Host code over the public C-ABI plus the library's memory pool.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    lmrs_config cfg;
    int64_t G = 0, P = 0;
    std::vector<float> params;   // host copy (the result once done)
    std::vector<lmrs_camera> cams;
    std::vector<float> targets;  // host copy, released at admission
    int32_t views_per_step = 0;
    double target_loss = 0.0;
    int32_t max_steps = 0;
    // device state while resident
    cudaStream_t st = nullptr;
    float* targets_dev = nullptr;
    size_t targets_bytes = 0;
    lmrs_scene* scene = nullptr;
    lmrs_job_info info;
};

}  // namespace

struct lmrs_server {
    lmrs_server_config cfg;
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Job*> queue;
    std::vector<Job*> active;  // scheduler thread only (read under mu for stats)
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    int64_t next_id = 1;
    int64_t finished = 0, iterations = 0, bytes_in_use = 0, bytes_peak = 0;
    std::thread thread;
    // batches of the current resident set, per (SH degree, cg_iters) group
    struct Group {
        std::vector<Job*> members;  // batched members first (n_batched of them), then the solo ones
        size_t n_batched = 0;
        lmrs_batch* batch = nullptr;
    };
    std::vector<Group> groups;
    bool groups_dirty = true;
};

namespace {

double secs(const lmrs_server* S) {
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

int64_t held_bytes(const Job* j) {
    return (j->scene ? lmrs_scene_device_bytes(j->scene) : 0) + (int64_t)j->targets_bytes;
}

void views_of_step(const Job* j, int64_t step, std::vector<int32_t>& out) {
    lmrs::uniform_views((int)j->cams.size(), j->views_per_step, j->cfg.seed, step, out);
}

// Device side of an admitted job; on failure the job is marked failed.
lmrs_status bring_up(Job* j) {
    if (cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking) != cudaSuccess) return LMRS_ERR_CUDA;
    j->targets_bytes = j->targets.size() * sizeof(float);
    void* t = nullptr;
    cudaError_t e = lmrs::pool_alloc(&t, j->targets_bytes, j->st);
    if (e == cudaSuccess) {
        j->targets_dev = static_cast<float*>(t);
        e = cudaMemcpyAsync(t, j->targets.data(), j->targets_bytes, cudaMemcpyHostToDevice, j->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(j->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LMRS_ERR_OOM : LMRS_ERR_CUDA;
    }
    std::vector<float>().swap(j->targets);  // the device copy is the one used from here on
    return lmrs_scene_create(&j->cfg, j->G, j->params.data(), j->cams.data(), (int32_t)j->cams.size(), j->targets_dev,
                             j->st, &j->scene);
}

void tear_down(Job* j) {
    if (j->scene) {
        lmrs_scene_destroy(j->scene);
        j->scene = nullptr;
    }
    if (j->targets_dev) {
        lmrs::pool_free(j->targets_dev, j->st);
        j->targets_dev = nullptr;
    }
    if (j->st) {
        cudaStreamSynchronize(j->st);
        cudaStreamDestroy(j->st);
        j->st = nullptr;
    }
    j->targets_bytes = 0;
}

void finish(lmrs_server* S, Job* j, lmrs_status status, bool converged) {
    if (status == LMRS_OK && j->scene) {
        if (lmrs_get_params(j->scene, j->params.data()) != LMRS_OK) status = LMRS_ERR_CUDA;
    }
    tear_down(j);
    std::lock_guard<std::mutex> lk(S->mu);
    j->info.state = status == LMRS_OK ? LMRS_JOB_DONE : LMRS_JOB_FAILED;
    j->info.status = status;
    j->info.converged = converged ? 1 : 0;
    j->info.t_done = secs(S);
    ++S->finished;
    S->cv_done.notify_all();
}

int64_t samples_per_step(const Job* j) {
    const int views = j->views_per_step > 0 ? std::min<int>(j->views_per_step, (int)j->cams.size()) : (int)j->cams.size();
    const double px = (double)j->cams[0].width * j->cams[0].height;
    const double frac = j->cfg.samples_per_tile > 0
                            ? std::min(1.0, (double)j->cfg.samples_per_tile / (j->cfg.tile_w * j->cfg.tile_h))
                            : std::min(1.0, j->cfg.sample_frac);
    return (int64_t)(px * frac * views);
}

double work_estimate(const Job* j) {
    const int views = j->views_per_step > 0 ? std::min<int>(j->views_per_step, (int)j->cams.size()) : (int)j->cams.size();
    return (double)j->G * views * j->max_steps;
}

// Admits queued jobs (policy order) while the budget and the slot count allow.
void admit(lmrs_server* S) {
    for (;;) {
        Job* j = nullptr;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->queue.empty() || (int)S->active.size() >= S->cfg.max_active) return;
            int64_t used = 0;
            for (const Job* a : S->active) used += std::max<int64_t>(a->info.footprint_est, held_bytes(a));
            auto pick = S->queue.begin();
            if (S->cfg.policy == 1) {
                // least estimated work (Gaussians x views per step x max_steps); the
                // queue is in arrival order, so ties go to the oldest
                pick = std::min_element(S->queue.begin(), S->queue.end(), [](const Job* a, const Job* b) {
                    return work_estimate(a) < work_estimate(b);
                });
            }
            Job* head = *pick;
            if (!S->active.empty() && used + head->info.footprint_est > S->cfg.budget_bytes) return;
            S->queue.erase(pick);
            j = head;
        }
        const lmrs_status rc = bring_up(j);
        if (rc != LMRS_OK) {
            finish(S, j, rc, false);
            continue;
        }
        std::lock_guard<std::mutex> lk(S->mu);
        j->info.state = LMRS_JOB_RUNNING;
        j->info.t_admit = secs(S);
        S->active.push_back(j);
        S->groups_dirty = true;
    }
}

void rebuild_groups(lmrs_server* S) {
    for (auto& g : S->groups)
        if (g.batch) lmrs_batch_destroy(g.batch);
    S->groups.clear();
    for (Job* j : S->active) {
        auto it = std::find_if(S->groups.begin(), S->groups.end(), [&](const lmrs_server::Group& g) {
            return g.members[0]->cfg.sh_degree == j->cfg.sh_degree && g.members[0]->cfg.cg_iters == j->cfg.cg_iters;
        });
        if (it == S->groups.end()) {
            S->groups.push_back({});
            it = S->groups.end() - 1;
        }
        it->members.push_back(j);
    }
    for (auto& g : S->groups) {
        // small jobs batched (they do not fill the device alone), large ones solo
        std::stable_partition(g.members.begin(), g.members.end(),
                              [&](const Job* j) { return samples_per_step(j) < S->cfg.solo_min_samples; });
        g.n_batched = (size_t)std::count_if(g.members.begin(), g.members.end(), [&](const Job* j) {
            return samples_per_step(j) < S->cfg.solo_min_samples;
        });
        if (g.n_batched < 2) g.n_batched = 0;  // one small job steps on its own
        std::vector<lmrs_scene*> sc;
        for (size_t i = 0; i < g.n_batched; ++i) sc.push_back(g.members[i]->scene);
        if (!sc.empty() &&
            lmrs_batch_create(sc.data(), (int32_t)sc.size(), S->cfg.setup_threads, nullptr, &g.batch) != LMRS_OK)
            g.batch = nullptr;
    }
    S->groups_dirty = false;
}

// Outcome of one step of one job.
struct StepOut {
    lmrs_status rc = LMRS_OK;
    lmrs_step_stats st{};
    bool reached = false;
    double full = -1.0;
};

// Whether the job reached its target after the step (the sampled loss, or
// the full-frame MSE once the sampled loss is within the gate).
void check_target(const lmrs_server* S, Job* j, StepOut& o) {
    if (o.rc != LMRS_OK) return;
    o.reached = o.st.loss <= j->target_loss;
    if (S->cfg.stop_full_frame) {
        o.reached = false;
        if (o.st.loss <= S->cfg.full_frame_gate * j->target_loss && lmrs_eval_mse(j->scene, &o.full) == LMRS_OK)
            o.reached = o.full <= j->target_loss;
    }
}

// One LM step of every member of the group and its target check: the
// batched members through the group's batch (a member the batch did not step
// steps alone), the solo members concurrently, each on its own stream from a
// host thread.
void step_group(lmrs_server* S, lmrs_server::Group& g, std::vector<StepOut>& out) {
    const size_t n = g.members.size();
    out.assign(n, StepOut{});
    std::vector<std::vector<int32_t>> views(n);
    for (size_t i = 0; i < n; ++i) views_of_step(g.members[i], g.members[i]->info.steps, views[i]);
    std::vector<size_t> alone;  // members stepped one by one
    if (g.n_batched > 0 && g.batch) {
        std::vector<int32_t> flat, nv(g.n_batched);
        std::vector<int64_t> steps(g.n_batched);
        std::vector<lmrs_step_stats> st(g.n_batched);
        for (size_t i = 0; i < g.n_batched; ++i) {
            flat.insert(flat.end(), views[i].begin(), views[i].end());
            nv[i] = (int32_t)views[i].size();
            steps[i] = g.members[i]->info.steps;
        }
        const bool ok = lmrs_batch_lm_step(g.batch, flat.data(), nv.data(), steps.data(), st.data()) == LMRS_OK;
        for (size_t i = 0; i < g.n_batched; ++i) {
            out[i].st = st[i];
            out[i].rc = ok ? LMRS_OK : lmrs_batch_scene_status(g.batch, (int32_t)i);
            if (out[i].rc == LMRS_ERR_NOT_PREPROCESSED) alone.push_back(i);  // not stepped: alone below
            else check_target(S, g.members[i], out[i]);
        }
    } else {
        for (size_t i = 0; i < g.n_batched; ++i) alone.push_back(i);
    }
    for (size_t i = g.n_batched; i < n; ++i) alone.push_back(i);
    std::atomic<size_t> next{0};
    auto work = [&] {
        cudaSetDevice(S->device);
        for (size_t k = next++; k < alone.size(); k = next++) {
            const size_t i = alone[k];
            Job* j = g.members[i];
            out[i].rc = lmrs_lm_step(j->scene, views[i].data(), (int32_t)views[i].size(), j->info.steps, &out[i].st);
            check_target(S, j, out[i]);
        }
    };
    const size_t nt = std::min<size_t>(alone.size(), (size_t)S->cfg.setup_threads);
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
    if (nt > 0) work();
    for (auto& t : pool) t.join();
}

void scheduler(lmrs_server* S) {
    cudaSetDevice(S->device);
    std::vector<StepOut> out;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop) break;
        }
        admit(S);
        if (S->active.empty()) continue;
        if (S->groups_dirty) rebuild_groups(S);
        std::vector<Job*> retire;
        std::vector<std::pair<Job*, lmrs_status>> failed;
        std::vector<bool> conv;
        for (auto& g : S->groups) {
            step_group(S, g, out);
            for (size_t i = 0; i < g.members.size(); ++i) {
                Job* j = g.members[i];
                if (out[i].rc != LMRS_OK) {
                    failed.push_back({j, out[i].rc});
                    continue;
                }
                const int64_t held = held_bytes(j);
                std::lock_guard<std::mutex> lk(S->mu);
                j->info.steps += 1;
                j->info.loss = out[i].st.loss;
                if (out[i].full >= 0.0) j->info.full_mse = out[i].full;
                j->info.footprint_peak = std::max(j->info.footprint_peak, held);
                if (out[i].reached || j->info.steps >= j->max_steps) {
                    retire.push_back(j);
                    conv.push_back(out[i].reached);
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            ++S->iterations;
            int64_t in_use = 0;
            for (const Job* a : S->active) in_use += held_bytes(a);
            S->bytes_in_use = in_use;
            S->bytes_peak = std::max(S->bytes_peak, in_use);
        }
        if (retire.empty() && failed.empty()) continue;
        for (auto& g : S->groups)
            if (g.batch) {
                lmrs_batch_destroy(g.batch);
                g.batch = nullptr;
            }
        S->groups_dirty = true;
        auto drop = [&](Job* j) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->active.erase(std::remove(S->active.begin(), S->active.end(), j), S->active.end());
        };
        for (size_t i = 0; i < retire.size(); ++i) {
            drop(retire[i]);
            finish(S, retire[i], LMRS_OK, conv[i]);
        }
        for (auto& f : failed) {
            drop(f.first);
            finish(S, f.first, f.second, false);
        }
    }
    // shutdown: release what is resident or queued
    for (auto& g : S->groups)
        if (g.batch) lmrs_batch_destroy(g.batch);
    S->groups.clear();
    std::vector<Job*> left;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        left = S->active;
        left.insert(left.end(), S->queue.begin(), S->queue.end());
        S->active.clear();
        S->queue.clear();
    }
    for (Job* j : left) finish(S, j, LMRS_ERR_TIMEOUT, false);
}

Job* find_job(lmrs_server* S, int64_t id) {
    auto it = S->jobs.find(id);
    return it == S->jobs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

lmrs_status lmrs_server_create(const lmrs_server_config* cfg, lmrs_server** out) {
    if (!cfg || !out || cfg->budget_bytes <= 0 || cfg->max_active < 1 || cfg->max_active > 1024 ||
        cfg->setup_threads < 1 || cfg->policy < 0 || cfg->policy > 1 || cfg->stop_full_frame < 0 ||
        cfg->stop_full_frame > 1)
        return LMRS_ERR_INVALID_ARG;
    lmrs_server* S = new lmrs_server();
    S->cfg = *cfg;
    if (!(S->cfg.tiles_per_pair > 0.0)) S->cfg.tiles_per_pair = 10.0;
    if (!(S->cfg.full_frame_gate > 0.0)) S->cfg.full_frame_gate = 1.25;
    if (S->cfg.solo_min_samples <= 0) S->cfg.solo_min_samples = 131072;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return LMRS_ERR_CUDA;
    }
    S->t0 = Clock::now();
    S->thread = std::thread(scheduler, S);
    *out = S;
    return LMRS_OK;
}

lmrs_status lmrs_server_submit(lmrs_server* S, const lmrs_config* cfg, int64_t n_gauss, const float* params_host,
                               const lmrs_camera* cams_host, int32_t n_cams, const float* targets_host,
                               int32_t views_per_step, double target_loss, int32_t max_steps, int64_t* job_id) {
    if (!S || !cfg || !params_host || !cams_host || !targets_host || !job_id || n_gauss <= 0 || n_cams <= 0 ||
        max_steps <= 0 || cfg->sh_degree < 0 || cfg->sh_degree > 3 || cfg->tile_w <= 0 || cfg->tile_h <= 0 ||
        cfg->tile_w * cfg->tile_h > 256 || cfg->cg_iters < 0 || cfg->cg_iters > lmrs::kMaxBatchIters)
        return LMRS_ERR_INVALID_ARG;
    for (int i = 0; i < n_cams; ++i)
        if (cams_host[i].width != cams_host[0].width || cams_host[i].height != cams_host[0].height ||
            cams_host[i].width <= 0 || cams_host[i].height <= 0)
            return LMRS_ERR_INVALID_ARG;
    auto j = std::make_unique<Job>();
    j->cfg = *cfg;
    j->G = n_gauss;
    j->P = n_gauss * (11 + 3 * (cfg->sh_degree + 1) * (cfg->sh_degree + 1));
    j->params.assign(params_host, params_host + j->P);
    j->cams.assign(cams_host, cams_host + n_cams);
    const size_t nt = (size_t)n_cams * cams_host[0].height * cams_host[0].width * 3;
    j->targets.assign(targets_host, targets_host + nt);
    j->views_per_step = views_per_step;
    j->target_loss = target_loss;
    j->max_steps = max_steps;
    std::memset(&j->info, 0, sizeof(j->info));
    j->info.state = LMRS_JOB_QUEUED;
    j->info.t_admit = -1.0;
    j->info.t_done = -1.0;
    j->info.full_mse = -1.0;
    j->info.footprint_est = lmrs_footprint_bytes(cfg, n_gauss, n_cams, cams_host[0].width, cams_host[0].height,
                                                 views_per_step, S->cfg.tiles_per_pair);
    if (j->info.footprint_est > S->cfg.budget_bytes) return LMRS_ERR_BUDGET;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return LMRS_ERR_INVALID_ARG;
    j->id = S->next_id++;
    j->info.t_submit = secs(S);
    *job_id = j->id;
    S->queue.push_back(j.get());
    S->jobs[j->id] = std::move(j);
    S->cv_work.notify_all();
    return LMRS_OK;
}

lmrs_status lmrs_server_poll(lmrs_server* S, int64_t id, lmrs_job_info* info) {
    if (!S || !info) return LMRS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Job* j = find_job(S, id);
    if (!j) return LMRS_ERR_INVALID_ARG;
    *info = j->info;
    return LMRS_OK;
}

lmrs_status lmrs_server_wait(lmrs_server* S, int64_t id, double timeout_s, lmrs_job_info* info) {
    if (!S) return LMRS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    Job* j = find_job(S, id);
    if (!j) return LMRS_ERR_INVALID_ARG;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)), [&] {
        return j->info.state == LMRS_JOB_DONE || j->info.state == LMRS_JOB_FAILED;
    });
    if (info) *info = j->info;
    return ok ? LMRS_OK : LMRS_ERR_TIMEOUT;
}

lmrs_status lmrs_server_result(lmrs_server* S, int64_t id, float* params_host) {
    if (!S || !params_host) return LMRS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Job* j = find_job(S, id);
    if (!j) return LMRS_ERR_INVALID_ARG;
    if (j->info.state != LMRS_JOB_DONE) return LMRS_ERR_NOT_PREPROCESSED;
    std::memcpy(params_host, j->params.data(), sizeof(float) * j->params.size());
    return LMRS_OK;
}

lmrs_status lmrs_server_forget(lmrs_server* S, int64_t id) {
    if (!S) return LMRS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Job* j = find_job(S, id);
    if (!j || (j->info.state != LMRS_JOB_DONE && j->info.state != LMRS_JOB_FAILED)) return LMRS_ERR_INVALID_ARG;
    S->jobs.erase(id);
    return LMRS_OK;
}

lmrs_status lmrs_server_get_stats(lmrs_server* S, lmrs_server_stats* out) {
    if (!S || !out) return LMRS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int32_t)S->queue.size();
    out->active = (int32_t)S->active.size();
    out->finished = S->finished;
    out->bytes_in_use = S->bytes_in_use;
    out->bytes_peak = S->bytes_peak;
    out->iterations = S->iterations;
    return LMRS_OK;
}

lmrs_status lmrs_server_destroy(lmrs_server* S) {
    if (!S) return LMRS_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->thread.joinable()) S->thread.join();
    delete S;
    lmrs::pool_trim();
    return LMRS_OK;
}

}  // extern "C"
