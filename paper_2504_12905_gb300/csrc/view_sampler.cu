// View sampling for the LM steps (Sec. 4.3), host code.
//
// Uniform mode: the views of step k are a partial Fisher-Yates draw of
// n_views camera indices, driven by SplitMix64 seeded from (seed, k).
//
// K-means mode (Sec. 4.3): every camera gets the feature
//   f_i = [normalised position (3), viewing direction (3)],
// positions centred on their mean and scaled by the largest distance from
// it (so they lie in the unit ball), the direction being the camera's +z
// axis in world space.  Lloyd's algorithm partitions the cameras into as
// many clusters as views per step (k-means++ initialisation from
// SplitMix64; ties go to the lower index; an emptied cluster keeps its
// centre; at most 100 iterations or until no assignment changes), and each
// step takes one camera uniformly from every cluster.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace lmrs {

uint64_t sm64_next(uint64_t& state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform draw in [0, 1) with 53 random bits.
static double sm64_unit(uint64_t& state) { return (double)(sm64_next(state) >> 11) * (1.0 / 9007199254740992.0); }

// Generator state of (seed, step, stream): every draw of a step has its own
// sequence.
static uint64_t step_state(uint64_t seed, int64_t step, uint64_t stream) {
    uint64_t s = seed;
    const uint64_t a = sm64_next(s);
    uint64_t t = a ^ (0xD1B54A32D192ED03ull * (uint64_t)(step + 1));
    const uint64_t b = sm64_next(t);
    uint64_t u = b ^ (0x8CB92BA72F3D8DD7ull * (stream + 1));
    return sm64_next(u);
}

void uniform_views(int n_cams, int n_views, uint64_t seed, int64_t step, std::vector<int32_t>& out) {
    const int k = (n_views <= 0 || n_views >= n_cams) ? n_cams : n_views;
    std::vector<int32_t> perm(n_cams);
    for (int i = 0; i < n_cams; ++i) perm[i] = i;
    uint64_t st = step_state(seed, step, 0);
    for (int i = 0; i < k && k < n_cams; ++i) {
        const int r = i + (int)std::floor(sm64_unit(st) * (double)(n_cams - i));
        std::swap(perm[i], perm[r]);
    }
    out.assign(perm.begin(), perm.begin() + k);
    std::sort(out.begin(), out.end());
}

}  // namespace lmrs

struct lmrs_view_sampler {
    int n = 0, k = 0;
    uint64_t seed = 0;
    std::vector<int32_t> label;
    std::vector<std::vector<int32_t>> members;
    int iterations = 0;
};

namespace {

void camera_features(const lmrs_camera* cams, int n, std::vector<double>& f) {
    f.assign((size_t)n * 6, 0.0);
    std::vector<double> pos((size_t)n * 3);
    double mean[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        const float* w = cams[i].world_to_cam;  // row-major [R | t]
        for (int a = 0; a < 3; ++a) {
            // centre = -R^T t
            double c = 0.0;
            for (int r = 0; r < 3; ++r) c -= (double)w[4 * r + a] * (double)w[4 * r + 3];
            pos[3 * i + a] = c;
            mean[a] += c;
        }
    }
    for (int a = 0; a < 3; ++a) mean[a] /= n;
    double rmax = 0.0;
    for (int i = 0; i < n; ++i) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double d = pos[3 * i + a] - mean[a];
            d2 += d * d;
        }
        rmax = std::max(rmax, std::sqrt(d2));
    }
    for (int i = 0; i < n; ++i) {
        const float* w = cams[i].world_to_cam;
        for (int a = 0; a < 3; ++a) {
            f[6 * i + a] = rmax > 0.0 ? (pos[3 * i + a] - mean[a]) / rmax : 0.0;
            f[6 * i + 3 + a] = (double)w[8 + a];  // third row of R: the camera's +z axis in world space
        }
    }
}

double dist2(const double* a, const double* b) {
    double s = 0.0;
    for (int j = 0; j < 6; ++j) {
        const double d = a[j] - b[j];
        s += d * d;
    }
    return s;
}

}  // namespace

extern "C" {

lmrs_status lmrs_view_sampler_create(const lmrs_camera* cams, int32_t n_cams, int32_t n_clusters, uint64_t seed,
                                     lmrs_view_sampler** out) {
    if (!out) return LMRS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cams || n_cams <= 0 || n_clusters <= 0) return LMRS_ERR_INVALID_ARG;
    auto* S = new lmrs_view_sampler();
    S->n = n_cams;
    S->k = std::min(n_clusters, n_cams);
    S->seed = seed;
    std::vector<double> f;
    camera_features(cams, n_cams, f);
    const int n = n_cams, k = S->k;
    // k-means++ initialisation
    std::vector<double> cen((size_t)k * 6);
    uint64_t st = lmrs::step_state(seed, -1, 1);
    int first = std::min(n - 1, (int)std::floor(lmrs::sm64_unit(st) * n));
    std::copy(&f[6 * first], &f[6 * first] + 6, &cen[0]);
    std::vector<double> d2(n);
    for (int i = 0; i < n; ++i) d2[i] = dist2(&f[6 * i], &cen[0]);
    for (int c = 1; c < k; ++c) {
        double tot = 0.0;
        for (int i = 0; i < n; ++i) tot += d2[i];
        int pick = 0;
        if (tot > 0.0) {
            const double thr = lmrs::sm64_unit(st) * tot;
            double run = 0.0;
            pick = n - 1;
            for (int i = 0; i < n; ++i) {
                run += d2[i];
                if (run > thr) {
                    pick = i;
                    break;
                }
            }
        } else {
            pick = c % n;  // every point coincides with a centre
        }
        std::copy(&f[6 * pick], &f[6 * pick] + 6, &cen[6 * c]);
        for (int i = 0; i < n; ++i) d2[i] = std::min(d2[i], dist2(&f[6 * i], &cen[6 * c]));
    }
    // Lloyd iterations
    S->label.assign(n, -1);
    for (int it = 0; it < 100; ++it) {
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            int best = 0;
            double bd = dist2(&f[6 * i], &cen[0]);
            for (int c = 1; c < k; ++c) {
                const double d = dist2(&f[6 * i], &cen[6 * c]);
                if (d < bd) {
                    bd = d;
                    best = c;
                }
            }
            if (S->label[i] != best) {
                S->label[i] = best;
                changed = true;
            }
        }
        S->iterations = it + 1;
        if (!changed) break;
        std::vector<double> sum((size_t)k * 6, 0.0);
        std::vector<int> cnt(k, 0);
        for (int i = 0; i < n; ++i) {
            ++cnt[S->label[i]];
            for (int j = 0; j < 6; ++j) sum[6 * S->label[i] + j] += f[6 * i + j];
        }
        for (int c = 0; c < k; ++c)
            if (cnt[c] > 0)
                for (int j = 0; j < 6; ++j) cen[6 * c + j] = sum[6 * c + j] / cnt[c];
    }
    S->members.assign(k, {});
    for (int i = 0; i < n; ++i) S->members[S->label[i]].push_back(i);
    *out = S;
    return LMRS_OK;
}

lmrs_status lmrs_view_sampler_destroy(lmrs_view_sampler* S) {
    if (!S) return LMRS_ERR_INVALID_ARG;
    delete S;
    return LMRS_OK;
}

lmrs_status lmrs_view_sampler_labels(const lmrs_view_sampler* S, int32_t* labels, int32_t* n_clusters,
                                     int32_t* iterations) {
    if (!S) return LMRS_ERR_INVALID_ARG;
    if (labels) std::copy(S->label.begin(), S->label.end(), labels);
    if (n_clusters) *n_clusters = S->k;
    if (iterations) *iterations = S->iterations;
    return LMRS_OK;
}

lmrs_status lmrs_view_sampler_draw(const lmrs_view_sampler* S, int64_t step, int32_t* views, int32_t* n_views) {
    if (!S || !views) return LMRS_ERR_INVALID_ARG;
    std::vector<int32_t> out;
    for (int c = 0; c < S->k; ++c) {
        const auto& m = S->members[c];
        if (m.empty()) continue;
        uint64_t st = lmrs::step_state(S->seed, step, 2 + (uint64_t)c);
        const int r = std::min((int)m.size() - 1, (int)std::floor(lmrs::sm64_unit(st) * (double)m.size()));
        out.push_back(m[r]);
    }
    std::sort(out.begin(), out.end());
    std::copy(out.begin(), out.end(), views);
    if (n_views) *n_views = (int32_t)out.size();  // fewer than the clusters only if one came out empty
    return LMRS_OK;
}

lmrs_status lmrs_uniform_views(int32_t n_cams, int32_t n_views, uint64_t seed, int64_t step, int32_t* views) {
    if (!views || n_cams <= 0) return LMRS_ERR_INVALID_ARG;
    std::vector<int32_t> out;
    lmrs::uniform_views(n_cams, n_views, seed, step, out);
    std::copy(out.begin(), out.end(), views);
    return LMRS_OK;
}

}  // extern "C"
