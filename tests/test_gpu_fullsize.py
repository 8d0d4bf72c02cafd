"""Parity at the full sizes of the benchmarked workloads, on outputs the
oracle computes one by one:
  moderate: 200k Gaussians, SH3, 8 of 24 views of 1024x672, 10% of every
            tile sampled;
  large:    1.5M Gaussians, SH3, 12 of 100 views of 1297x840, 25% sampled
            (FP32 per-sample caches here: the benchmark's BF16-cache mode
            reports its own difference from them);
with the benchmark's scenes, first view sets, seed and damping.  Compared:
the whole sample set and tile lists bit for bit, the residuals and J v of
4096 random samples, and the damped operator, diag(J^T W J) and J^T W r of
the parameters of 256 random Gaussians.  Targets are seeded noise (the
shared input generator), so no oracle input comes from the CUDA path."""
import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

from gpu_common import Pair

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-5
OP_TOL = 1e-4


WORKLOADS = {
    # scene, views per step, sampled fraction (the benchmark's)
    "moderate": (syn.moderate_scene, 8, 0.1),
    "large": (syn.large_scene, 12, 0.25),
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def full(request):
    make, nviews, frac = WORKLOADS[request.param]
    sc = make()  # the benchmark's scene (same default seed)
    tgt = syn.noise_targets(np.random.default_rng(5), len(sc.cams), sc.height, sc.width)
    pair = Pair(sc, tgt, sample_frac=frac, lambda_=0.1, damping_mode=0, cg_iters=8, seed=0x5EED)
    views = syn.view_subset(np.random.default_rng(77), len(sc.cams), nviews)  # the first benchmarked view set
    pair.begin(list(views), step=3)
    # the oracle follows the device's outcome at its flagged samples
    # (gpu_common.adopt_device_decisions): every comparison below is exact
    flagged, flipped, worst = pair.adopt()
    print(f"{request.param}: {flagged} of {pair.S} samples flagged, {flipped} taken the other way, "
          f"worst score {worst:.3f}")
    assert worst <= 1.0
    rng = np.random.default_rng(2)
    pair.sample_idx = np.sort(rng.choice(pair.S, 4096, replace=False)).astype(np.int64)
    pair.gids = np.sort(rng.choice(sc.n_gauss, 256, replace=False)).astype(np.int32)
    _, _, flags = pair.orc.render_samples()
    pair.flags = flags != 0
    yield pair
    pair.gpu.close()


def _param_index(G, K3, g, j):
    if j < 3:
        return 3 * g + j
    if j < 6:
        return 3 * G + 3 * g + j - 3
    if j < 10:
        return 6 * G + 4 * g + j - 6
    if j == 10:
        return 10 * G + g
    return 11 * G + K3 * g + j - 11


def _blocks(pair, vec):
    """The gids' parameter blocks of a P-vector, (n, Pg)."""
    G = pair.scene.n_gauss
    K3 = 3 * (pair.scene.sh_degree + 1) ** 2
    Pg = 11 + K3
    idx = np.array([[_param_index(G, K3, int(g), j) for j in range(Pg)] for g in pair.gids])
    return vec[idx]


def test_samples_and_tile_lists_bit_exact(full):
    off, tile_off = full.lmrs.lmrs_get_samples(full.gpu.h, full.gpu.n_views, full.gpu.n_tiles)
    ref = full.orc.samples()
    np.testing.assert_array_equal(tile_off, ref["tile_off"])
    np.testing.assert_array_equal(off, ref["off"])
    ranges, ids = full.lmrs.lmrs_get_tile_lists(full.gpu.h, full.gpu.n_views, full.gpu.n_tiles)
    r_ref, ids_ref = full.orc.lists()
    assert len(ids) == len(ids_ref) > 10_000_000
    np.testing.assert_array_equal(ids, ids_ref)
    len_gpu, len_ref = ranges[:, 1] - ranges[:, 0], r_ref[:, 1] - r_ref[:, 0]
    np.testing.assert_array_equal(len_gpu, len_ref)


def test_sampled_residuals_and_jvp(full):
    resid = full.zeros(full.S * 3)
    full.lmrs.lmrs_render(full.gpu.h, None, resid)
    r = full.host(resid).reshape(-1, 3)[full.sample_idx]
    rgb_ref, fl = full.orc.render_samples_subset(full.sample_idx)
    # a sample is flagged when any of its alpha or termination tests lies
    # within the oracle's relative margin of the threshold; at these sizes a
    # sample makes hundreds of alpha tests, so ~1.5-2% are flagged (compared
    # too: the oracle takes the device's outcome there)
    assert (fl == 0).mean() > 0.97
    # residual = colour - target: the device's colour at the sampled pixels
    smp = full.orc.samples()
    cams = np.asarray(full.views)[smp["slot"][full.sample_idx]]
    targets = full.targets_np[cams, smp["py"][full.sample_idx], smp["px"][full.sample_idx]].astype(np.float64)
    np.testing.assert_allclose(r + targets, rgb_ref, atol=PIX_TOL, rtol=0)
    v = np.random.default_rng(3).standard_normal(full.P).astype(np.float32)
    u = full.zeros(full.S * 3)
    full.lmrs.lmrs_jvp(full.gpu.h, full.cuda(v), u)
    u_got = full.host(u).reshape(-1, 3)[full.sample_idx]
    u_ref = full.orc.jvp_subset(v.astype(np.float64), full.sample_idx)
    err = np.linalg.norm(u_got - u_ref) / np.linalg.norm(u_ref)
    print(f"J v of 4096 samples: {err:.3e}")
    assert err <= OP_TOL, err


def test_operator_diag_rhs_of_sampled_gaussians(full):
    full.lmrs.lmrs_jtj_diag(full.gpu.h)
    d = full.zeros(full.P)
    full.lmrs.lmrs_jtj_diag(full.gpu.h, d)
    D_got = _blocks(full, full.host(d))
    D_ref = full.orc.diag_gauss(full.gids)
    err = np.linalg.norm(D_got - D_ref) / np.linalg.norm(D_ref)
    assert err <= OP_TOL, f"diag {err:.2e}"
    v = np.random.default_rng(4).standard_normal(full.P).astype(np.float32)
    v64 = v.astype(np.float64)
    out = full.zeros(full.P)
    full.lmrs.lmrs_jtjv(full.gpu.h, full.cuda(v), out)
    got = _blocks(full, full.host(out))
    ref = full.orc.apply_gauss(v64, np.zeros(full.P), full.gids)  # lambda I damping
    err_op = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    b = full.zeros(full.P)
    full.lmrs.lmrs_rhs(full.gpu.h, b)
    b_got = _blocks(full, full.host(b))
    b_ref = _rhs_gauss(full)
    err_b = np.linalg.norm(b_got - b_ref) / np.linalg.norm(b_ref)
    print(f"256 Gaussians: diag {err:.3e}, operator {err_op:.3e}, right-hand side {err_b:.3e}")
    assert err_op <= OP_TOL and err_b <= OP_TOL


def _rhs_gauss(full):
    """J^T W r restricted to the sampled Gaussians' blocks (oracle)."""
    _, r_all, _ = full.orc.render_samples()
    w = full.orc.samples()["w"]
    return full.orc.vjp_gauss(r_all * w[:, None], full.gids)


def test_bf16_cache_mode_against_the_oracle(full):
    """BF16 per-sample caches (the final colour of every sample stored in
    BF16, cache_bf16=1) against the FP64 oracle, on the paths that read the
    cache: J^T W r (lmrs_rhs) and diag(J^T W J) (lmrs_jtj_diag) of the sampled
    Gaussians, and the solution of one LM step against the same step with
    FP32 caches, in the A-norm of the device's damped operator (the oracle's
    PCG over the whole parameter vector is beyond this size).  The cache
    enters through the suffix (C_final - C_<=n) / (1 - alpha_n) of the alpha
    cotangent: BF16 keeps 8 significant bits of C_final, so the suffix of a
    late entry carries an absolute error of about 2^-9 C_final, the same sign
    at every entry of a sample.  The damped operator of the PCG loop
    recomputes the colour and does not read it.  Measured on the 200k
    workload: J^T W r 9.1e-3, diag 5.7e-4, solution 7.4e-2 (the 8 PCG
    iterations amplify the right-hand side's error); held at about twice
    that.  The FP32 caches (the default, 12 bytes per sample) meet the 1e-4
    bars above."""
    torch = full.torch
    cfg = dict(full.cfg, cache_bf16=1)
    gpu16 = full.lmrs.Scene(torch.from_numpy(full.scene.params).cuda(), full.scene.cams, full.scene.n_gauss,
                            full.scene.sh_degree, targets=full.targets, **cfg)
    try:
        gpu16.preprocess(full.views, 3)
        full.lmrs.lmrs_render(gpu16.h)
        b = full.zeros(full.P)
        full.lmrs.lmrs_rhs(gpu16.h, b)
        b_ref = _rhs_gauss(full)
        err_b = np.linalg.norm(_blocks(full, full.host(b)) - b_ref) / np.linalg.norm(b_ref)
        d = full.zeros(full.P)
        full.lmrs.lmrs_jtj_diag(gpu16.h, d)
        D_ref = full.orc.diag_gauss(full.gids)
        err_d = np.linalg.norm(_blocks(full, full.host(d)) - D_ref) / np.linalg.norm(D_ref)
        # one LM step (solve only: its parameters are not used again) in both cache modes
        xs = []
        for cache in (0, 1):
            sc = full.lmrs.Scene(torch.from_numpy(full.scene.params).cuda(), full.scene.cams, full.scene.n_gauss,
                                 full.scene.sh_degree, targets=full.targets, **dict(full.cfg, cache_bf16=cache))
            full.lmrs.lmrs_lm_step(sc.h, full.views, 3)
            x = full.zeros(full.P)
            full.lmrs.lmrs_get_solution(sc.h, x)
            xs.append(x)
            sc.close()
        e = xs[1] - xs[0]
        Ae, Ax = full.zeros(full.P), full.zeros(full.P)
        full.lmrs.lmrs_jtj_diag(full.gpu.h)
        full.lmrs.lmrs_jtjv(full.gpu.h, e, Ae)
        full.lmrs.lmrs_jtjv(full.gpu.h, xs[0], Ax)
        err_x = float(torch.sqrt(torch.clamp(e @ Ae, min=0.0) / (xs[0] @ Ax)))
        print(f"BF16 caches vs FP64 oracle, 256 Gaussians: J^T W r {err_b:.3e}, diag {err_d:.3e}; "
              f"LM-step solution vs FP32 caches, A-norm {err_x:.3e}")
        assert err_b <= 2e-2 and err_d <= 2e-3 and err_x <= 0.15
    finally:
        gpu16.close()
