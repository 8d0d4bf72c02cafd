"""Pins of the FP64 oracle against things other than itself: published
values, closed forms, finite differences, textbook solvers and invariants.

A plausible mistake anywhere in the oracle (a dropped term, a sign, a
transposed index) should fail at least one of these."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2504_12905_gb300 import synthetic as syn

from helpers import fd_jacobian, jvp_jacobian, normwise_rel, small_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Published values
# ---------------------------------------------------------------------------

def test_splitmix64_published_sequences():
    g = _golden("splitmix64.json")
    assert oracle.splitmix64(0, 1)[0] == int(g["seed_0"][0], 16)
    assert [int(x) for x in oracle.splitmix64(1234567, 5)] == g["seed_1234567"]


def test_colour_bound_is_the_papers():
    # c = Y_0 * sh_dc + 0.5 in [0, 1]  <=>  |sh_dc| <= 0.5 / Y_0 (Sec. 4.5: ~1.77)
    g = _golden("paper_constants.json")
    y0 = oracle.sh_basis(0, 0.0, 0.0, 1.0)[0]
    assert round(0.5 / y0, 2) == g["colour_parameter_bound"]["value"]


def test_parameter_count_matches_jacobian_example():
    # 14 parameters per Gaussian and 3 colour channels reproduce the Sec. 4.1
    # "exceeding 100 TB" example; one fewer group would not.
    g = _golden("paper_constants.json")["jacobian_example"]
    sc = small_scene(1)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0)
    pg = osc.n_params // sc.n_gauss
    assert pg == 14
    rows = g["views"] * g["width"] * g["height"] * 3
    tb = rows * g["gaussians"] * pg * g["bytes_per_entry"] / 1e12
    assert tb > g["lower_bound_tb"]
    assert rows * g["gaussians"] * (pg - 3) * g["bytes_per_entry"] / 1e12 < g["lower_bound_tb"]


# ---------------------------------------------------------------------------
# Spherical harmonics: orthonormal on the sphere (exact Gauss-Legendre x
# trapezoid quadrature for polynomials of degree <= 6).
# ---------------------------------------------------------------------------

def test_sh_basis_orthonormal():
    zs, wz = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phis = 2 * np.pi * np.arange(nphi) / nphi
    gram = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            Y = oracle.sh_basis(3, r * math.cos(ph), r * math.sin(ph), z)
            gram += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_degree_one_is_linear_in_direction():
    # l = 1 functions are sqrt(3/(4 pi)) times the coordinates (y, z, x)
    Y = oracle.sh_basis(1, 0.6, 0.0, 0.8)
    k = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[1:], [0.0, 0.8 * k, 0.6 * k], atol=1e-15)


# ---------------------------------------------------------------------------
# Closed forms of the forward model (Sec. 3, Eq. 4)
# ---------------------------------------------------------------------------

def _axis_camera(size=64, dist=3.0):
    """Camera on the -x axis looking at the origin; principal point at the
    centre of pixel (size/2, size/2)."""
    cam = syn.look_at_camera([-dist, 0.0, 0.0], size, size)
    cam["cx"] = size / 2 + 0.5
    cam["cy"] = size / 2 + 0.5
    return np.array([cam])


def _one_gauss_params(mean, log_scale, opacity_logit, sh_dc, quat=(1, 0, 0, 0)):
    return syn.pack_params(np.array([mean], float), np.array([[log_scale] * 3], float),
                           np.array([quat], float), np.array([opacity_logit], float),
                           np.array([[sh_dc]], float))


def test_single_gaussian_centre_pixel_is_opacity_times_colour():
    cams = _axis_camera()
    theta, sh = 0.4, [0.3, -0.5, 1.1]
    p = _one_gauss_params([0, 0, 0], -3.0, theta, sh)
    osc = oracle.OracleScene(p, cams, 1, 0)
    osc.begin_step([0])
    img, _ = osc.render_full(0)
    o = 1 / (1 + math.exp(-float(np.float32(theta))))
    y0 = 1 / (2 * math.sqrt(math.pi))
    c = y0 * np.asarray(np.float32(sh), float) + 0.5
    np.testing.assert_allclose(img[32, 32], o * c, rtol=1e-12)


def test_two_cocentred_gaussians_composite_front_to_back():
    cams = _axis_camera()
    th1, th2 = 0.7, -0.2
    sh1, sh2 = [0.5, 0.1, -0.4], [-0.9, 0.8, 0.2]
    p = syn.pack_params(np.array([[-1.0, 0, 0], [0.5, 0, 0]]), np.full((2, 3), -3.0),
                        np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]]), np.array([th2, th1]),
                        np.array([[sh2], [sh1]]))  # index order opposite to depth order
    osc = oracle.OracleScene(p, cams, 2, 0)
    osc.begin_step([0])
    img, _ = osc.render_full(0)
    f32 = lambda x: float(np.float32(x))
    a1 = 1 / (1 + math.exp(-f32(th1)))
    a2 = 1 / (1 + math.exp(-f32(th2)))
    y0 = 1 / (2 * math.sqrt(math.pi))
    c1 = y0 * np.asarray(np.float32(sh1), float) + 0.5
    c2 = y0 * np.asarray(np.float32(sh2), float) + 0.5
    # camera at x = -3 looking +x: the Gaussian at x = -1 (index 0) is in front
    front_a, front_c, back_a, back_c = a2, c2, a1, c1
    expect = front_a * front_c + (1 - front_a) * back_a * back_c
    np.testing.assert_allclose(img[32, 32], expect, rtol=1e-12)


def test_front_to_back_termination_closed_form():
    # five co-centred Gaussians in depth order with alphas .95 .95 .95 .95 .1:
    # transmittance before the 4th is 1.25e-4 and the 4th would take it below
    # 1e-4, so compositing stops there and the 5th is never reached either.
    cams = _axis_camera()
    xs = [-1.5, -1.0, -0.5, 0.0, 0.5]
    alphas = [0.95, 0.95, 0.95, 0.95, 0.1]
    logits = [math.log(a / (1 - a)) for a in alphas]
    sh = [[0.2, -0.3, 0.4], [-0.6, 0.5, 0.1], [0.9, 0.0, -0.8], [1.2, 1.2, 1.2], [-1.0, 1.0, 0.3]]
    p = syn.pack_params(np.array([[x, 0, 0] for x in xs]), np.full((5, 3), -3.0),
                        np.tile([1.0, 0, 0, 0], (5, 1)), np.array(logits), np.array([[c] for c in sh]))
    osc = oracle.OracleScene(p, cams, 5, 0)
    osc.begin_step([0])
    img, flags = osc.render_full(0)
    assert flags[32, 32] == 0
    y0 = 1 / (2 * math.sqrt(math.pi))
    a = [1 / (1 + math.exp(-float(np.float32(t)))) for t in logits]
    cols = [y0 * np.asarray(np.float32(c), float) + 0.5 for c in sh]
    T, expect = 1.0, np.zeros(3)
    for k in range(3):
        expect += cols[k] * a[k] * T
        T *= 1 - a[k]
    np.testing.assert_allclose(img[32, 32], expect, rtol=1e-12)


def test_isotropic_projection_closed_form():
    # an isotropic Gaussian at distance z on the optical axis projects to the
    # principal point with covariance (f s / z)^2 I + 0.3 I
    cams = _axis_camera(size=64, dist=3.0)
    s = math.exp(float(np.float32(-2.0)))
    p = _one_gauss_params([0, 0, 0], -2.0, 0.0, [0, 0, 0])
    osc = oracle.OracleScene(p, cams, 1, 0)
    osc.begin_step([0])
    f = osc.features(0)[0]
    fpx = float(cams[0]["fx"])
    var = (fpx * s / 3.0) ** 2 + 0.3
    np.testing.assert_allclose(f[:2], [32.5, 32.5], atol=1e-9)
    np.testing.assert_allclose(f[2:5], [1 / var, 0.0, 1 / var], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(f[5], 0.5, rtol=1e-15)


# ---------------------------------------------------------------------------
# Derivatives: central finite differences of the FP64 forward model
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed,deg", [(11, 0), (12, 1), (13, 3)])
def test_jvp_and_vjp_match_finite_differences(seed, deg):
    sc = small_scene(seed, sh_degree=deg)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, deg, sample_frac=1.0)
    views = [0, 1]
    osc.begin_step(views)
    _, _, flags = osc.render_samples()
    Jfd = fd_jacobian(osc, views)
    Jf = jvp_jacobian(osc)
    keep = np.repeat(flags == 0, 3)
    assert keep.mean() > 0.99
    scale = np.abs(Jfd[keep]).max()
    assert scale > 1e-3
    np.testing.assert_allclose(Jf[keep], Jfd[keep], atol=2e-6 * scale)
    # rows of J from the reverse pass: J^T e_i for a few samples
    rng = np.random.default_rng(seed)
    for i in rng.choice(np.nonzero(keep)[0], 12, replace=False):
        e = np.zeros(3 * osc.n_samples)
        e[i] = 1.0
        np.testing.assert_allclose(osc.vjp(e.reshape(-1, 3)), Jfd[i], atol=2e-6 * scale)


def test_adjoint_identity_tiny_config():
    sc = syn.tiny_scene()
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0)
    osc.begin_step([0, 1, 2, 3])
    rng = np.random.default_rng(5)
    v = rng.standard_normal(osc.n_params)
    u = rng.standard_normal((osc.n_samples, 3))
    lhs = float((u * osc.jvp(v)).sum())
    rhs = float((osc.vjp(u) * v).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


@pytest.mark.parametrize("weight_mode,frac", [(0, 1.0), (1, 0.3)])
def test_diag_is_weighted_column_norms(weight_mode, frac):
    sc = small_scene(21, sh_degree=1)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 1, sample_frac=frac, weight_mode=weight_mode)
    osc.begin_step([0, 1])
    J = jvp_jacobian(osc)
    w = np.repeat(osc.samples()["w"], 3)
    D = osc.diag()
    np.testing.assert_allclose(D, (w[:, None] * J * J).sum(0), rtol=1e-10, atol=1e-14 * D.max())
    if weight_mode == 1:
        assert np.all(osc.samples()["w"] > 1.0)


# ---------------------------------------------------------------------------
# The damped operator (Eq. 8) and PCG (Alg. 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("damping_mode", [0, 1])
def test_operator_is_dense_product_symmetric_pd(damping_mode):
    sc = small_scene(31, sh_degree=0)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, sample_frac=0.5, weight_mode=1,
                             lambda_=0.1, damping_mode=damping_mode)
    osc.begin_step([0, 1], step=3)
    J = jvp_jacobian(osc)
    w = np.repeat(osc.samples()["w"], 3)
    D = osc.diag()
    A = J.T @ (w[:, None] * J) + 0.1 * np.diag(D if damping_mode == 1 else np.ones_like(D))
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal(osc.n_params), rng.standard_normal(osc.n_params)
    Aa, Ab = osc.apply(a, D), osc.apply(b, D)
    np.testing.assert_allclose(Aa, A @ a, rtol=1e-10, atol=1e-12 * np.abs(A @ a).max())
    assert abs(a @ Ab - Aa @ b) <= 1e-10 * abs(a @ Ab)
    assert a @ Aa > 0 and b @ Ab > 0


def test_pcg_reaches_dense_solution():
    sc = small_scene(41, n_gauss=4, sh_degree=0)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, lambda_=0.1, damping_mode=0)
    osc.begin_step([0, 1])
    J = jvp_jacobian(osc)
    D = osc.diag()
    A = J.T @ J + 0.1 * np.eye(osc.n_params)
    b = osc.rhs()
    _, resid, _ = osc.render_samples()
    np.testing.assert_allclose(b, J.T @ resid.reshape(-1), rtol=1e-9, atol=1e-12 * np.abs(b).max())
    x_ref = np.linalg.solve(A, b)
    x, st = osc.cg(b, D, 3 * osc.n_params)
    assert normwise_rel(x, x_ref) < 1e-8


def test_pcg_first_iterate_and_monotone_error():
    sc = small_scene(42, n_gauss=5, sh_degree=0)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, lambda_=0.05, damping_mode=1)
    osc.begin_step([0, 1])
    J = jvp_jacobian(osc)
    D = osc.diag()
    A = J.T @ J + 0.05 * np.diag(D)
    b = osc.rhs()
    minv = osc.precond(D)
    z0 = minv * b
    x1, _ = osc.cg(b, D, 1)
    np.testing.assert_allclose(x1, (b @ z0) / (z0 @ A @ z0) * z0, rtol=1e-10, atol=1e-14)
    # A-norm of the error never grows along the iterations (on the support)
    sup = D > 0
    x_ref = np.zeros_like(b)
    x_ref[sup] = np.linalg.solve(A[np.ix_(sup, sup)], b[sup])
    errs = []
    for it in range(1, 12):
        x, _ = osc.cg(b, D, it)
        e = x - x_ref
        errs.append(e @ A @ e)
    assert all(e2 <= e1 * (1 + 1e-9) for e1, e2 in zip(errs, errs[1:]))


def test_scaling_weights_and_lambda_leaves_solution_unchanged():
    sc = small_scene(43, n_gauss=5, sh_degree=0, size=64)
    kw = dict(sample_frac=0.1, lambda_=0.1)
    # 64x64 image: every tile is full, so weight_mode 1 is w = 256/26 everywhere
    c = 256 / 26
    o0 = oracle.OracleScene(sc.params, sc.cams, 5, 0, weight_mode=0, damping_mode=0, **kw)
    kw1 = dict(kw)
    kw1["lambda_"] = 0.1 * c
    o1 = oracle.OracleScene(sc.params, sc.cams, 5, 0, weight_mode=1, damping_mode=0, **kw1)
    x = []
    for o in (o0, o1):
        o.begin_step([0, 1], step=2)
        D = o.diag()
        b = o.rhs()
        x.append(o.cg(b, D, 6)[0])
    assert normwise_rel(x[1], x[0]) < 1e-10
    # with diagonal damping the weight scale alone cancels
    o2 = oracle.OracleScene(sc.params, sc.cams, 5, 0, weight_mode=1, damping_mode=1, **kw)
    o3 = oracle.OracleScene(sc.params, sc.cams, 5, 0, weight_mode=0, damping_mode=1, **kw)
    y = []
    for o in (o2, o3):
        o.begin_step([0, 1], step=2)
        D = o.diag()
        y.append(o.cg(o.rhs(), D, 6)[0])
    assert normwise_rel(y[0], y[1]) < 1e-10


# ---------------------------------------------------------------------------
# Step size (Sec. 4.5, App. D) and the LM update (Alg. 1)
# ---------------------------------------------------------------------------

def test_step_size_rule_closed_form():
    sc = small_scene(51, n_gauss=3)
    osc = oracle.OracleScene(sc.params, sc.cams, 3, 0)
    G = 3
    x = np.zeros(osc.n_params)
    dc = 11 * G  # first SH entry
    assert osc.step_size(x, 0) == 0.05          # warm-up
    assert osc.step_size(x, 9) == 0.05
    assert osc.step_size(x, 10) == 0.2          # nothing to bound
    x[dc + 4] = -12.5                            # |x_dc| max = 12.5 -> 1/12.5
    x[0] = 1e6                                   # non-colour entries do not bound
    assert osc.step_size(x, 10) == pytest.approx(0.08, rel=1e-15)
    x[dc + 4] = 2.0                              # 1/2 > cap
    assert osc.step_size(x, 10) == 0.2


def test_lm_step_descends():
    sc = syn.tiny_scene()
    rng = np.random.default_rng(7)
    target_params = syn.perturb(rng, sc.params)
    tgt = oracle.OracleScene(target_params, sc.cams, sc.n_gauss, 0)
    tgt.begin_step([0, 1, 2, 3])
    targets = np.stack([tgt.render_full(s)[0] for s in range(4)]).astype(np.float32)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, targets=targets, lambda_=1e-2, cg_iters=10)
    views = [0, 1, 2, 3]
    osc.begin_step(views, 0)
    _, r0, _ = osc.render_samples()
    b = osc.rhs()
    x, st = osc.lm_step(views, 0)
    assert b @ x > 0                      # x is a descent direction for 0.5 |r|^2
    assert st[1] == 0.05
    osc.begin_step(views, 0)
    _, r1, _ = osc.render_samples()
    assert (r1 ** 2).sum() < (r0 ** 2).sum()


# ---------------------------------------------------------------------------
# Binning and sampling (integer work)
# ---------------------------------------------------------------------------

def _ellipse_scene():
    """300 large anisotropic Gaussians on a ragged 100 x 70 view, 8 of them
    too faint (o < 1/255) to reach the alpha threshold anywhere."""
    rng = np.random.default_rng(41)
    G = 300
    means = rng.uniform(-0.6, 0.6, (G, 3))
    ls = rng.normal(-2.6, 0.5, (G, 3))
    q = rng.standard_normal((G, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.normal(0.0, 1.5, G)
    opac[:8] = -7.0
    sh = np.zeros((G, 1, 3))
    sh[:, 0, :] = rng.uniform(-0.8, 0.8, (G, 3))
    cams = syn.ring_cameras(3, 3.0, 100, 70, elev_deg=20.0)
    return syn.Scene(G, 0, syn.pack_params(means, ls, q, opac, sh), cams, 41)


def _min_level(f, tx, ty, tw, th, W, H):
    """Smallest d^T Sigma2^-1 d over the tile's pixel-centre columns and its
    band of pixel-centre rows taken as an interval, in FP64: per column the
    quadratic in dy is minimised at its vertex clamped into the band."""
    mux, muy, A, B, C = f[0], f[1], f[2], f[3], f[4]
    lo = ty * th + 0.5 - muy
    hi = min(ty * th + th, H) - 0.5 - muy
    dx = np.arange(tx * tw, min(tx * tw + tw, W)) + 0.5 - mux
    dy = np.clip(-B * dx / C, lo, hi)
    return float((A * dx * dx + 2.0 * B * dx * dy + C * dy * dy).min())


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 32)])
def test_tile_lists_are_the_tiles_the_alpha_ellipse_reaches(tw, th):
    """A Gaussian's list covers the tiles of its 3-sigma rectangle where the
    ellipse alpha >= 1/255 (level 2 ln(255 o), plus a slack of 0.02) meets a
    pixel-centre column within the tile row's band, sorted by (depth,
    index).  Checked against the FP64 features by a separate formulation
    (per column, the vertex of the quadratic in dy), leaving out tiles within
    a rounding margin of the level; every tile left out has alpha < 1/255 at
    all of its pixels, so the culling changes no pixel."""
    sc = _ellipse_scene()
    W, H = 100, 70
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, tile_w=tw, tile_h=th)
    osc.begin_step([2, 0])
    ranges, ids = osc.lists()
    T, ntx = osc.n_tiles, osc.tiles_x
    dropped = kept = decided = 0
    for slot in range(2):
        vis, depth, rect = osc.geom(slot)
        f = osc.features(slot)
        lists = [list(ids[ranges[slot * T + t, 0]:ranges[slot * T + t, 1]]) for t in range(T)]
        for t in range(T):
            tx, ty = t % ntx, t // ntx
            cand = [g for g in range(sc.n_gauss) if vis[g] and rect[g, 0] <= tx <= rect[g, 1]
                    and rect[g, 2] <= ty <= rect[g, 3]]
            order = sorted(cand, key=lambda g: (float(depth[g]), g))
            got = lists[t]
            # a subsequence of the rectangle's depth order
            pos = [order.index(g) for g in got]
            assert pos == sorted(pos) and len(set(got)) == len(got)
            for g in order:
                tau = 2.0 * math.log(255.0 * f[g, 5]) + 0.02
                inside = g in got
                kept += inside
                dropped += not inside
                if tau <= 0.0:
                    assert not inside
                    continue
                m = _min_level(f[g], tx, ty, tw, th, W, H)
                if abs(m - tau) > 2e-3 * max(tau, 1.0) + 1e-3:
                    assert inside == (m < tau), (slot, t, g, m, tau)
                    decided += 1
                if not inside:
                    px = np.arange(tx * tw, min(tx * tw + tw, W)) + 0.5 - f[g, 0]
                    py = np.arange(ty * th, min(ty * th + th, H)) + 0.5 - f[g, 1]
                    dx, dy = np.meshgrid(px, py)
                    q = f[g, 2] * dx * dx + 2.0 * f[g, 3] * dx * dy + f[g, 4] * dy * dy
                    assert f[g, 5] * np.exp(-0.5 * q).max() < 1.0 / 255.0
    # the test decides nearly every entry, and the ellipse drops a good share
    assert decided >= 0.99 * (kept + dropped - 8 * 2 * 4)
    assert dropped >= 0.1 * (kept + dropped) and kept > 500


def _list_scenes():
    rng = np.random.default_rng(5)
    tiny = syn.tiny_scene()
    ragged = syn.tiny_scene(seed=99, n_gauss=1500, width=100, height=70, sh_degree=1)
    ell = _ellipse_scene()
    return {
        "tiny": (tiny, syn.noise_targets(rng, 4, 64, 64), [0, 1, 2, 3], dict(lambda_=1e-2)),
        "ragged_sh1_10pct": (ragged, syn.noise_targets(rng, 4, 70, 100), [3, 1],
                             dict(sample_frac=0.1, weight_mode=1, lambda_=0.1)),
        "ellipse_8x32": (ell, syn.noise_targets(rng, 3, 70, 100), [2, 0],
                         dict(tile_w=8, tile_h=32, lambda_=0.1)),
    }


@pytest.mark.parametrize("name", ["tiny", "ragged_sh1_10pct", "ellipse_8x32"])
def test_ellipse_lists_change_no_result(name):
    """The tile lists that follow the alpha >= 1/255 ellipse against the
    3-sigma rectangles of 3DGS (Sec. 3 defers the lists to it): every
    ellipse list is a subsequence of its rectangle list, and full frames,
    sampled renders and their flags, J v, J^T u, diag(J^T W J), J^T W r and
    the damped operator come out bit for bit the same.  An ellipse that
    missed a pixel with alpha >= 1/255 would change them."""
    sc, tgt, views, cfg = _list_scenes()[name]
    osc = {m: oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, sc.sh_degree, targets=tgt, list_mode=m, **cfg)
           for m in (0, 1)}
    for o in osc.values():
        o.begin_step(views, 3)
    (r0, i0), (r1, i1) = osc[0].lists(), osc[1].lists()
    for t in range(len(r0)):
        a, b = list(i0[r0[t, 0]:r0[t, 1]]), list(i1[r1[t, 0]:r1[t, 1]])
        it = iter(b)
        assert all(g in it for g in a), t  # subsequence, same order
    assert len(i0) < 0.9 * len(i1)
    for slot in range(len(views)):
        (im0, f0), (im1, f1) = osc[0].render_full(slot), osc[1].render_full(slot)
        np.testing.assert_array_equal(im0, im1)
        np.testing.assert_array_equal(f0, f1)
    for a, b in zip(osc[0].render_samples(), osc[1].render_samples()):
        np.testing.assert_array_equal(a, b)
    rng = np.random.default_rng(8)
    v = rng.standard_normal(osc[0].n_params)
    u = rng.standard_normal((osc[0].n_samples, 3))
    np.testing.assert_array_equal(osc[0].jvp(v), osc[1].jvp(v))
    np.testing.assert_array_equal(osc[0].vjp(u), osc[1].vjp(u))
    D0, D1 = osc[0].diag(), osc[1].diag()
    np.testing.assert_array_equal(D0, D1)
    np.testing.assert_array_equal(osc[0].rhs(), osc[1].rhs())
    np.testing.assert_array_equal(osc[0].apply(v, D0), osc[1].apply(v, D1))


def test_faint_gaussians_have_no_entries():
    sc = _ellipse_scene()
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0)
    osc.begin_step([0, 1])
    vis, _, _ = osc.geom(0)
    _, ids = osc.lists()
    assert vis[:8].any()  # visible, but alpha < 1/255 everywhere
    assert not np.isin(ids, np.arange(8)).any()


def test_fp32_rectangles_agree_with_fp64_geometry():
    # The FP32 decision pass and the FP64 features are separate code paths;
    # away from tile boundaries they must pick the same tile rectangle.
    sc = syn.tiny_scene()
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0)
    osc.begin_step([0, 1, 2, 3])
    checked = 0
    for slot in range(4):
        vis, depth, rect = osc.geom(slot)
        f = osc.features(slot)
        for g in np.nonzero(vis)[0]:
            A, B, Cc = f[g, 2:5]
            det = A * Cc - B * B
            cov = np.array([[Cc, -B], [-B, A]]) / det  # inverse of the conic
            lam = 0.5 * (cov[0, 0] + cov[1, 1]) + math.sqrt(max(0.25 * (cov[0, 0] + cov[1, 1]) ** 2 - np.linalg.det(cov), 0.1))
            r = 3 * math.sqrt(lam)
            if abs(r - round(r)) < 1e-3:
                continue
            r = math.ceil(r)
            lo = (f[g, 0] - r) / 16, (f[g, 1] - r) / 16
            hi = (f[g, 0] + r) / 16, (f[g, 1] + r) / 16
            if min(abs(v - round(v)) for v in lo + hi) < 1e-4:
                continue
            x0 = max(math.floor(lo[0]), 0); x1 = min(math.floor(hi[0]), osc.tiles_x - 1)
            y0 = max(math.floor(lo[1]), 0); y1 = min(math.floor(hi[1]), osc.tiles_y - 1)
            assert list(rect[g]) == [x0, x1, y0, y1]
            checked += 1
    assert checked > 500


def test_sampler_counts_and_distinct_offsets():
    cams = syn.ring_cameras(2, 3.0, 100, 70)  # ragged edge tiles: 7x5 tiles
    sc = small_scene(61)
    osc = oracle.OracleScene(sc.params, cams, sc.n_gauss, 0, sample_frac=0.1, weight_mode=1)
    osc.begin_step([1, 0], step=5)
    s = osc.samples()
    T = osc.n_tiles
    assert (osc.tiles_x, osc.tiles_y) == (7, 5)
    for slot in range(2):
        for t in range(T):
            tx, ty = t % 7, t // 7
            n = min(16, 100 - 16 * tx) * min(16, 70 - 16 * ty)
            k = max(1, min(n, int(math.floor(0.1 * n + 0.5))))
            b, e = s["tile_off"][slot * T + t], s["tile_off"][slot * T + t + 1]
            assert e - b == k
            off = s["off"][b:e]
            assert len(set(off.tolist())) == k and off.max() < n
            np.testing.assert_allclose(s["w"][b:e], n / k)
            assert np.all((s["px"][b:e] // 16 == tx) & (s["py"][b:e] // 16 == ty))
            assert np.all((s["px"][b:e] < 100) & (s["py"][b:e] < 70))
    assert s["tile_off"][16 * 0 + 0 + 1] == 26  # full tile, 10% of 256


def test_sampler_full_tile_is_permutation_and_keyed():
    full = oracle.sample_tile(9, 3, 2, 7, 256, 256)
    assert sorted(full.tolist()) == list(range(256))
    a = oracle.sample_tile(9, 3, 2, 7, 256, 26)
    np.testing.assert_array_equal(a, full[:26])  # partial shuffle is a prefix
    for other in [(10, 3, 2, 7), (9, 4, 2, 7), (9, 3, 1, 7), (9, 3, 2, 8)]:
        assert not np.array_equal(oracle.sample_tile(*other, 256, 26), a)
    # uniformity: every offset is drawn about equally often over many tiles
    counts = np.zeros(256)
    for t in range(4000):
        counts[oracle.sample_tile(1, 0, 0, t, 256, 32)] += 1
    expect = 4000 * 32 / 256
    assert np.abs(counts - expect).max() < 6 * math.sqrt(expect)


# ---- importance distributions of the residual sampler (supplementary) ----

def _importance_scene():
    sc = syn.tiny_scene(seed=41, n_gauss=300, width=32, height=32)
    tgt = syn.noise_targets(np.random.default_rng(2), len(sc.cams), 32, 32)
    return sc, tgt


@pytest.mark.parametrize("dist", [1, 2])
def test_importance_estimate_is_unbiased(dist):
    """E_q[sum_i w_i |r_i|^2] over the draws equals the loss over the pixels
    q can draw (the Monte Carlo identity behind the weights): every pixel for
    q_residual; for q_Gaussian the pixels some Gaussian composites, plus
    every pixel of a tile that has none (drawn uniformly)."""
    sc, tgt = _importance_scene()
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, targets=tgt, samples_per_tile=8, sample_dist=dist)
    views = [0, 2]
    o.begin_step(views, 0)
    full = 0.0
    for slot, cam in enumerate(views):
        r2 = ((o.render_full(slot)[0] - tgt[cam]) ** 2).sum(-1)
        if dist == 2:
            cnt = o.pixel_counts(slot)
            for ty in range(2):
                for tx in range(2):
                    blk = (slice(16 * ty, 16 * ty + 16), slice(16 * tx, 16 * tx + 16))
                    full += r2[blk][cnt[blk] > 0].sum() if (cnt[blk] > 0).any() else r2[blk].sum()
        else:
            full += r2.sum()
    est = []
    for step in range(300):
        o.begin_step(views, step)
        w = o.samples()["w"]
        r = o.render_samples()[1]
        est.append(float((w[:, None] * r ** 2).sum()))
    est = np.array(est)
    assert abs(est.mean() - full) <= 4.0 * est.std() / np.sqrt(len(est)) + 1e-9 * full


def test_importance_residual_weights_match_their_pixels():
    """q_residual: each draw's weight is total / (K e^{|r|}) of the drawn pixel."""
    sc, tgt = _importance_scene()
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, targets=tgt, samples_per_tile=8, sample_dist=1)
    o.begin_step([1], 3)
    smp = o.samples()
    img = o.render_full(0)[0]
    a = np.exp(np.sqrt(((img - tgt[1]) ** 2).sum(-1)))
    tile = (smp["py"] // 16) * 2 + smp["px"] // 16
    for t in range(4):
        ys, xs = np.mgrid[(t // 2) * 16:(t // 2) * 16 + 16, (t % 2) * 16:(t % 2) * 16 + 16]
        total = a[ys, xs].sum()
        m = tile == t
        np.testing.assert_allclose(smp["w"][m], total / (8 * a[smp["py"][m], smp["px"][m]]), rtol=1e-9)


def test_importance_gaussian_draws_only_covered_pixels():
    """q_Gaussian: a pixel no Gaussian composites is never drawn (unless the
    whole tile is empty, where the draw is uniform)."""
    sc, tgt = _importance_scene()
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, targets=tgt, samples_per_tile=16, sample_dist=2)
    o.begin_step([0], 5)
    smp = o.samples()
    covered = o.pixel_counts(0) > 0
    tile = (smp["py"] // 16) * 2 + smp["px"] // 16
    for t in range(4):
        ys, xs = np.mgrid[(t // 2) * 16:(t // 2) * 16 + 16, (t % 2) * 16:(t % 2) * 16 + 16]
        m = tile == t
        if covered[ys, xs].any():
            assert covered[smp["py"][m], smp["px"][m]].all()


def test_decision_outcomes_are_adopted_from_planted_values():
    """The oracle's handling of near-threshold decisions (alpha skip and
    clamp, termination within the flagging margins): with the oracle's own
    residuals and J v as the evidence every flagged sample keeps mask 0;
    with the values of the other outcome planted at every flagged sample,
    the adoption recovers that outcome everywhere, and the oracle's sample
    renders and J v then equal the planted values.  The flipped decisions
    move J^T W r, so exact sums need the adopted outcomes."""
    from gpu_common import adopt_device_decisions
    sc = syn.tiny_scene(n_gauss=3000, sh_degree=1)
    tgt = syn.noise_targets(np.random.default_rng(3), 4, 64, 64)
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 1, targets=tgt, sample_frac=1.0, lambda_=0.1,
                           seed=0x5EED)
    o.begin_step([0, 1, 2, 3], 2)
    rgb, res, fl = o.render_samples()
    idx = np.nonzero(fl)[0]
    assert len(idx) >= 5
    v = np.random.default_rng(1).standard_normal(o.n_params)
    u = o.jvp(v)
    b0 = o.rhs()
    assert adopt_device_decisions(o, res, u, v) == (len(idx), 0, 0.0)
    nn, rgb_m, u_m = o.sample_outcomes(v, idx, 4)
    assert np.all(nn >= 1)
    np.testing.assert_array_equal(rgb_m[:, 0], rgb[idx])
    np.testing.assert_array_equal(u_m[:, 0], u[idx])
    res2, u2 = res.copy(), u.copy()
    res2[idx] = rgb_m[:, 1] - (rgb[idx] - res[idx])
    u2[idx] = u_m[:, 1]
    n_fl, n_flip, worst = adopt_device_decisions(o, res2, u2, v)
    assert (n_fl, n_flip, worst) == (len(idx), len(idx), 0.0)
    rgb_f, res_f, _ = o.render_samples()
    np.testing.assert_array_equal(res_f, res2)
    np.testing.assert_array_equal(o.jvp(v), u2)
    assert np.linalg.norm(o.rhs() - b0) > 1e-6 * np.linalg.norm(b0)
    o.clear_flips()
    np.testing.assert_array_equal(o.rhs(), b0)
