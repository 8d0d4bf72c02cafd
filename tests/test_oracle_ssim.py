"""Pins of the oracle's diagonal SSIM term (supplementary material, "Results
with SSIM loss"): the SSIM value against a separate evaluation through
scipy's image correlation, closed forms, the own-pixel derivative against
central differences, and the stacked least-squares operator against dense
Jacobians."""
import numpy as np
import pytest

import oracle

from helpers import jvp_jacobian, small_scene

scipy_ndimage = pytest.importorskip("scipy.ndimage")

C1, C2 = 0.01 ** 2, 0.03 ** 2


def _window():
    """11 x 11 Gaussian window, sigma 1.5, as the outer product of the
    normalised 1D window."""
    t = np.arange(-5, 6, dtype=np.float64)
    g = np.exp(-t * t / (2 * 1.5 ** 2))
    g /= g.sum()
    return np.outer(g, g)


def _ssim_map(X, Y):
    """SSIM per pixel and channel, zero padding (Wang et al. 2004)."""
    win = _window()
    out = np.empty_like(X)
    for ch in range(3):
        x, y = X[..., ch], Y[..., ch]
        f = lambda a: scipy_ndimage.correlate(a, win, mode="constant", cval=0.0)
        mx, my = f(x), f(y)
        vx, vy, cxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
        out[..., ch] = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return out


def _images(seed, H=19, W=23):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (H, W, 3))
    Y = np.clip(X + rng.normal(0.0, 0.15, (H, W, 3)), 0.0, 1.0)
    return X, Y


PIXELS = [(0, 0), (22, 18), (11, 9), (3, 15), (20, 1), (6, 6)]


def test_ssim_matches_scipy_correlation_everywhere():
    X, Y = _images(1)
    ref = _ssim_map(X, Y)
    H, W = X.shape[:2]
    for py in range(H):
        for px in range(W):
            s, _ = oracle.ssim_pixel(X, Y, px, py)
            np.testing.assert_allclose(1.0 - s, ref[py, px], rtol=0, atol=1e-12)


def test_identical_images_have_zero_residual_and_derivative():
    X, _ = _images(2)
    for px, py in PIXELS:
        s, d = oracle.ssim_pixel(X, X, px, py)
        np.testing.assert_allclose(s, 0.0, atol=1e-14)
        # SSIM is maximal (1) at X = Y, so its derivative vanishes there
        np.testing.assert_allclose(d, 0.0, atol=1e-10)


def test_constant_images_closed_form():
    a, b = 0.3, 0.7
    X = np.full((21, 21, 3), a)
    Y = np.full((21, 21, 3), b)
    s, d = oracle.ssim_pixel(X, Y, 10, 10)
    ssim = (2 * a * b + C1) / (a * a + b * b + C1)  # variances and covariance vanish
    np.testing.assert_allclose(1.0 - s, ssim, rtol=1e-11)  # E[X^2] - mu^2 cancels to ~1e-16 against C2
    # derivative: only the luminance factor moves, d mu_x = g0
    g0 = _window()[5, 5]
    dssim = g0 * (2 * b * (a * a + b * b + C1) - (2 * a * b + C1) * 2 * a) / (a * a + b * b + C1) ** 2
    np.testing.assert_allclose(d, -dssim, rtol=1e-9)


@pytest.mark.parametrize("seed", [3, 4])
def test_derivative_matches_central_differences(seed):
    X, Y = _images(seed)
    h = 1e-6
    for px, py in PIXELS:
        _, d = oracle.ssim_pixel(X, Y, px, py)
        for ch in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[py, px, ch] += h
            Xm[py, px, ch] -= h
            fd = (oracle.ssim_pixel(Xp, Y, px, py)[0][ch] - oracle.ssim_pixel(Xm, Y, px, py)[0][ch]) / (2 * h)
            assert abs(d[ch] - fd) <= 1e-6 * max(abs(fd), 1e-3), (px, py, ch, d[ch], fd)
    # and the other channels do not move with this one
    Xp = X.copy()
    Xp[5, 5, 0] += 1e-3
    s0, _ = oracle.ssim_pixel(X, Y, 5, 5)
    s1, _ = oracle.ssim_pixel(Xp, Y, 5, 5)
    assert s1[1] == s0[1] and s1[2] == s0[2] and s1[0] != s0[0]


def _ssim_scene(weight=0.2, **cfg):
    sc = small_scene(51, sh_degree=1)
    tgt_sc = small_scene(52, sh_degree=1)
    o = oracle.OracleScene(tgt_sc.params, sc.cams, sc.n_gauss, 1)
    o.begin_step([0, 1])
    targets = np.stack([o.render_full(v)[0] for v in range(2)]).astype(np.float32)
    base = dict(sample_frac=0.4, weight_mode=1, lambda_=0.1, damping_mode=1, ssim_weight=weight)
    base.update(cfg)
    osc = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 1, targets=targets, **base)
    osc.begin_step([1, 0], step=2)
    return osc, targets


def test_scene_ssim_values_are_those_of_the_full_frames():
    osc, targets = _ssim_scene()
    s, d, flags = osc.ssim()
    smp = osc.samples()
    assert (flags == 0).mean() > 0.9
    for slot, cam in enumerate([1, 0]):
        img = osc.render_full(slot)[0]
        ref = 1.0 - _ssim_map(img, targets[cam].astype(np.float64))
        m = smp["slot"] == slot
        np.testing.assert_allclose(s[m], ref[smp["py"][m], smp["px"][m]], rtol=0, atol=1e-12)
    assert np.abs(s).max() > 1e-2 and np.abs(d).max() > 1e-2


@pytest.mark.parametrize("damping_mode", [0, 1])
def test_operator_rhs_diag_are_the_stacked_least_squares(damping_mode):
    """With the SSIM term the residual vector stacks r and sqrt(lam_s) s; the
    Jacobian of s at a sample is d times the colour's row (the diagonal
    approximation), so J^T W J becomes J^T diag(w (1 + lam_s d^2)) J and the
    right-hand side J^T W (r + lam_s d s)."""
    lam_s = 0.2
    osc, _ = _ssim_scene(lam_s, damping_mode=damping_mode)
    J = jvp_jacobian(osc)
    w = np.repeat(osc.samples()["w"], 3)
    s, d, _ = osc.ssim()
    s, d = s.reshape(-1), d.reshape(-1)
    om = w * (1.0 + lam_s * d * d)
    D = osc.diag()
    np.testing.assert_allclose(D, (om[:, None] * J * J).sum(0), rtol=1e-10, atol=1e-14 * D.max())
    A = J.T @ (om[:, None] * J) + 0.1 * np.diag(D if damping_mode == 1 else np.ones_like(D))
    rng = np.random.default_rng(7)
    v = rng.standard_normal(osc.n_params)
    Av = osc.apply(v, D)
    np.testing.assert_allclose(Av, A @ v, rtol=1e-10, atol=1e-12 * np.abs(A @ v).max())
    _, r, _ = osc.render_samples()
    b = osc.rhs()
    b_ref = J.T @ (w * (r.reshape(-1) + lam_s * d * s))
    np.testing.assert_allclose(b, b_ref, rtol=1e-9, atol=1e-12 * np.abs(b_ref).max())
    # the SSIM term changes the system: the weights are not all 1 + 0
    assert np.abs(om / w - 1.0).max() > 1e-3


def test_zero_weight_is_the_mse_system():
    on, _ = _ssim_scene(0.2)
    off, _ = _ssim_scene(0.0)
    s, d, _ = off.ssim()
    assert not s.any() and not d.any()
    v = np.random.default_rng(8).standard_normal(on.n_params)
    D_on, D_off = on.diag(), off.diag()
    assert np.linalg.norm(D_on - D_off) > 1e-6 * np.linalg.norm(D_off)
    J = jvp_jacobian(off)
    w = np.repeat(off.samples()["w"], 3)
    np.testing.assert_allclose(off.apply(v, D_off), J.T @ (w * (J @ v)) + 0.1 * D_off * v, rtol=1e-10,
                               atol=1e-12 * np.abs(D_off).max())
