"""The diagonal SSIM term (supplementary material, "Results with SSIM loss",
weights 1.0 / 0.2) on the device against the oracle.

Per-sample values: the device renders the frames in FP32 and evaluates the
window statistics in FP32 (centred, so without the E[X^2] - mu^2
cancellation); the oracle does both in FP64.  s is compared at 5e-6
absolute + 1e-4 relative.  d = -N / (B1 B2) carries the factor 1/B2 with
B2 >= C2 = 9e-4: a frame error of at most e inside the window moves every
window statistic by at most 2e (values in [0, 1]) and B2 by at most 8e, so
|delta d| <= 8 (g0 + |d|) e / C2 on top of the FP32 arithmetic, which an
FP32 emulation of the kernel's formulas on FP64 frames puts below 1e-5
relative to max(|d|, 0.1); d is compared at 1e-4 max(|d|, 0.1) plus that
propagated frame error, e measured per sample over its window (the frames
themselves are held to 1e-5).  Samples whose window holds a pixel the
oracle flags near a compositing decision are left out of the per-sample
comparison and bound the operator comparison through their contribution.
Operator, diag and right-hand side: 1e-4 normwise, as for the MSE term."""
import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

from gpu_common import Pair, assert_pvec_close, oracle_targets
from helpers import normwise_rel

pytestmark = pytest.mark.gpu

OP_TOL = 1e-4
LAM_S = 0.2


def _near(sh_degree=1, **cfg):
    """Targets rendered from perturbed parameters: s small, as in a fit."""
    sc = syn.tiny_scene(seed=5, n_gauss=1200, width=96, height=72, sh_degree=sh_degree)
    tgt = oracle_targets(sc, syn.perturb(np.random.default_rng(8), sc.params, 0.03))
    base = dict(sample_frac=0.3, weight_mode=1, ssim_weight=LAM_S)
    base.update(cfg)
    return Pair(sc, tgt, **base), [2, 0, 3]


def _noise(**cfg):
    """Uniform-noise targets: s near 1."""
    sc = syn.tiny_scene(seed=99, n_gauss=1500, width=100, height=70, sh_degree=1)
    tgt = syn.noise_targets(np.random.default_rng(17), len(sc.cams), 70, 100)
    base = dict(sample_frac=0.25, ssim_weight=LAM_S)
    base.update(cfg)
    return Pair(sc, tgt, **base), [3, 1]


CASES = {
    "near": lambda: _near(),
    "near_sh0_tile32x8": lambda: _near(0, tile_w=32, tile_h=8),
    "noise": lambda: _noise(),
    "noise_importance": lambda: _noise(sample_dist=1, samples_per_tile=24),
}


@pytest.fixture(params=list(CASES))
def case(request):
    pair, views = CASES[request.param]()
    pair.begin(views, step=4)
    pair.lmrs.lmrs_render(pair.gpu.h)
    return pair


def _unflagged(pair):
    _, _, rflags = pair.orc.render_samples()
    _, _, sflags = pair.orc.ssim()
    dflags = pair.orc.sample_flags()
    return (rflags == 0) & (sflags == 0) & (dflags == 0)


C2 = 0.03 ** 2


def _g0():
    t = np.arange(-5, 6, dtype=np.float64)
    g = np.exp(-t * t / 4.5)
    g /= g.sum()
    return g[5] * g[5]


def _window_frame_error(pair):
    """Per sample, the largest |FP32 frame - FP64 frame| inside its 11x11
    window (any channel)."""
    import scipy.ndimage
    torch = pair.torch
    nv = len(pair.views)
    H, W = pair.scene.cams[0]["height"], pair.scene.cams[0]["width"]
    img = torch.zeros((nv, H, W, 3), device="cuda")
    pair.lmrs.lmrs_render(pair.gpu.h, img)
    got = pair.host(img)
    smp = pair.orc.samples()
    e = np.zeros(pair.S)
    for slot in range(nv):
        ref, flags = pair.orc.render_full(slot)
        err = np.abs(got[slot] - ref).max(axis=2)
        err[flags != 0] = 0.0  # their samples are left out (window flag)
        assert err.max() <= 1e-5
        win = scipy.ndimage.maximum_filter(err, size=11, mode="constant", cval=0.0)
        m = smp["slot"] == slot
        e[m] = win[smp["py"][m], smp["px"][m]]
    return e


def test_ssim_values(case):
    e_win = _window_frame_error(case)
    s, d = case.lmrs.lmrs_get_ssim(case.gpu.h, case.S)
    s_ref, d_ref, _ = case.orc.ssim()
    keep = _unflagged(case)
    assert keep.mean() > 0.9
    ds = np.abs(s[keep] - s_ref[keep])
    dd = np.abs(d[keep] - d_ref[keep])
    assert np.all(ds <= 5e-6 + 1e-4 * np.abs(s_ref[keep])), ds.max()
    bound = 1e-4 * np.maximum(np.abs(d_ref[keep]), 0.1) + \
        8.0 * (_g0() + np.abs(d_ref[keep])) * e_win[keep][:, None] / C2
    assert np.all(dd <= bound), (dd / bound).max()
    # the propagated part stays small against the values compared
    assert np.median(bound) <= 0.02 * np.median(np.abs(d_ref[keep])) + 1e-4
    assert np.all(s >= 0.0)
    # the term is not degenerate here
    assert np.abs(s_ref).max() > 1e-3 and np.abs(d_ref).max() > 1e-2


def _slack(pair, v):
    """J^T diag(w (1 + lam_s d^2)) J v over the flagged samples."""
    flagged = ~_unflagged(pair)
    w = pair.orc.samples()["w"]
    _, d_ref, _ = pair.orc.ssim()
    om = (w * flagged)[:, None] * (1.0 + LAM_S * d_ref * d_ref)
    return np.linalg.norm(pair.orc.vjp(pair.orc.jvp(v) * om))


def test_operator_diag_rhs(case):
    case.lmrs.lmrs_jtj_diag(case.gpu.h)
    d = case.zeros(case.P)
    case.lmrs.lmrs_jtj_diag(case.gpu.h, d)
    D_ref = case.orc.diag()
    assert_pvec_close(case.host(d), D_ref, OP_TOL, "diag with the SSIM rows")
    v = np.random.default_rng(4).standard_normal(case.P).astype(np.float32)
    v64 = v.astype(np.float64)
    out = case.zeros(case.P)
    case.lmrs.lmrs_jtjv(case.gpu.h, case.cuda(v), out)
    ref = case.orc.apply(v64, D_ref)
    slack = _slack(case, v64)
    err = np.linalg.norm(case.host(out) - ref)
    assert err <= OP_TOL * np.linalg.norm(ref) + 3.0 * slack, (err, slack)
    assert slack <= 0.2 * np.linalg.norm(ref)
    b = case.zeros(case.P)
    case.lmrs.lmrs_rhs(case.gpu.h, b)
    b_ref = case.orc.rhs()
    flagged = ~_unflagged(case)
    if flagged.any():
        s_ref, d_ref, _ = case.orc.ssim()
        _, r, _ = case.orc.render_samples()
        w = case.orc.samples()["w"]
        slack_b = np.linalg.norm(case.orc.vjp((r + LAM_S * d_ref * s_ref) * (w * flagged)[:, None]))
    else:
        slack_b = 0.0
    assert np.linalg.norm(case.host(b) - b_ref) <= OP_TOL * np.linalg.norm(b_ref) + 3.0 * slack_b
    # the SSIM rows change the system
    off = Pair(case.scene, case.targets_np, **{**case.cfg, "ssim_weight": 0.0})
    off.begin(case.views, step=4)
    assert normwise_rel(off.orc.diag(), D_ref) > 1e-3
    off.gpu.close()


def test_lm_step_loss_includes_the_term():
    pair, views = _near()
    st = pair.lmrs.lmrs_lm_step(pair.gpu.h, views, 4)
    _, st_ref = pair.orc.lm_step(views, 4)
    assert st.loss == pytest.approx(st_ref[0], rel=1e-5)
    # and it is more than the MSE part alone
    pair.orc.set_params(pair.scene.params.astype(np.float64))
    pair.orc.begin_step(views, 4)
    _, r, _ = pair.orc.render_samples()
    w = pair.orc.samples()["w"]
    mse = float((w[:, None] * r * r).sum() / (3 * w.sum()))
    assert st.loss > mse * (1 + 1e-3)


def test_render_images_with_the_term_are_the_frames():
    pair, views = _near()
    pair.begin(views, step=1)
    import torch
    img = torch.zeros((len(views), 72, 96, 3), device="cuda")
    pair.lmrs.lmrs_render(pair.gpu.h, img)
    got = pair.host(img)
    for slot in range(len(views)):
        ref, flags = pair.orc.render_full(slot)
        ok = flags == 0
        assert ok.mean() > 0.99
        assert np.abs(got[slot][ok] - ref[ok]).max() <= 1e-5


def test_off_is_an_error_for_the_getter():
    pair, views = _near(ssim_weight=0.0)
    pair.begin(views)
    pair.lmrs.lmrs_render(pair.gpu.h)
    with pytest.raises(Exception):
        pair.lmrs.lmrs_get_ssim(pair.gpu.h, pair.S)
