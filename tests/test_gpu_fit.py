"""The LM-RS fit loop and the full-frame MSE on the device."""
import numpy as np
import pytest

import oracle
from oracle import views as ov
from paper_2504_12905_gb300 import synthetic as syn

from gpu_common import oracle_targets
from helpers import normwise_rel

pytestmark = pytest.mark.gpu


def _scene(torch, lmrs, params, sc, targets, **cfg):
    base = dict(sample_frac=0.5, lambda_=0.1, damping_mode=0, cg_iters=4, seed=0x5EED)
    base.update(cfg)
    t = torch.from_numpy(targets).cuda()
    s = lmrs.Scene(torch.from_numpy(params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree, targets=t, **base)
    s._t = t
    return s


def _setup():
    sc = syn.tiny_scene(n_gauss=800)
    sc = syn.Scene(sc.n_gauss, 0, sc.params, syn.hemisphere_cameras(10, 3.0, 64, 64), sc.seed)
    tgt = oracle_targets(sc, sc.params)
    start = syn.perturb(np.random.default_rng(4), sc.params, 0.03)
    return sc, tgt, start


def test_eval_mse_matches_full_renders_and_oracle():
    import torch

    from paper_2504_12905_gb300 import lmrs
    sc, tgt, start = _setup()
    s = _scene(torch, lmrs, start, sc, tgt)
    mse = lmrs.lmrs_eval_mse(s.h)
    n = len(sc.cams)
    img = torch.zeros((n, 64, 64, 3), device="cuda")
    lmrs.lmrs_preprocess(s.h, list(range(n)), 0)
    lmrs.lmrs_render(s.h, img)
    lmrs.lmrs_synchronize(s.h)
    direct = float(((img.cpu().numpy().astype(np.float64) - tgt) ** 2).mean())
    assert mse == pytest.approx(direct, rel=1e-6)
    o = oracle.OracleScene(start, sc.cams, sc.n_gauss, 0)
    o.begin_step(list(range(n)))
    ref = np.mean([((o.render_full(v)[0] - tgt[v]) ** 2).mean() for v in range(n)])
    assert mse == pytest.approx(ref, rel=1e-4)


def test_fit_equals_manual_steps_and_follows_the_schedule():
    import torch

    from paper_2504_12905_gb300 import lmrs
    sc, tgt, start = _setup()
    a = _scene(torch, lmrs, start, sc, tgt)
    recs = lmrs.lmrs_fit(a.h, n_steps=5, views_first=3, views_later=3, cg_first=4, cg_later=4, switch_step=0,
                         view_mode=0, seed=77)
    b = _scene(torch, lmrs, start, sc, tgt)
    for k in range(5):
        views = ov.uniform_views(len(sc.cams), 3, 77, k)
        st = lmrs.lmrs_lm_step(b.h, views, k)
        assert recs[k].loss == pytest.approx(st.loss, rel=1e-5)
    pa = np.zeros(a.n_params, np.float32)
    pb = np.zeros(b.n_params, np.float32)
    lmrs.lmrs_get_params(a.h, pa)
    lmrs.lmrs_get_params(b.h, pb)
    assert normwise_rel(pa - start, pb - start) <= 1e-3
    # the schedule: views and PCG iterations switch at switch_step
    c = _scene(torch, lmrs, start, sc, tgt)
    recs = lmrs.lmrs_fit(c.h, n_steps=6, views_first=2, views_later=5, cg_first=3, cg_later=6, switch_step=3,
                         view_mode=1, seed=5)
    assert [r.n_views for r in recs] == [2, 2, 2, 5, 5, 5]
    assert [r.cg_iters for r in recs] == [3, 3, 3, 6, 6, 6]


def test_kmeans_fit_reduces_the_full_frame_error():
    import torch

    from paper_2504_12905_gb300 import lmrs
    sc, tgt, start = _setup()
    s = _scene(torch, lmrs, start, sc, tgt)
    before = lmrs.lmrs_eval_mse(s.h)
    recs = lmrs.lmrs_fit(s.h, n_steps=12, views_first=4, cg_first=5, view_mode=1, eval_every=4, seed=3)
    evals = [r.psnr for r in recs if r.mse_full >= 0]
    assert len(evals) == 3
    assert recs[-1].mse_full < before
    assert all(r.ms > 0 for r in recs)
