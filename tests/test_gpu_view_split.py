"""The operator in two view groups (view_split: the second group's
preprocessing-JVP and raster on a helper stream beside the first group's
raster) against the FP64 oracle, and against the one-group operator on the
same device.  Both sum the same per-view terms; only the arrival order of
the float atomics differs, so the two device results agree far inside the
oracle bar."""
import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

from gpu_common import Pair, assert_groups_close, assert_pvec_close
from helpers import normwise_rel

pytestmark = pytest.mark.gpu

OP_TOL = 1e-4
CG_TOL = 1e-3


def _scene(n_views=6, n_gauss=3000, width=160, height=120, sh_degree=2, seed=41):
    rng = np.random.default_rng(seed)
    params = syn.draw_gaussians(rng, n_gauss, sh_degree, means=syn.blob_means(rng, n_gauss, n_blobs=6))
    cams = syn.hemisphere_cameras(n_views, 3.0, width, height)
    tgt = syn.noise_targets(rng, n_views, height, width)
    return syn.Scene(n_gauss, sh_degree, params, cams, seed), tgt


@pytest.mark.parametrize("view_split", [1, 3, -1])
@pytest.mark.parametrize("damping_mode", [0, 1])
def test_split_operator_matches_oracle_and_one_group(view_split, damping_mode):
    sc, tgt = _scene()
    views = [5, 0, 3, 1, 4, 2]
    cfg = dict(sample_frac=0.25, damping_mode=damping_mode, lambda_=0.1)
    one = Pair(sc, tgt, **cfg)
    two = Pair(sc, tgt, view_split=view_split, **cfg)
    v = np.random.default_rng(4).standard_normal(one.P).astype(np.float32)
    outs = []
    for pair in (one, two):
        pair.begin(views, step=3)
        assert pair.adopt()[2] <= 1.0
        pair.lmrs.lmrs_jtj_diag(pair.gpu.h)
        out = pair.zeros(pair.P)
        pair.lmrs.lmrs_jtjv(pair.gpu.h, pair.cuda(v), out)
        outs.append(pair.host(out))
    D_ref = two.orc.diag()
    ref = two.orc.apply(v.astype(np.float64), D_ref)
    assert_pvec_close(outs[1], ref, OP_TOL, "(J^T W J + lambda D) v, two view groups")
    assert_groups_close(two, outs[1], ref, OP_TOL)
    d = normwise_rel(outs[1], outs[0])
    print(f"view_split {view_split}: two groups vs one {d:.2e}")
    assert d <= 1e-5
    one.gpu.close()
    two.gpu.close()


@pytest.mark.parametrize("view_split", [2, 5])
def test_split_lm_step_matches_one_group(view_split):
    """A whole LM step (its PCG runs the operator in two groups at every
    iteration) against the one-group step: solution, loss, step size."""
    sc, tgt = _scene(n_views=8, n_gauss=4000, sh_degree=3, seed=43)
    views = list(range(8))
    res = []
    for vs in (0, view_split):
        pair = Pair(sc, tgt, sample_frac=0.1, damping_mode=0, lambda_=0.1, cg_iters=8, view_split=vs)
        st = pair.lmrs.lmrs_lm_step(pair.gpu.h, views, 4)
        x = np.zeros(pair.P, np.float32)
        pair.lmrs.lmrs_get_solution(pair.gpu.h, x)
        res.append((st, x))
        pair.gpu.close()
    (st0, x0), (st1, x1) = res
    d = normwise_rel(x1, x0)
    print(f"view_split {view_split}: LM-step solution, two groups vs one {d:.2e}")
    assert d <= 1e-4
    assert st1.loss == pytest.approx(st0.loss, rel=1e-6)
    assert st1.eta == pytest.approx(st0.eta, rel=1e-4)
    assert st1.rz0 == pytest.approx(st0.rz0, rel=1e-6)


def test_view_split_is_validated():
    from paper_2504_12905_gb300 import lmrs
    sc, _ = _scene(n_views=2, n_gauss=100)
    import torch
    with pytest.raises(lmrs.LmrsError):
        lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree, view_split=-2)
