"""Importance distributions of the residual sampler (q_residual,
q_Gaussian; supplementary material) on the device against the oracle."""
import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

from gpu_common import Pair, assert_pvec_close
from helpers import normwise_rel

pytestmark = pytest.mark.gpu

OP_TOL = 1e-4


def _case(dist, seed=17):
    rng = np.random.default_rng(seed)
    sc = syn.tiny_scene(seed=99, n_gauss=1500, width=100, height=70, sh_degree=1)
    tgt = syn.noise_targets(rng, len(sc.cams), 70, 100)
    pair = Pair(sc, tgt, samples_per_tile=24, sample_dist=dist)
    pair.begin([3, 1], step=2)
    return pair


@pytest.mark.parametrize("dist", [1, 2])
def test_importance_draws_and_weights(dist):
    pair = _case(dist)
    off, tile_off = pair.lmrs.lmrs_get_samples(pair.gpu.h, pair.gpu.n_views, pair.gpu.n_tiles)
    ref = pair.orc.samples()
    flags = pair.orc.sample_flags()
    np.testing.assert_array_equal(tile_off, ref["tile_off"])
    keep = flags == 0
    assert keep.mean() > 0.95
    np.testing.assert_array_equal(off[keep], ref["off"][keep])
    w = pair.lmrs.lmrs_get_sample_weights(pair.gpu.h, pair.S)
    np.testing.assert_allclose(w[keep], ref["w"][keep], rtol=1e-5)
    # every weight is 1 / (K q) > 0 and a tile's draws stay inside it
    assert np.all(w > 0) and np.all(off < 256)


@pytest.mark.parametrize("dist", [1, 2])
def test_importance_operator_parity(dist):
    """The damped operator and J^T W r under the importance weights match the
    oracle.  Draws the oracle flags (near a bin edge, or in a tile with a
    pixel near a compositing decision) may land on other pixels in FP32; the
    error bound adds three times the oracle's own contribution of its flagged
    draws (the GPU's draws there are as many, with weights of the same
    size)."""
    pair = _case(dist)
    flags = pair.orc.sample_flags().astype(bool)
    pair.lmrs.lmrs_render(pair.gpu.h)
    pair.lmrs.lmrs_jtj_diag(pair.gpu.h)
    D_ref = pair.orc.diag()
    rng = np.random.default_rng(4)
    v = rng.standard_normal(pair.P).astype(np.float32)
    v64 = v.astype(np.float64)
    w = pair.orc.samples()["w"]
    out = pair.zeros(pair.P)
    pair.lmrs.lmrs_jtjv(pair.gpu.h, pair.cuda(v), out)
    ref = pair.orc.apply(v64, D_ref)
    slack = np.linalg.norm(pair.orc.vjp(pair.orc.jvp(v64) * (w * flags)[:, None]))
    assert np.linalg.norm(pair.host(out) - ref) <= OP_TOL * np.linalg.norm(ref) + 3.0 * slack
    b = pair.zeros(pair.P)
    pair.lmrs.lmrs_rhs(pair.gpu.h, b)
    b_ref = pair.orc.rhs()
    r = pair.orc.render_samples()[1]
    slack_b = np.linalg.norm(pair.orc.vjp(r * (w * flags)[:, None]))
    assert np.linalg.norm(pair.host(b) - b_ref) <= OP_TOL * np.linalg.norm(b_ref) + 3.0 * slack_b
    # the bound is informative: the flagged part is a small share of the whole
    assert slack <= 0.2 * np.linalg.norm(ref)
