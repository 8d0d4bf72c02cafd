"""Host logic of the fit server: the footprint model of the admission test
(no device needed)."""
import pytest

from paper_2504_12905_gb300 import build as lmrs_build


@pytest.fixture(scope="module")
def lmrs():
    lmrs_build.build()
    from paper_2504_12905_gb300 import lmrs as m
    return m


def test_footprint_model_is_monotone_and_linear(lmrs):
    cfg = lmrs.lmrs_config_default(sh_degree=1, samples_per_tile=32)
    f = lambda **k: lmrs.lmrs_footprint_bytes(cfg, **{**dict(n_gauss=20000, n_cams=16, width=512, height=512,
                                                              views_per_step=8, tiles_per_pair=8.0), **k})
    base = f()
    assert base > 0
    assert f(n_gauss=40000) > base and f(views_per_step=12) > base and f(tiles_per_pair=16.0) > base
    # one more camera adds its target image (H x W x 3 floats) and its camera record, nothing per step
    d1, d2 = f(n_cams=17) - base, f(n_cams=18) - f(n_cams=17)
    assert d1 == d2 and 512 * 512 * 12 <= d1 < 512 * 512 * 12 + 256
    # views_per_step <= 0 or above n_cams means every view
    assert f(views_per_step=0) == f(views_per_step=16) == f(views_per_step=99)
    # the P-vectors alone: 9 x 4 P bytes with P = G (11 + 3 (d+1)^2)
    P = 20000 * (11 + 12)
    assert base > 9 * 4 * P + 16 * 512 * 512 * 12


def test_footprint_model_rejects_bad_input(lmrs):
    cfg = lmrs.lmrs_config_default(sh_degree=0)
    assert lmrs.lmrs_footprint_bytes(cfg, 0, 4, 64, 64) == 0
    assert lmrs.lmrs_footprint_bytes(cfg, 100, 0, 64, 64) == 0
    assert lmrs.lmrs_footprint_bytes(cfg, 100, 4, 0, 64) == 0
    bad = lmrs.lmrs_config_default(sh_degree=4)
    assert lmrs.lmrs_footprint_bytes(bad, 100, 4, 64, 64) == 0
