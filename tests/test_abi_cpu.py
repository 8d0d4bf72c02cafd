"""CPU-side checks of the boundary: the library builds for sm_103a, loads
without a GPU, exports every entry point declared in include/lmrs.h, and
rejects bad arguments with status codes before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2504_12905_gb300 import build as lbuild
from paper_2504_12905_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "lmrs.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lmrs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = lbuild.build()
    return C.CDLL(path), path


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), f"{n} declared in lmrs.h but not exported by {path}"


def test_binding_covers_the_header():
    from paper_2504_12905_gb300 import lmrs
    assert sorted(lmrs.EXPORTS) == _declared()


def test_config_default_and_status_strings(lib):
    from paper_2504_12905_gb300 import lmrs
    cfg = lmrs.lmrs_config_default()
    assert (cfg.tile_w, cfg.tile_h, cfg.cg_iters, cfg.damping_mode) == (16, 16, 8, 1)
    assert (cfg.lr_warm, cfg.lr_cap, cfg.color_bound, cfg.warm_iters) == (0.05, 0.2, 1.0, 10)
    assert lmrs.lmrs_status_str(5) == "LMRS_ERR_NUMERIC"
    assert lmrs.lmrs_status_str(99) == "LMRS_ERR_UNKNOWN"


@pytest.mark.parametrize("bad", [dict(sh_degree=4), dict(tile_w=32, tile_h=16), dict(sample_frac=0.0),
                                 dict(damping_mode=2), dict(weight_mode=3), dict(cg_iters=-1)])
def test_bad_config_rejected_before_device(bad):
    from paper_2504_12905_gb300 import lmrs
    sc = syn.tiny_scene(n_gauss=4)
    cfg = lmrs.lmrs_config_default(**bad)
    with pytest.raises(lmrs.LmrsError) as e:
        lmrs.lmrs_scene_create(cfg, sc.n_gauss, sc.params, sc.cams)
    assert e.value.status == 1


def test_mixed_camera_sizes_rejected():
    from paper_2504_12905_gb300 import lmrs
    cams = np.concatenate([syn.ring_cameras(1, 3.0, 64, 64), syn.ring_cameras(1, 3.0, 32, 64)])
    with pytest.raises(lmrs.LmrsError):
        lmrs.lmrs_scene_create(lmrs.lmrs_config_default(), 4, syn.tiny_scene(n_gauss=4).params, cams)


def test_null_scene_is_an_error():
    from paper_2504_12905_gb300 import lmrs
    assert lmrs.lib().lmrs_synchronize(None) == 1
    assert lmrs.lmrs_num_params(None) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2504_12905_gb300 import lmrs
    monkeypatch.setattr(lmrs, "_LIB", None)
    monkeypatch.setattr(lmrs, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        lmrs.lib()


def test_release_build_reports_no_debug_checks(lib):
    L, _ = lib
    L.lmrs_debug_build.restype = C.c_int32
    assert L.lmrs_debug_build() == 0


def test_debug_library_is_selected_by_the_environment(monkeypatch):
    """LMRS_DEBUG_LIBRARY=1 points the binding at the bounds-checked build,
    which lives beside the release build; nothing else does."""
    from paper_2504_12905_gb300 import lmrs
    monkeypatch.delenv("LMRS_DEBUG_LIBRARY", raising=False)
    release = lmrs.library_path()
    monkeypatch.setenv("LMRS_DEBUG_LIBRARY", "1")
    debug = lmrs.library_path()
    monkeypatch.setenv("LMRS_DEBUG_LIBRARY", "0")
    assert lmrs.library_path() == release
    assert release == lbuild.library_path() and debug == lbuild.library_path(debug=True)
    assert os.path.dirname(release) != os.path.dirname(debug)
    assert os.path.basename(release) == os.path.basename(debug)


def test_debug_build_compiles_and_reports_itself():
    """The bounds-checked build compiles for sm_103a with LMRS_DEBUG defined
    and exports the same entry points."""
    path = lbuild.build(debug=True)
    L = C.CDLL(path)
    L.lmrs_debug_build.restype = C.c_int32
    assert L.lmrs_debug_build() == 1
    for n in _declared():
        assert hasattr(L, n), f"{n} not exported by {path}"
