"""The bounds-checked build (LMRS_DEBUG, include/lmrs.h) as a stand-in for a
memory checker: it is built beside the release library, the computation of
tests/debug_case.py runs with it in a child process, and

  * every index check passes (the debug word is 0 after each stage);
  * its results equal the release library's from the same inputs: bit for
    bit where no float atomics are involved (residuals, J v), within 1e-6
    normwise where they order the sums (J^T u, b, D, the operator), and the
    parameters after two LM steps within 1e-5 of the update (8 PCG
    iterations carry the last-bit differences of the atomics-ordered sums
    into the solution).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import normwise_rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from paper_2504_12905_gb300 import lmrs
import debug_case
assert lmrs.lmrs_debug_build() == 1, "not the LMRS_DEBUG library"
out, words = debug_case.run()
np.savez(sys.argv[1], **out)
print(json.dumps(words))
"""


def test_debug_build_checks_pass_and_results_agree(tmp_path):
    from paper_2504_12905_gb300 import build, lmrs

    import debug_case

    build.build(debug=True)
    path = tmp_path / "debug_out.npz"
    env = dict(os.environ, LMRS_DEBUG_LIBRARY="1")
    r = subprocess.run([sys.executable, "-c", CHILD, str(path), HERE], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    words = json.loads(r.stdout.strip().splitlines()[-1])
    print("debug words:", words)
    assert words and all(w == 0 for w in words.values()), words

    assert lmrs.lmrs_debug_build() == 0
    rel, words_rel = debug_case.run()
    assert all(w == 0 for w in words_rel.values())
    dbg = np.load(path)
    for name in ("residuals", "jv"):
        np.testing.assert_array_equal(dbg[name], rel[name], err_msg=name)
    for name in ("vjp", "rhs", "diag", "operator"):
        e = normwise_rel(dbg[name].astype(np.float64), rel[name].astype(np.float64))
        assert e <= 1e-6, (name, e)
    from paper_2504_12905_gb300 import synthetic as syn
    p0 = syn.tiny_scene(seed=99, n_gauss=1500, width=100, height=70, sh_degree=1).params.astype(np.float64)
    step = np.linalg.norm(rel["params"].astype(np.float64) - p0)
    diff = np.linalg.norm(dbg["params"].astype(np.float64) - rel["params"])
    print(f"parameters after two LM steps: {diff:.3e} apart, update {step:.3e}")
    assert diff <= 1e-5 * step
    np.testing.assert_allclose(dbg["losses"], rel["losses"], rtol=1e-6)
