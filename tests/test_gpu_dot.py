"""The PCG inner products are FP64-grade.  Each thread accumulates its FP32
products with compensated arithmetic (Dot2: TwoProduct by FMA and Knuth's
TwoSum, Ogita, Rump and Oishi 2005) and the threads' (sum, error) pairs
are added in FP64.  For non-negative terms Dot2's error is at most
gamma_n^2 times the sum, gamma_n ~ n 2^-24 with n the terms per thread (here
at most ~40: 11.8M terms over 1216 blocks of 256 threads), about 5e-12,
plus the FP64 rounding of the cross-thread sum.

Checked on r0^T z0 = sum b_j (M^-1 b)_j of a PCG solve on the 200k-Gaussian
workload's parameter vector: the host forms the same FP32 vectors (M^-1
from the device's FP32 diagonal with the preconditioner's FP32 formula,
z = M^-1 b rounded to FP32), and the exact dot of those FP32 numbers (every
product is exact in FP64, math.fsum rounds their sum once)."""
import math

import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("damping_mode", [0, 1])
def test_r0_z0_matches_the_exact_dot_of_the_same_fp32_vectors(damping_mode):
    import torch

    from paper_2504_12905_gb300 import lmrs
    sc = syn.moderate_scene()
    rng = np.random.default_rng(21)
    tgt = torch.from_numpy(syn.noise_targets(rng, len(sc.cams), sc.height, sc.width)).cuda()
    lam = 0.1
    s = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree, targets=tgt,
                   sample_frac=0.1, lambda_=lam, damping_mode=damping_mode, cg_iters=8, seed=0x5EED)
    try:
        s.preprocess(list(range(8)), 0)
        lmrs.lmrs_render(s.h)
        d = torch.zeros(s.n_params, device="cuda")
        lmrs.lmrs_jtj_diag(s.h, d)
        # a right-hand side spanning twelve decades, with both signs
        b = (rng.standard_normal(s.n_params) * 10.0 ** rng.uniform(-6, 6, s.n_params)).astype(np.float32)
        x = torch.zeros(s.n_params, device="cuda")
        st = lmrs.lmrs_cg_solve(s.h, torch.from_numpy(b).cuda(), x, 0)
        D = d.cpu().numpy()
        lam32 = np.float32(lam)
        dd = (np.float32(1.0) + lam32) * D if damping_mode == 1 else D + lam32
        with np.errstate(divide="ignore"):
            m = np.where(dd > 0, np.float32(1.0) / dd, np.float32(0.0)).astype(np.float32)
        z = (m * b).astype(np.float32)
        exact = math.fsum((b.astype(np.float64) * z.astype(np.float64)).tolist())
        rel = abs(st.rz0 - exact) / exact
        print(f"damping {damping_mode}: r0^T z0 = {st.rz0:.17g}, exact {exact:.17g}, relative error {rel:.2e}")
        assert rel <= 1e-11
    finally:
        s.close()
