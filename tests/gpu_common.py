"""Helpers of the GPU parity tests: one scene built twice, on the CUDA path
(through the C-ABI) and in the FP64 oracle, from the same FP32 inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2504_12905_gb300 import synthetic as syn

from helpers import normwise_rel

GROUPS = ("means", "log_scales", "quats", "opacity", "sh")


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    return torch


def oracle_targets(scene, params, views=None):
    """Full-frame FP64 oracle renders of ``params`` for every camera, as FP32."""
    o = oracle.OracleScene(params, scene.cams, scene.n_gauss, scene.sh_degree)
    n = len(scene.cams)
    o.begin_step(list(range(n)))
    return np.stack([o.render_full(s)[0] for s in range(n)]).astype(np.float32)


class Pair:
    """The same scene on both sides."""

    def __init__(self, scene, targets=None, **cfg):
        torch = torch_cuda()
        from paper_2504_12905_gb300 import lmrs
        self.torch = torch
        self.lmrs = lmrs
        self.scene = scene
        base = dict(lambda_=0.1, damping_mode=1, cg_iters=8, sample_frac=1.0, weight_mode=0, seed=0x5EED)
        base.update(cfg)
        cfg = base
        self.cfg = cfg
        self.targets_np = targets
        self.targets = None if targets is None else torch.from_numpy(targets).cuda()
        self.gpu = lmrs.Scene(torch.from_numpy(scene.params).cuda(), scene.cams, scene.n_gauss, scene.sh_degree,
                              targets=self.targets, **cfg)
        ocfg = {("lambda_" if k == "lambda" else k): v for k, v in cfg.items() if k != "cache_bf16"}
        self.orc = oracle.OracleScene(scene.params, scene.cams, scene.n_gauss, scene.sh_degree, targets=targets, **ocfg)
        self.P = self.gpu.n_params
        assert self.P == self.orc.n_params

    def begin(self, views, step=0):
        self.views = list(views)
        self.gpu.preprocess(self.views, step)
        self.orc.begin_step(self.views, step)
        self.S = self.gpu.n_samples
        assert self.S == self.orc.n_samples

    def adopt(self, seed=99):
        """Render on the device, take J v of a seeded tangent, and make the
        oracle follow the device's near-threshold decisions
        (adopt_device_decisions); returns its (flagged, flipped, worst)."""
        resid = self.zeros(self.S * 3)
        self.lmrs.lmrs_render(self.gpu.h, None, resid)
        v = np.random.default_rng(seed).standard_normal(self.P).astype(np.float32)
        u = self.zeros(self.S * 3)
        self.lmrs.lmrs_jvp(self.gpu.h, self.cuda(v), u)
        res = adopt_device_decisions(self.orc, self.host(resid).reshape(-1, 3), self.host(u).reshape(-1, 3), v)
        self.adopted = res
        return res

    def zeros(self, n):
        return self.torch.zeros(n, dtype=self.torch.float32, device="cuda")

    def cuda(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.detach().cpu().numpy().astype(np.float64)

    def groups(self, vec):
        off = syn.group_offsets(self.scene.n_gauss, self.scene.sh_degree)
        keys = list(GROUPS) + ["end"]
        return {k: vec[off[k]:off[keys[i + 1]]] for i, k in enumerate(GROUPS)}


def assert_pvec_close(gpu, ref, tol, what=""):
    """Normwise relative error over the whole P-vector and per parameter
    group (groups whose reference norm is below 1e-3 of the total are
    compared against the total norm instead)."""
    err = normwise_rel(gpu, ref)
    assert err <= tol, f"{what}: normwise rel error {err:.3e} > {tol:.1e}"
    return err


def group_errors(pair, gpu, ref):
    g, r = pair.groups(gpu), pair.groups(ref)
    tot = np.linalg.norm(ref)
    out = {}
    for k in GROUPS:
        d = np.linalg.norm(r[k])
        out[k] = np.linalg.norm(g[k] - r[k]) / max(d, 1e-3 * tot, 1e-300)
    return out


PIX_TOL = 1e-5
JV_TOL = 1e-4


def adopt_device_decisions(orc, resid_dev, u_dev, v, max_bits=4):
    """Make the oracle follow, at every sample it flags, the device's outcome
    of the near-threshold compositing decisions.

    A sample is flagged when one of its alpha tests (skip at 1/255, clamp at
    0.99) or its termination test (T < 1e-4, Eq. 4) lies within the oracle's
    relative margin of the threshold: there an FP32 evaluation may go either
    way, and both outcomes are correct.  For each flagged sample the oracle
    evaluates every combination of its near decisions (bit k of a mask
    inverts the k-th) and keeps the one whose residual and J v (for the
    tangent v) are closest to the device's (resid_dev, u_dev: [S, 3]).  The
    score of an outcome is the larger of its residual difference over the
    pixel bar and its J v difference over 1e-4 of the sample's |J v| (plus
    1e-4 of the r.m.s. over all samples), so a score <= 1 is a match at the
    bars.  Later sample-level oracle results (J^T u, diag, the right-hand
    side, the operator) follow the chosen outcomes, and those sums compare
    with no allowance for flagged samples.  Returns (flagged, flipped,
    worst score of the chosen outcomes)."""
    orc.clear_flips()
    rgb_ref, resid_ref, flags = orc.render_samples()
    fl = np.nonzero(flags)[0].astype(np.int64)
    if len(fl) == 0:
        return 0, 0, 0.0
    tgt = rgb_ref[fl] - resid_ref[fl]
    _, rgb_m, u_m = orc.sample_outcomes(np.asarray(v, np.float64), fl, max_bits)
    u_floor = JV_TOL * np.sqrt(np.mean(np.asarray(u_dev, np.float64) ** 2))
    e_r = np.abs(resid_dev[fl][:, None, :] - (rgb_m - tgt[:, None, :])).max(axis=2) / PIX_TOL
    e_u = np.abs(u_dev[fl][:, None, :] - u_m).max(axis=2) / (JV_TOL * np.abs(u_m).max(axis=2) + u_floor)
    score = np.maximum(e_r, e_u)
    score[np.isnan(score)] = np.inf  # masks beyond the sample's near decisions
    best = np.argmin(score, axis=1).astype(np.uint32)  # ties: the lowest mask (mask 0 = the oracle's own)
    orc.set_flips(fl, best)
    return len(fl), int((best != 0).sum()), float(score[np.arange(len(fl)), best].max())


def assert_groups_close(pair, got, ref, tol):
    """Per parameter group: |got - ref| <= tol max(|ref|, 1e-3 |ref_total|)."""
    g, r = pair.groups(got), pair.groups(ref)
    tot = np.linalg.norm(ref)
    for k in GROUPS:
        err = np.linalg.norm(g[k] - r[k])
        allow = tol * max(np.linalg.norm(r[k]), 1e-3 * tot)
        assert err <= allow, f"{k}: {err:.3e} > {allow:.3e}"
