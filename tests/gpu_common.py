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


def flagged_contribution(pair, v):
    """J^T W J v restricted to the samples the oracle flags as near one of the
    per-pixel compositing decisions (alpha >= 1/255, T < 1e-4 of Eq. 4): an
    FP32 evaluation may legitimately decide those differently, so their whole
    contribution bounds the extra difference they can cause."""
    _, _, flags = pair.orc.render_samples()
    w = pair.orc.samples()["w"]
    u = pair.orc.jvp(np.asarray(v, np.float64)) * (w * (flags != 0))[:, None]
    return pair.orc.vjp(u)


def assert_groups_close(pair, got, ref, tol, slack=None):
    """Per parameter group: |got - ref| <= tol max(|ref|, 1e-3 |ref_total|)
    + 2 |slack| (slack: a P-vector, e.g. flagged_contribution)."""
    g, r = pair.groups(got), pair.groups(ref)
    sl = pair.groups(slack) if slack is not None else None
    tot = np.linalg.norm(ref)
    for k in GROUPS:
        err = np.linalg.norm(g[k] - r[k])
        allow = tol * max(np.linalg.norm(r[k]), 1e-3 * tot) + (2.0 * np.linalg.norm(sl[k]) if sl else 0.0)
        assert err <= allow, f"{k}: {err:.3e} > {allow:.3e}"
