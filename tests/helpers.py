"""Shared helpers for the tests: small seeded scenes and dense Jacobians from
the oracle."""
from __future__ import annotations

import numpy as np

from paper_2504_12905_gb300 import synthetic as syn


def small_scene(seed, n_gauss=6, sh_degree=0, n_views=2, size=32, spread=0.3, log_scale=-1.5,
                sh_high=0.3):
    """A handful of large Gaussians near the origin, seen by ``n_views``
    ring cameras; colours kept away from the clamp at 0."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, (n_gauss, 3))
    ls = rng.normal(log_scale, 0.2, (n_gauss, 3))
    q = rng.standard_normal((n_gauss, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.normal(0.0, 1.0, n_gauss)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n_gauss, K, 3))
    sh[:, 0, :] = rng.uniform(-0.8, 0.8, (n_gauss, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_high / K, (n_gauss, K - 1, 3))
    params = syn.pack_params(means, ls, q, opac, sh)
    cams = syn.ring_cameras(n_views, 3.0, size, size, elev_deg=20.0)
    return syn.Scene(n_gauss, sh_degree, params, cams, seed)


def fd_jacobian(osc, views, h=1e-6, step=0):
    """Central-difference Jacobian of the sampled residual vector (rows
    (sample, channel)) with respect to every parameter."""
    base = osc.get_params()
    osc.begin_step(views, step)
    S = osc.n_samples
    J = np.zeros((3 * S, base.size))
    for j in range(base.size):
        p = base.copy()
        p[j] += h
        osc.set_params(p)
        osc.begin_step(views, step)
        up, _, _ = osc.render_samples()
        p[j] -= 2 * h
        osc.set_params(p)
        osc.begin_step(views, step)
        dn, _, _ = osc.render_samples()
        J[:, j] = (up - dn).reshape(-1) / (2 * h)
    osc.set_params(base)
    osc.begin_step(views, step)
    return J


def jvp_jacobian(osc):
    """Dense Jacobian assembled column by column from the oracle's JVP."""
    P = osc.n_params
    J = np.zeros((3 * osc.n_samples, P))
    e = np.zeros(P)
    for j in range(P):
        e[:] = 0.0
        e[j] = 1.0
        J[:, j] = osc.jvp(e).reshape(-1)
    return J


def normwise_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)
