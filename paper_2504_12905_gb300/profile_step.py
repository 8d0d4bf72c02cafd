"""Runs LM steps of a named synthetic workload, for profilers.

    python -m paper_2504_12905_gb300.profile_step --workload moderate --steps 1

Workloads (seeded, as in the benchmark; the targets are uniform noise, which
does not change the work of a step):
  tiny      1,000 Gaussians, SH0, 4 views 64x64, all pixels, 10 PCG iterations
  moderate  200k Gaussians, SH3, 8 of 24 views 1024x672, 10% per tile, 8 PCG iterations
  large     1.5M Gaussians, SH3, 12 of 100 views 1297x840, 25% per tile, BF16 caches, 8 PCG iterations
"""
from __future__ import annotations

import argparse

import numpy as np

WORKLOADS = {
    "tiny": dict(make="tiny_scene", views=4, cfg=dict(sample_frac=1.0, cg_iters=10, lambda_=1e-2, damping_mode=0)),
    "moderate": dict(make="moderate_scene", views=8,
                     cfg=dict(sample_frac=0.1, cg_iters=8, lambda_=0.1, damping_mode=0)),
    "large": dict(make="large_scene", views=12,
                  cfg=dict(sample_frac=0.25, cg_iters=8, lambda_=0.1, damping_mode=0, cache_bf16=1)),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="moderate")
    ap.add_argument("--steps", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    from . import lmrs
    from . import synthetic as syn

    wl = WORKLOADS[args.workload]
    sc = getattr(syn, wl["make"])()
    rng = np.random.default_rng(1)
    nc = len(sc.cams)
    targets = torch.from_numpy(syn.noise_targets(rng, nc, sc.height, sc.width)).cuda()
    scene = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree, targets=targets,
                       seed=0x5EED, **wl["cfg"])
    vr = np.random.default_rng(77)
    for k in range(args.steps):
        st = lmrs.lmrs_lm_step(scene.h, syn.view_subset(vr, nc, min(wl["views"], nc)), k)
        print(f"step {k}: loss {st.loss:.6g} eta {st.eta:.4g} samples {st.n_samples} entries {st.n_pairs}")
    torch.cuda.synchronize()
    scene.close()


if __name__ == "__main__":
    main()
