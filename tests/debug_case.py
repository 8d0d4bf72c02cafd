"""The computation the bounds-checked build is run on (tests/test_gpu_debug_build.py):
the ragged 100x70 scene at SH1, 25% sampling, through every kernel that takes
indexes from the lists (the forward render and its compact lists, J v, J^T u,
the right-hand side, the diagonal, the fused operator, two LM steps).  Returns
the results and the scene's debug word after each stage."""
import numpy as np


def run():
    import torch

    from paper_2504_12905_gb300 import lmrs
    from paper_2504_12905_gb300 import synthetic as syn

    rng = np.random.default_rng(17)
    sc = syn.tiny_scene(seed=99, n_gauss=1500, width=100, height=70, sh_degree=1)
    tgt = torch.from_numpy(syn.noise_targets(rng, len(sc.cams), 70, 100)).cuda()
    s = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree, targets=tgt,
                   sample_frac=0.25, lambda_=0.1, damping_mode=0, cg_iters=8, seed=0x5EED)
    out, words = {}, {}
    s.preprocess([3, 1, 0], 5)
    S, P = s.n_samples, s.n_params

    def z(n):
        return torch.zeros(n, dtype=torch.float32, device="cuda")

    res = z(3 * S)
    lmrs.lmrs_render(s.h, None, res)
    words["render"] = lmrs.lmrs_debug_status(s.h)
    v = torch.from_numpy(np.random.default_rng(5).standard_normal(P).astype(np.float32)).cuda()
    u = z(3 * S)
    lmrs.lmrs_jvp(s.h, v, u)
    g, b, d, a = z(P), z(P), z(P), z(P)
    lmrs.lmrs_vjp(s.h, u, g)
    lmrs.lmrs_rhs(s.h, b)
    lmrs.lmrs_jtj_diag(s.h, d)
    lmrs.lmrs_jtjv(s.h, v, a)
    words["derivatives"] = lmrs.lmrs_debug_status(s.h)
    st = [lmrs.lmrs_lm_step(s.h, [3, 1, 0], 12), lmrs.lmrs_lm_step(s.h, [2, 0], 13)]
    words["lm_steps"] = lmrs.lmrs_debug_status(s.h)
    q = z(P)
    lmrs.lmrs_get_params(s.h, q)
    torch.cuda.synchronize()
    for name, t in (("residuals", res), ("jv", u), ("vjp", g), ("rhs", b), ("diag", d), ("operator", a),
                    ("params", q)):
        out[name] = t.cpu().numpy()
    out["losses"] = np.array([x.loss for x in st])
    s.close()
    return out, words
