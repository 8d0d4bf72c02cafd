"""Batched LM steps (all scenes' PCG iterations in one launch per phase,
replayed as a CUDA graph) against solo LM steps of the same scenes and
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2504_12905_gb300 import synthetic as syn

from helpers import normwise_rel

pytestmark = pytest.mark.gpu


def _scenes(n=5, seed=23):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        G = int(rng.integers(300, 2500))
        nv = int(rng.integers(2, 6))
        size = int(rng.choice([48, 64, 80]))
        sub = np.random.default_rng([seed, i])
        params = syn.draw_gaussians(sub, G, 0, means=syn.blob_means(sub, G, n_blobs=4))
        cams = syn.hemisphere_cameras(nv, 3.0, size, size)
        tgt = syn.noise_targets(sub, nv, size, size)
        out.append((syn.Scene(G, 0, params, cams, i), tgt))
    return out


def _make(torch, lmrs, sc, tgt, stream, **extra):
    t = torch.from_numpy(tgt).cuda()
    s = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, 0, targets=t, stream=stream,
                   samples_per_tile=32, lambda_=0.1, damping_mode=0, cg_iters=8, seed=0x5EED, **extra)
    s._t = t
    return s


def test_persistent_launch_matches_the_graph_of_phases():
    """The persistent cooperative launch (every phase of every PCG
    iteration, grid barriers between them) against the graph of per-phase
    launches on the same scenes, and both against the scenes' own solo
    steps.  Two steps (12 and 13: the graph form's second one replays the
    captured graph), each from the same starting parameters in every run, so
    that the runs differ only in the summation order of the float atomics
    (blocks arrive in any order), not in inputs that an earlier step already
    moved apart: these small fits amplify a last-bit difference in their
    parameters by 40x and more in the next step's solve.  The spread of two
    graph runs is printed beside the difference of the two forms."""
    import torch

    from paper_2504_12905_gb300 import lmrs

    scenes = _scenes(n=6, seed=31)
    views = [list(range(len(sc.cams))) for sc, _ in scenes]
    start = [np.ascontiguousarray(sc.params, np.float32) for sc, _ in scenes]
    runs = []
    for mode in (0, 0, 1):
        streams = [torch.cuda.Stream() for _ in scenes]
        sc_b = [_make(torch, lmrs, sc, tgt, streams[i].cuda_stream) for i, (sc, tgt) in enumerate(scenes)]
        b = lmrs.lmrs_batch_create([s.h for s in sc_b], n_threads=3)
        lmrs.lmrs_batch_set_persistent(b, mode)
        out = []
        for step in (12, 13):
            for s, x0 in zip(sc_b, start):
                lmrs.lmrs_set_params(s.h, x0)
            st = lmrs.lmrs_batch_lm_step(b, views, [step] * len(scenes))
            xs = []
            for s in sc_b:
                x = np.zeros(s.n_params, np.float32)
                lmrs.lmrs_get_solution(s.h, x)
                xs.append(x)
            out.append((st, xs))
        lmrs.lmrs_batch_destroy(b)
        for s in sc_b:
            s.close()
        runs.append(out)
    solo = [_make(torch, lmrs, sc, tgt, None) for sc, tgt in scenes]
    for k, step in enumerate((12, 13)):
        (st0, x0), (_, xg), (st1, x1) = runs[0][k], runs[1][k], runs[2][k]
        spread = max(normwise_rel(xg[i], x0[i]) for i in range(len(scenes)))
        diff = max(normwise_rel(x1[i], x0[i]) for i in range(len(scenes)))
        print(f"step {step}: persistent vs graph {diff:.2e}, graph vs graph {spread:.2e}")
        for i, s in enumerate(solo):
            lmrs.lmrs_set_params(s.h, start[i])
            st = lmrs.lmrs_lm_step(s.h, views[i], step)
            xs = np.zeros(s.n_params, np.float32)
            lmrs.lmrs_get_solution(s.h, xs)
            assert normwise_rel(x1[i], x0[i]) <= 1e-4, (step, i)
            assert normwise_rel(x1[i], xs) <= 1e-3, (step, i)
            assert st1[i].loss == pytest.approx(st0[i].loss, rel=1e-6)
            assert st1[i].eta == pytest.approx(st.eta, rel=1e-4)
            assert st1[i].rz0 == pytest.approx(st0[i].rz0, rel=1e-6)
    for s in solo:
        s.close()


def test_grid_barrier_wait_runs_out_and_the_device_stays_usable():
    """The persistent launch's grid barrier: a launch whose barrier expects
    one block more than it has cannot complete; every wait runs out after
    the timeout and the call reports LMRS_ERR_TIMEOUT.  A complete barrier
    passes before and after, on the same device."""
    import time

    from paper_2504_12905_gb300 import lmrs
    assert lmrs.lmrs_grid_barrier_selftest(0, 1.0) == lmrs.LMRS_OK
    t0 = time.perf_counter()
    assert lmrs.lmrs_grid_barrier_selftest(1, 0.25) == 6  # LMRS_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.2
    assert lmrs.lmrs_grid_barrier_selftest(0, 1.0) == lmrs.LMRS_OK


def test_batch_matches_solo_steps_and_oracle():
    import torch

    from paper_2504_12905_gb300 import lmrs

    scenes = _scenes()
    streams = [torch.cuda.Stream() for _ in scenes]
    batch_sc = [_make(torch, lmrs, sc, tgt, streams[i].cuda_stream) for i, (sc, tgt) in enumerate(scenes)]
    solo_sc = [_make(torch, lmrs, sc, tgt, None) for sc, tgt in scenes]
    b = lmrs.lmrs_batch_create([s.h for s in batch_sc], n_threads=3)
    views = [list(range(len(sc.cams))) for sc, _ in scenes]
    for step in (10, 11):  # two steps: the second replays the captured graph
        st_b = lmrs.lmrs_batch_lm_step(b, views, [step] * len(scenes))
        for i, s in enumerate(solo_sc):
            st = lmrs.lmrs_lm_step(s.h, views[i], step)
            xs = np.zeros(s.n_params, np.float32)
            xb = np.zeros(s.n_params, np.float32)
            lmrs.lmrs_get_solution(s.h, xs)
            lmrs.lmrs_get_solution(batch_sc[i].h, xb)
            assert normwise_rel(xb, xs) <= 1e-3, (step, i)
            assert st_b[i].eta == pytest.approx(st.eta, rel=1e-4)
            assert st_b[i].loss == pytest.approx(st.loss, rel=1e-6)
            assert st_b[i].rz0 == pytest.approx(st.rz0, rel=1e-5)
            pb = np.zeros(s.n_params, np.float32)
            ps = np.zeros(s.n_params, np.float32)
            lmrs.lmrs_get_params(batch_sc[i].h, pb)
            lmrs.lmrs_get_params(s.h, ps)
            assert normwise_rel(pb - scenes[i][0].params, ps - scenes[i][0].params) <= 1e-3
    # the first batch step of scene 0 against the FP64 oracle (A-norm, as for solo steps)
    sc, tgt = scenes[0]
    fresh = _make(torch, lmrs, sc, tgt, streams[0].cuda_stream)
    b1 = lmrs.lmrs_batch_create([fresh.h], n_threads=1)
    lmrs.lmrs_batch_lm_step(b1, [views[0]], [10])
    x = np.zeros(fresh.n_params, np.float32)
    lmrs.lmrs_get_solution(fresh.h, x)
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, 0, targets=tgt, samples_per_tile=32, lambda_=0.1,
                           damping_mode=0, cg_iters=8, seed=0x5EED)
    o.begin_step(views[0], 10)
    D = o.diag()
    x_ref, _ = o.lm_step(views[0], 10)
    o.set_params(sc.params.astype(np.float64))
    o.begin_step(views[0], 10)
    e = x.astype(np.float64) - x_ref
    a_norm = np.sqrt(max(e @ o.apply(e, D), 0.0)) / np.sqrt(x_ref @ o.apply(x_ref, D))
    assert a_norm <= 1e-3
    lmrs.lmrs_batch_destroy(b1)
    lmrs.lmrs_batch_destroy(b)


def test_batch_with_the_ssim_term_matches_solo():
    import torch

    from paper_2504_12905_gb300 import lmrs

    scenes = _scenes(3, seed=31)
    streams = [torch.cuda.Stream() for _ in scenes]
    batch_sc = [_make(torch, lmrs, sc, tgt, streams[i].cuda_stream, ssim_weight=0.2)
                for i, (sc, tgt) in enumerate(scenes)]
    solo_sc = [_make(torch, lmrs, sc, tgt, None, ssim_weight=0.2) for sc, tgt in scenes]
    b = lmrs.lmrs_batch_create([s.h for s in batch_sc], n_threads=2)
    views = [list(range(len(sc.cams))) for sc, _ in scenes]
    st_b = lmrs.lmrs_batch_lm_step(b, views, [3] * len(scenes))
    for i, s in enumerate(solo_sc):
        st = lmrs.lmrs_lm_step(s.h, views[i], 3)
        xs = np.zeros(s.n_params, np.float32)
        xb = np.zeros(s.n_params, np.float32)
        lmrs.lmrs_get_solution(s.h, xs)
        lmrs.lmrs_get_solution(batch_sc[i].h, xb)
        assert normwise_rel(xb, xs) <= 1e-3, i
        assert st_b[i].loss == pytest.approx(st.loss, rel=1e-6)
    lmrs.lmrs_batch_destroy(b)


def test_batch_rejects_mixed_configs():
    import torch

    from paper_2504_12905_gb300 import lmrs

    (sc, tgt), = _scenes(1)
    a = _make(torch, lmrs, sc, tgt, None)
    b = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, 0, cg_iters=5)
    with pytest.raises(lmrs.LmrsError):
        lmrs.lmrs_batch_create([a.h, b.h])
    with pytest.raises(lmrs.LmrsError):
        lmrs.lmrs_batch_create([a.h, a.h])


def test_autotune_tile_times_every_shape():
    import torch

    from paper_2504_12905_gb300 import lmrs

    (sc, tgt), = _scenes(1, seed=5)
    params = torch.from_numpy(sc.params).cuda()
    t = torch.from_numpy(tgt).cuda()
    cfg = lmrs.lmrs_config_default(sh_degree=0, samples_per_tile=32, lambda_=0.1, damping_mode=0, cg_iters=4)
    shapes = [(16, 16), (32, 8), (8, 32), (8, 8)]
    views = list(range(len(sc.cams)))
    best, ms = lmrs.lmrs_autotune_tile(cfg, sc.n_gauss, params, sc.cams, t, views, shapes, reps=2)
    assert 0 <= best < len(shapes)
    assert (ms > 0).all() and ms[best] == ms.min()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(params.cpu().numpy(), sc.params)  # the caller's parameters are untouched
    with pytest.raises(lmrs.LmrsError):
        lmrs.lmrs_autotune_tile(cfg, sc.n_gauss, params, sc.cams, t, views, [(32, 16)], reps=1)


def test_full_batch_of_64_scenes_against_oracle_on_sampled_scenes():
    """The benchmarked batch at full size (64 scenes of 5k-50k Gaussians,
    4-16 views of 256x256, 32 samples per tile, the benchmark's seeds and
    tile shape; seeded noise targets): one batched LM step of all 64 scenes,
    then the solutions of the smallest, the median and the largest scene
    against the oracle's LM step, in the A-norm, and their losses."""
    import torch

    from paper_2504_12905_gb300 import lmrs

    scenes = syn.small_fit_scenes()
    prng = np.random.default_rng(4321)
    starts = [syn.perturb(prng, sc.params) for sc in scenes]
    trng = np.random.default_rng(6)
    tgts = [syn.noise_targets(trng, len(sc.cams), sc.height, sc.width) for sc in scenes]
    cfg = dict(samples_per_tile=32, lambda_=0.1, damping_mode=0, cg_iters=8, seed=0x5EED, tile_w=16, tile_h=16)
    streams = [torch.cuda.Stream() for _ in scenes]
    gpu = []
    for i, sc in enumerate(scenes):
        t = torch.from_numpy(tgts[i]).cuda()
        s = lmrs.Scene(torch.from_numpy(starts[i]).cuda(), sc.cams, sc.n_gauss, 0, targets=t,
                       stream=streams[i].cuda_stream, **cfg)
        s._t = t
        gpu.append(s)
    b = lmrs.lmrs_batch_create([s.h for s in gpu], n_threads=4)
    views = [list(range(len(sc.cams))) for sc in scenes]
    st = lmrs.lmrs_batch_lm_step(b, views, [10] * len(scenes))
    order = np.argsort([sc.n_gauss for sc in scenes])
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        sc = scenes[i]
        x = np.zeros(gpu[i].n_params, np.float32)
        lmrs.lmrs_get_solution(gpu[i].h, x)
        o = oracle.OracleScene(starts[i], sc.cams, sc.n_gauss, 0, targets=tgts[i], **cfg)
        o.begin_step(views[i], 10)
        D = o.diag()
        x_ref, st_ref = o.lm_step(views[i], 10)
        o.set_params(starts[i].astype(np.float64))
        o.begin_step(views[i], 10)
        e = x.astype(np.float64) - x_ref
        a_norm = np.sqrt(max(e @ o.apply(e, D), 0.0)) / np.sqrt(x_ref @ o.apply(x_ref, D))
        assert a_norm <= 1e-3, (i, sc.n_gauss, a_norm)
        assert st[i].loss == pytest.approx(st_ref[0], rel=1e-5)
    lmrs.lmrs_batch_destroy(b)
    for s in gpu:
        s.close()
