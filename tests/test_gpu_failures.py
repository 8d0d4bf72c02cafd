"""Host-visible failure paths of the library, made on the host side: no
kernel faults, traps or hangs.

* Non-finite parameters (a NaN colour coefficient) make the PCG meet a
  non-finite r^T z / p^T A p: lmrs_lm_step returns LMRS_ERR_NUMERIC, the
  parameters are left as they were, and the scene steps again once it is
  given finite parameters; in a batch only the bad scene reports it.
* A device allocation larger than what is free (most of the device memory
  held by torch first) returns LMRS_ERR_OOM from lmrs_preprocess before any
  kernel runs; the same scene preprocesses and steps once memory is free.
* lmrs_server_wait with a zero timeout on a job still running returns
  LMRS_ERR_TIMEOUT, and a second wait sees the job finish."""
import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

LMRS_ERR_OOM = 2
LMRS_ERR_NUMERIC = 5
LMRS_ERR_TIMEOUT = 6


def _tiny(seed, nan=False):
    sc = syn.tiny_scene(seed=seed)
    p = sc.params.copy()
    if nan:
        # the red DC coefficient of every Gaussian: every rendered colour is NaN
        K3 = 3 * (sc.sh_degree + 1) ** 2
        p[11 * sc.n_gauss::K3] = np.nan
    rng = np.random.default_rng(seed)
    tgt = syn.noise_targets(rng, len(sc.cams), sc.height, sc.width)
    return sc, p, tgt


def _scene(lmrs, torch, sc, p, tgt):
    t = torch.from_numpy(tgt).cuda()
    return lmrs.Scene(torch.from_numpy(p).cuda(), sc.cams, sc.n_gauss, sc.sh_degree, targets=t, lambda_=1e-2,
                      damping_mode=1, cg_iters=4, seed=3)


def test_non_finite_parameters_give_numeric_and_no_update():
    import torch

    from paper_2504_12905_gb300 import lmrs
    sc, p_bad, tgt = _tiny(5, nan=True)
    s = _scene(lmrs, torch, sc, p_bad, tgt)
    views = [0, 1, 2, 3]
    with pytest.raises(lmrs.LmrsError) as e:
        lmrs.lmrs_lm_step(s.h, views, 0)
    assert e.value.status == LMRS_ERR_NUMERIC
    after = np.zeros(s.n_params, np.float32)
    lmrs.lmrs_get_params(s.h, after)
    np.testing.assert_array_equal(after, p_bad)  # NaN where they were, nothing else moved
    # the scene stays usable: finite parameters step normally
    _, p_ok, _ = _tiny(5)
    lmrs.lmrs_set_params(s.h, np.ascontiguousarray(p_ok))
    st = lmrs.lmrs_lm_step(s.h, views, 1)
    lmrs.lmrs_get_params(s.h, after)
    assert np.isfinite(st.loss) and st.eta == pytest.approx(0.05) and np.isfinite(after).all()
    assert np.abs(after - p_ok).max() > 0.0
    s.close()


def test_batch_reports_numeric_for_the_bad_scene_only():
    import torch

    from paper_2504_12905_gb300 import lmrs
    good = _tiny(6)
    bad = _tiny(7, nan=True)
    scenes = [_scene(lmrs, torch, *good), _scene(lmrs, torch, *bad)]
    B = lmrs.lmrs_batch_create([s.h for s in scenes], n_threads=2)
    try:
        with pytest.raises(lmrs.LmrsError) as e:
            lmrs.lmrs_batch_lm_step(B, [[0, 1, 2, 3], [0, 1, 2, 3]], [0, 0])
        assert e.value.status == LMRS_ERR_NUMERIC
        assert lmrs.lmrs_batch_scene_status(B, 0) == lmrs.LMRS_OK
        assert lmrs.lmrs_batch_scene_status(B, 1) == LMRS_ERR_NUMERIC
    finally:
        lmrs.lmrs_batch_destroy(B)
    p0 = np.zeros(scenes[0].n_params, np.float32)
    p1 = np.zeros(scenes[1].n_params, np.float32)
    lmrs.lmrs_get_params(scenes[0].h, p0)
    lmrs.lmrs_get_params(scenes[1].h, p1)
    assert np.isfinite(p0).all() and np.abs(p0 - good[1]).max() > 0.0  # the good scene stepped
    np.testing.assert_array_equal(p1, bad[1])  # the bad one did not move
    for s in scenes:
        s.close()


def test_device_allocation_failure_is_oom_and_the_scene_recovers():
    import torch

    from paper_2504_12905_gb300 import lmrs
    # 1M Gaussians (SH0): creating the scene takes ~0.6 GB; one LM step over
    # 8 views of 1024 x 672 needs a few GB more (~400 B per (view, Gaussian)
    # pair plus the tile lists)
    rng = np.random.default_rng(9)
    G = 1_000_000
    params = syn.draw_gaussians(rng, G, 0, means=syn.blob_means(rng, G, n_blobs=8))
    cams = syn.hemisphere_cameras(8, 3.0, 1024, 672)
    s = lmrs.Scene(torch.from_numpy(params).cuda(), cams, G, 0, sample_frac=0.1, lambda_=0.1, damping_mode=0,
                   cg_iters=2)
    views = list(range(8))
    torch.cuda.synchronize()
    held = []
    try:
        # hold all but ~2 GB of the free device memory
        free, _ = torch.cuda.mem_get_info()
        while free > (3 << 30):
            held.append(torch.empty(min(8 << 30, free - (2 << 30)), dtype=torch.uint8, device="cuda"))
            free, _ = torch.cuda.mem_get_info()
        with pytest.raises(lmrs.LmrsError) as e:
            s.preprocess(views, 0)
        assert e.value.status == LMRS_ERR_OOM, e.value
    finally:
        del held
        torch.cuda.empty_cache()
    s.preprocess(views, 0)  # the same scene, now with room
    assert s.n_pairs > 0
    st = lmrs.lmrs_lm_step(s.h, views, 0)
    assert np.isfinite(st.loss)
    s.close()


def test_server_wait_times_out_then_sees_the_job_finish():
    from paper_2504_12905_gb300 import lmrs
    rng = np.random.default_rng(13)
    G = 4000
    params = syn.draw_gaussians(rng, G, 1, means=syn.blob_means(rng, G, n_blobs=4))
    cams = syn.hemisphere_cameras(8, 3.0, 128, 128)
    tgt = syn.noise_targets(rng, 8, 128, 128)
    cfg = lmrs.lmrs_config_default(sh_degree=1, samples_per_tile=32, lambda_=0.1, damping_mode=0, cg_iters=4, seed=1)
    srv = lmrs.lmrs_server_create(8 << 30, max_active=4, setup_threads=2)
    try:
        jid = lmrs.lmrs_server_submit(srv, cfg, G, params, cams, tgt, views_per_step=8, max_steps=30)
        status, info = lmrs.lmrs_server_wait(srv, jid, 0.0)
        assert status == LMRS_ERR_TIMEOUT and info.state not in (lmrs.JOB_DONE, lmrs.JOB_FAILED)
        status, info = lmrs.lmrs_server_wait(srv, jid, 180.0)
        assert status == lmrs.LMRS_OK and info.state == lmrs.JOB_DONE and info.steps == 30
    finally:
        lmrs.lmrs_server_destroy(srv)
