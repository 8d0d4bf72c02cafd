"""lmrs_step_size_noalloc: the step-size entry point for callers that cannot
call cudaMalloc (their device memory belongs to another allocator, or an
allocation would stall a latency-critical loop).  It keeps its scratch in a
static device array; this checks it against lmrs_step_size on two calls in a
row, so a result left in the shared scratch by the first call would show in
the second.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_2504_12905_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_noalloc_step_size_matches_scene_entry_point():
    import torch

    from paper_2504_12905_gb300 import lmrs

    assert torch.cuda.is_available()
    G, deg = 50_000, 1  # 25 blocks of 2048 Gaussians, ragged last block
    rng = np.random.default_rng(11)
    params = syn.draw_gaussians(rng, G, deg)
    cams = syn.ring_cameras(2, 3.0, 64, 64)
    cfg = dict(lr_warm=0.05, lr_cap=0.2, color_bound=1.0, warm_iters=10)
    scene = lmrs.Scene(torch.from_numpy(params).cuda(), cams, G, deg, **cfg)
    P = scene.n_params
    dc0 = 11 * G
    K3 = 3 * (deg + 1) ** 2
    # first call: a large colour entry near the end; second call: everything
    # smaller, so a stale maximum from the first call would give a wrong eta
    for call, (scale, spike) in enumerate([(3.0, 40.0), (2.0, 0.0)]):
        x = rng.normal(0.0, scale, P).astype(np.float32)
        if spike:
            x[dc0 + (G - 7) * K3 + 2] = -spike
        xd = torch.from_numpy(x).cuda()
        for step in (3, 12):
            ref = lmrs.lmrs_step_size(scene.h, xd, step)
            got = lmrs.lmrs_step_size_noalloc(xd, G, deg, step, **cfg)
            assert got == pytest.approx(ref, rel=1e-12, abs=0.0), (call, step, got, ref)
        m = float(np.abs(x[dc0:].reshape(G, K3)[:, :3]).max())
        assert got == pytest.approx(min(0.2, 1.0 / m), rel=1e-12)
        # the same call on a stream of the caller's (a torch stream)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        got_s = lmrs.lmrs_step_size_noalloc(xd, G, deg, 12, stream=side, **cfg)
        assert got_s == pytest.approx(ref, rel=1e-12, abs=0.0), (call, got_s, ref)
    scene.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2504_12905_gb300 import lmrs

    x = torch.zeros(16, device="cuda")
    with pytest.raises(lmrs.LmrsError) as e:
        lmrs.lmrs_step_size_noalloc(x, 8_388_609, 0, 12, 0.05, 0.2, 1.0, 10)
    assert e.value.status == 7  # LMRS_ERR_BUDGET
    with pytest.raises(lmrs.LmrsError) as e:
        lmrs.lmrs_step_size_noalloc(x, 10, 4, 12, 0.05, 0.2, 1.0, 10)
    assert e.value.status == 1
