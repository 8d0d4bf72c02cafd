"""The multi-rank host logic of bench.py with two gloo ranks on CPU: the
ranks run as independent replicas and exchange only a barrier, the maximum
of their times and the sum of their counts."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    reps = bench.Replicas(rank, world, rank, backend="gloo")
    reps.barrier()
    ms = reps.max(10.0 + rank)           # the slowest rank's time
    done = reps.sum(3 + rank)            # rank-local counts
    rate = bench.job_rate(5, world, ms)  # 5 units per rank
    reps.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "done": done, "rate": rate}, f)


def test_two_gloo_replicas_agree_on_max_sum_and_rate(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["ms"] == 11.0
        assert r["done"] == 7.0
        assert r["rate"] == pytest.approx(2 * 5 / 0.011)


def test_single_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas(0, 1, 0)
    reps.barrier()
    assert reps.max(4.5) == 4.5 and reps.sum(3) == 3.0
    reps.close()
    assert bench.job_rate(8, 1, 500.0) == pytest.approx(16.0)


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-500:]
    assert r.stdout.strip() == ""
