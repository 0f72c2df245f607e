"""The benchmark's multi-GPU bookkeeping on CPU: two gloo ranks (world size 2).

Each rank matches its own slice (weak scaling, no data-path collective); the
only cross-rank step is the max of the ranks' times, and the whole-job rate
counts every rank's voxels over that slowest time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank            # rank 1 is slower
    m = bench.reduce_max(ms, dist)
    rate = bench.whole_job_rate(world, 4096, m)
    q.put((rank, m, rate, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert out[0][2] == pytest.approx(2 * 4096 / 15.0 * 1e3)
    assert out[0][3] != out[1][3]     # distinct slices per rank


def test_single_process_needs_no_group():
    import bench
    assert bench.reduce_max(12.5, None) == 12.5
    assert bench.whole_job_rate(1, 4096, 40.0) == pytest.approx(102400.0)


def test_bench_starts_its_own_ranks():
    """`bench.py --gpus 2` without a launcher starts two ranks itself
    (torch.distributed.run on 127.0.0.1); the GPU-free dry run checks that
    both ranks join, and that rank 0 alone prints the line with n_gpus 2."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR",
                                                             "MASTER_PORT")}
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--dry-run", "--steps", "3",
                        "--warmup", "3"], capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert p.returncode == 0, p.stderr[-2000:]
    assert "rank 0 of 2 ready" in p.stderr and "rank 1 of 2 ready" in p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[-1])
    assert out["n_gpus"] == 2 and out["steps"] == 3 and out["dry_run"] is True
    assert out["value"] == pytest.approx(2 * 4096 / out["ms_per_step"] * 1e3)
