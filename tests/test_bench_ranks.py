"""The multi-rank aggregation of bench.py on two gloo ranks (CPU, no GPU): each
rank solves its own problems (weak scaling, no data-path collective); the
job's time is the slowest rank's, for the device-timed value and for the
end-to-end value alike, and the job rate counts every rank's solves."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench._max_over_ranks(1.0 + rank, world, "cpu")    # rank 1 is slower here
        e = bench._max_over_ranks(3.0 - rank, world, "cpu")    # rank 0 is slower here
        out.put((rank, t, e, bench._job_rate(world, 3, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r[0] for r in res] == [0, 1]
    for rank, t, e, rate in res:
        assert t == 2.0 and e == 3.0                     # both ranks see the slowest rank
        assert rate == pytest.approx(2 * 3 / 2.0)        # 2 ranks x 3 solves in 2 s


def test_one_rank_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(2.5, 1) == 2.5
    assert bench._job_rate(1, 4, 2.0) == 2.0


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun with two ranks, rank 1 of the reference arm exits 0 without work
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
