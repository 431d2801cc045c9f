"""Host logic of direction shards (no GPU): the split of the directions, the
cross-shard sum over two gloo ranks called through the C-ABI callback type,
and the thread-level sum that several shards of one process use.

L^-1 is block-diagonal in angle (Sec. 4.2), so a problem's directions can be
divided among contexts; the shards then exchange only sums (the angular
reduction D and the residual norms)."""
import ctypes
import os
import socket
import threading

import numpy as np
import pytest

from paper_2008_02205_gb300 import REDUCE_FN
from paper_2008_02205_gb300.shard import ThreadReducer, split_directions


def _call(cb, arr):
    """Call a REDUCE_FN through its C function pointer, as the library does."""
    f = ctypes.cast(cb, REDUCE_FN)
    return f(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), arr.size, None)


@pytest.mark.parametrize("m,k", [(40, 2), (40, 3), (12, 5), (272, 8), (7, 7)])
def test_split_covers_every_direction_once(m, k):
    parts = split_directions(m, k)
    assert len(parts) == k and all(len(p) > 0 for p in parts)
    assert np.array_equal(np.concatenate(parts), np.arange(m))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        split_directions(m, m + 1)


def test_thread_reducer_sums_every_shard():
    k, n = 3, 17
    red = ThreadReducer(k, timeout=20.0)
    out, rcs = [None] * k, [None] * k

    def run(r):
        arr = np.arange(n, dtype=np.float64) * (r + 1)
        got = []
        for _ in range(3):                  # repeated sums reuse the barrier
            rcs[r] = _call(red.callbacks[r], arr)
            got.append(arr.copy())
            arr = arr * (r + 1)
        out[r] = got
    th = [threading.Thread(target=run, args=(r,)) for r in range(k)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert rcs == [0, 0, 0]
    i = np.arange(n, dtype=np.float64)
    # sum 1: i (1 + 2 + 3); sum 2: 6i (1 + 2 + 3); sum 3: 36i (1 + 2 + 3)
    for r in range(k):
        assert np.array_equal(out[r][0], 6.0 * i)
        assert np.array_equal(out[r][1], 36.0 * i)
        assert np.array_equal(out[r][2], 216.0 * i)


def test_thread_reducer_gives_up_when_a_shard_is_missing():
    red = ThreadReducer(2, timeout=0.5)
    assert _call(red.callbacks[0], np.ones(3)) == 1     # the other shard never arrives


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
        from paper_2008_02205_gb300.shard import torch_reducer
        cb = torch_reducer()
        a = np.full(9, rank + 1.0)
        rc1 = _call(cb, a)
        b = np.array([float(rank)])
        rc2 = _call(cb, b)
        out.put((rank, rc1, a.tolist(), rc2, b.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_through_the_callback():
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
    for rank, rc1, a, rc2, b in res:
        assert rc1 == 0 and rc2 == 0
        assert a == [3.0] * 9 and b == [1.0]
