"""Direction shards: one transport problem split over several contexts.

L^-1 is block-diagonal in angle (Sec. 4.2), so the directions of a problem
can be divided among contexts, one per GPU, each created with its own subset
of ordinates and weights.  The shards exchange only sums (the angular
reduction D and the step-residual norms), through the cross-shard sum
callback of the C ABI (mlpg_set_reduce); the outer scattering solve is
replicated on identical data.  This module plans the split and provides two
sums: across torch.distributed ranks (one process per GPU; the gloo backend
moves the host buffer) and across threads of one process (several shards of
one problem on one device, each stepped by its own thread; the threads meet
at a barrier on the host, never inside a kernel).
"""
from __future__ import annotations

import threading

import numpy as np

from . import REDUCE_FN, TransportProblem, mlpg_set_reduce


def split_directions(m: int, shards: int):
    """Contiguous, balanced split of m directions over `shards` shards: the
    index array of each (sizes differ by at most one; none empty)."""
    if not 1 <= shards <= m:
        raise ValueError(f"cannot split {m} directions over {shards} shards")
    base, extra = divmod(m, shards)
    out, k = [], 0
    for r in range(shards):
        c = base + (1 if r < extra else 0)
        out.append(np.arange(k, k + c))
        k += c
    return out


def _view(buf, count):
    return np.ctypeslib.as_array(buf, shape=(int(count),))


def torch_reducer(group=None):
    """A REDUCE_FN summing the host buffer over the ranks of a
    torch.distributed process group (a CPU-capable backend such as gloo)."""
    import torch
    import torch.distributed as dist

    def fn(buf, count, user):
        try:
            t = torch.from_numpy(_view(buf, count))     # shares the library's host buffer
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return 0
        except Exception:
            return 1
    return REDUCE_FN(fn)


class ThreadReducer:
    """Sums over k shards of one process, each driven by its own thread: every
    shard deposits its partial sums, waits at a barrier (with a timeout, so
    that a shard that failed cannot hang the others), and reads the total."""

    def __init__(self, shards: int, timeout: float = 120.0):
        self.k = shards
        self.timeout = timeout
        self.barrier = threading.Barrier(shards)
        self.lock = threading.Lock()
        self.parts = {}
        self.callbacks = [REDUCE_FN(self._make(r)) for r in range(shards)]

    def _make(self, rank):
        def fn(buf, count, user):
            try:
                v = _view(buf, count)
                with self.lock:
                    self.parts[rank] = v.copy()
                self.barrier.wait(self.timeout)          # every partial is in
                total = np.sum([self.parts[r] for r in range(self.k)], axis=0)
                self.barrier.wait(self.timeout)          # every shard has read them
                v[:] = total
                return 0
            except threading.BrokenBarrierError:
                return 1
        return fn


class ShardedProblem:
    """One problem as `shards` contexts (directions split by
    split_directions), stepped concurrently by one thread each on this
    process's device.  Returns the same scalar flux as the unsplit problem."""

    def __init__(self, prob, shards: int, **options):
        self.parts = split_directions(prob.m, shards)
        self.reducer = ThreadReducer(shards)
        self.tps = []
        try:
            for r, idx in enumerate(self.parts):
                tp = TransportProblem(prob.x, prob.R, prob.omega[idx], prob.w[idx], prob.sigma_t, prob.sigma_s,
                                      prob.q, inflow=prob.inflow, lo=tuple(prob.lo), hi=tuple(prob.hi), **options)
                mlpg_set_reduce(tp.ctx, self.reducer.callbacks[r])
                self.tps.append(tp)
            self._each(lambda tp: tp.integrate().assemble())
        except Exception:
            self.close()
            raise

    def _each(self, f):
        errs = [None] * len(self.tps)

        def run(r):
            try:
                f(self.tps[r])
            except Exception as e:         # the barrier timeout releases the others
                errs[r] = e
                self.reducer.barrier.abort()
        th = [threading.Thread(target=run, args=(r,)) for r in range(len(self.tps))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for e in errs:
            if e is not None:
                raise e

    def step(self, dt):
        self._each(lambda tp: tp.step(dt))

    def run(self, dt, steps):
        for _ in range(steps):
            self.step(dt)
        return self.scalar_flux()

    def scalar_flux(self, kind=0):
        return self.tps[0].scalar_flux(kind)

    def state(self):
        """The angular flux [n][m] gathered from the shards in direction order."""
        return np.concatenate([tp.state() for tp in self.tps], axis=1)

    def close(self):
        for tp in self.tps:
            tp.close()
        self.tps = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


__all__ = ["split_directions", "torch_reducer", "ThreadReducer", "ShardedProblem"]
