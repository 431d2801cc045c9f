"""Continuous-batching serving loop over independent transport problems.

Requests (a point set, its quadrature and materials, a number of backward-
Euler steps) arrive over time.  The loop admits arrived requests in order
while the device memory they are estimated to need fits the budget and a
slot is free, keeps every admitted problem's operators and flux state
resident on the device, and advances all admitted problems together: each
iteration is one ``mlpg_step_batch`` call, which steps every context on its
own stream so that their kernels overlap.  Admitted requests are set up
(integration and assembly on their own streams) by a background thread, so
that the resident problems keep stepping meanwhile.  A problem leaves as soon as its
last step is done (its memory and slot go to the next arrivals), with its
latency measured from its arrival.  A problem that cannot be set up, or whose
step fails (an iteration cap, say), leaves with its error and its memory
freed; the others carry on, since the batched call reports each context's own
status.  All compute goes through the C ABI; this module only schedules.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    problem: object             # an mlpg_inputs.Problem (or anything the backend accepts)
    steps: int
    dt: float
    arrival: float = 0.0        # seconds after the start of the run
    options: dict = field(default_factory=dict)


@dataclass
class Result:
    request: Request
    flux: np.ndarray | None = None
    device_bytes: int | None = None   # device memory the problem held at its last step (when known)
    admitted: float = 0.0
    finished: float = 0.0
    error: str | None = None

    @property
    def latency(self):
        return self.finished - self.request.arrival


def estimate_bytes(problem, precision_mixed: bool = True, restart: int = 20) -> int:
    """Device memory of one problem, from its size: the overlap pattern (mean
    row length from the kernel extents), the integrated forms, the operator
    arrays, the materialised FP64 operator, the block inverses and the Krylov
    vectors.  An admission estimate, not an allocation count."""
    x = np.asarray(problem.x)
    n, dim = x.shape
    m = len(problem.w)
    R = float(np.mean(problem.R))
    ball = math.pi * (2 * R) ** 2 if dim == 2 else 4.0 / 3.0 * math.pi * (2 * R) ** 3
    nnz = n * min(n, max(1.0, ball * n))
    nmats = 3 + 3 * dim + dim * dim + 2 * dim
    K = 1 + dim + dim * (dim + 1) // 2
    b = nnz * (4 + 8 * nmats + 12 * K + 8 * m)          # pattern, forms, A64/A32, L64
    b += n * m * 16 * (4 + (2 if precision_mixed else 0))  # block inverses (+ FP16 copy)
    vec = 4 if precision_mixed else 8
    b += n * m * (vec * (restart + 4) + 8 * 8)            # Krylov basis + FP64 state/work
    return int(b)


class LibraryBackend:
    """Runs requests on the GPU library through ``TransportProblem``."""

    def __init__(self):
        import paper_2008_02205_gb300 as pkg
        self.pkg = pkg
        # the device current in the scheduling thread: set-up threads create their contexts there
        self.device = None
        try:
            import torch
            if torch.cuda.is_available():
                self.device = torch.cuda.current_device()
        except ImportError:
            pass

    def thread_init(self):
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)

    def open(self, req: Request):
        tp = self.pkg.TransportProblem.from_problem(req.problem, **req.options)
        try:
            tp.integrate().assemble()
        except Exception:
            tp.close()
            raise
        return tp

    def step(self, handles, dts):
        """One concurrent step of every handle; returns None or an error
        message per handle."""
        st = self.pkg.mlpg_step_batch([h.ctx for h in handles], dts, raise_on_error=False)
        return [None if s == 0 else f"step failed (status {s}): {self.pkg.mlpg_last_error(h.ctx)}"
                for s, h in zip(st, handles)]

    def flux(self, h):
        return h.scalar_flux()

    def device_bytes(self, h):
        return int(h.stats()["device_bytes"])

    def close(self, h):
        h.close()


class Server:
    """FIFO admission under a device-memory budget and a slot limit; one
    concurrent step of every admitted problem per iteration.

    A backend provides open(request) -> handle, step(handles, dts) -> None
    (all done) or a per-handle list of None / error message, flux(handle) and
    close(handle)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 16, backend=None, clock=time.perf_counter,
                 estimate=estimate_bytes, sleep=time.sleep, open_workers: int = 1):
        """open_workers > 0: admitted requests are set up (integrate +
        assemble, on their own streams) by that many background threads while
        the resident problems keep stepping; they join the batch once ready.
        open_workers = 0: set up inline, in the scheduling thread."""
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.backend = backend if backend is not None else LibraryBackend()
        self.clock = clock
        self.estimate = estimate
        self.sleep = sleep
        self.open_workers = int(open_workers)
        self.peak_active = 0
        self.iterations = 0
        self.steps_during_open = 0   # batched steps taken while some admitted request was being set up

    def run(self, requests):
        pending = sorted(requests, key=lambda r: r.arrival)
        results = {id(r): Result(r) for r in requests}
        active = []          # [request, handle, bytes, steps done]
        opening = []         # [request, future, bytes]: admitted, being set up
        used = 0
        t0 = self.clock()
        pool = None
        if self.open_workers > 0:
            from concurrent.futures import ThreadPoolExecutor
            pool = ThreadPoolExecutor(max_workers=self.open_workers, thread_name_prefix="mlpg-open",
                                      initializer=getattr(self.backend, "thread_init", None))

        def retire(a, error=None):
            nonlocal used
            res = results[id(a[0])]
            if error is None:
                res.flux = self.backend.flux(a[1])
            else:
                res.error = error
            measure = getattr(self.backend, "device_bytes", None)
            if measure is not None:
                res.device_bytes = measure(a[1])
            self.backend.close(a[1])
            res.finished = self.clock() - t0
            used -= a[2]

        def opened(req, need, handle=None, error=None):
            nonlocal used
            res = results[id(req)]
            if error is not None:       # bad input, geometry, device memory: this request only
                res.error = f"open failed: {error}"
                res.finished = self.clock() - t0
                used -= need
            else:
                active.append([req, handle, need, 0])

        try:
            while pending or active or opening:
                now = self.clock() - t0
                while pending and pending[0].arrival <= now and len(active) + len(opening) < self.max_active:
                    req = pending[0]
                    need = self.estimate(req.problem, req.options.get("precision", 0) == 1)   # 1: mixed
                    res = results[id(req)]
                    if need > self.budget:      # can never fit: refuse it
                        pending.pop(0)
                        res.error = f"needs {need} bytes, budget {self.budget}"
                        res.admitted = res.finished = now
                        continue
                    if used + need > self.budget:
                        break                   # wait for memory to free up (FIFO)
                    pending.pop(0)
                    res.admitted = self.clock() - t0
                    used += need
                    if pool is not None:
                        opening.append([req, pool.submit(self.backend.open, req), need])
                        continue
                    try:
                        handle = self.backend.open(req)
                    except Exception as e:
                        opened(req, need, error=e)
                        continue
                    opened(req, need, handle)
                # set-ups that finished join the batch
                still = []
                for o in opening:
                    if o[1].done():
                        try:
                            opened(o[0], o[2], o[1].result())
                        except Exception as e:
                            opened(o[0], o[2], error=e)
                    else:
                        still.append(o)
                opening = still
                if not active:
                    if opening:                 # nothing to step: wait for a set-up
                        from concurrent.futures import FIRST_COMPLETED, wait
                        wait([o[1] for o in opening], timeout=0.01, return_when=FIRST_COMPLETED)
                    elif pending:               # idle until the next arrival
                        wait_s = pending[0].arrival - (self.clock() - t0)
                        if wait_s > 0:
                            self.sleep(min(wait_s, 0.01))
                    continue
                self.peak_active = max(self.peak_active, len(active))
                if opening:
                    self.steps_during_open += 1
                errors = self.backend.step([a[1] for a in active], [a[0].dt for a in active])
                if errors is None:
                    errors = [None] * len(active)
                self.iterations += 1
                keep = []
                for a, err in zip(active, errors):
                    if err is not None:
                        retire(a, err)
                        continue
                    a[3] += 1
                    if a[3] >= a[0].steps:
                        retire(a)
                    else:
                        keep.append(a)
                active = keep
        finally:                                # an escaping error still releases every context
            for a in active:
                try:
                    self.backend.close(a[1])
                except Exception:
                    pass
            for o in opening:
                try:
                    self.backend.close(o[1].result())
                except Exception:
                    pass
            if pool is not None:
                pool.shutdown(wait=True)
        return [results[id(r)] for r in requests]


def latency_percentiles(results, qs=(50, 99)):
    lat = np.array([r.latency for r in results if r.error is None])
    return {f"p{q}": float(np.percentile(lat, q)) for q in qs} if len(lat) else {}
