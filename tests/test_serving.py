"""Host logic of the continuous-batching serving loop (no GPU): admission in
arrival order under the memory budget and the slot limit, one concurrent step
of every admitted problem per iteration, retirement after the last step,
refusal of requests that can never fit, latencies from arrival."""
import numpy as np

from paper_2008_02205_gb300.serving import Request, Server, latency_percentiles


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4
        return self.t

    def sleep(self, s):
        self.t += s


class FakeProblem:
    def __init__(self, size):
        self.size = size


class FakeBackend:
    def __init__(self):
        self.open_sizes = {}
        self.calls = []
        self.steps = {}

    def open(self, req):
        h = id(req)
        self.open_sizes[h] = req.problem.size
        self.steps[h] = 0
        return h

    def step(self, handles, dts):
        self.calls.append((list(handles), sum(self.open_sizes[h] for h in handles)))
        for h in handles:
            self.steps[h] += 1

    def flux(self, h):
        return np.full(3, float(self.steps[h]))

    def close(self, h):
        del self.open_sizes[h]


def _server(budget, max_active=8):
    clk, be = FakeClock(), FakeBackend()
    srv = Server(budget, max_active=max_active, backend=be, clock=clk, sleep=clk.sleep,
                 estimate=lambda p, mixed: p.size, open_workers=0)
    return srv, be


def test_budget_slots_and_step_counts():
    reqs = [Request(FakeProblem(s), steps=k + 2, dt=0.1, arrival=0.0) for k, s in enumerate([6, 6, 3, 2, 5])]
    srv, be = _server(budget=10, max_active=2)
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    for handles, used in be.calls:
        assert len(handles) <= 2 and used <= 10
    for r in res:
        assert r.flux[0] == r.request.steps          # exactly `steps` steps each
        assert r.latency >= 0 and r.finished >= r.admitted
    # FIFO: nobody overtakes an earlier arrival that is waiting for memory
    admitted = [r.admitted for r in res]
    assert admitted == sorted(admitted)
    assert srv.peak_active == 2


def test_refuses_what_can_never_fit_and_serves_the_rest():
    reqs = [Request(FakeProblem(50), steps=1, dt=0.1), Request(FakeProblem(4), steps=3, dt=0.1)]
    srv, be = _server(budget=10)
    res = srv.run(reqs)
    assert res[0].error is not None and res[0].flux is None
    assert res[1].error is None and res[1].flux[0] == 3


def test_late_arrivals_join_a_running_batch():
    reqs = [Request(FakeProblem(1), steps=50, dt=0.1, arrival=0.0),
            Request(FakeProblem(1), steps=5, dt=0.1, arrival=0.002)]
    srv, be = _server(budget=10)
    res = srv.run(reqs)
    # the second request ran while the first was still active
    assert any(len(h) == 2 for h, _ in be.calls)
    assert res[1].finished < res[0].finished
    p = latency_percentiles(res)
    assert set(p) == {"p50", "p99"} and p["p99"] >= p["p50"] > 0


def test_idle_until_first_arrival():
    reqs = [Request(FakeProblem(1), steps=2, dt=0.1, arrival=0.5)]
    srv, be = _server(budget=10)
    res = srv.run(reqs)
    assert res[0].admitted >= 0.5 and res[0].flux[0] == 2


class FailingBackend(FakeBackend):
    """Fails to open problems of size `bad_open` and fails the step of
    problems of size `bad_step` once they have taken `after` steps."""

    def __init__(self, bad_open=None, bad_step=None, after=0):
        super().__init__()
        self.bad_open, self.bad_step, self.after = bad_open, bad_step, after
        self.closed = []

    def open(self, req):
        if req.problem.size == self.bad_open:
            raise RuntimeError("geometry")
        return super().open(req)

    def step(self, handles, dts):
        errs = []
        for h in handles:
            if self.open_sizes[h] == self.bad_step and self.steps[h] >= self.after:
                errs.append("not converged")
            else:
                errs.append(None)
        self.calls.append((list(handles), sum(self.open_sizes[h] for h in handles)))
        for h, e in zip(handles, errs):
            if e is None:
                self.steps[h] += 1
        return errs

    def close(self, h):
        self.closed.append(h)
        super().close(h)


def _failing_server(budget, **kw):
    clk, be = FakeClock(), FailingBackend(**kw)
    return Server(budget, backend=be, clock=clk, sleep=clk.sleep, estimate=lambda p, mixed: p.size,
                  open_workers=0), be


def test_a_request_that_cannot_be_opened_fails_alone():
    reqs = [Request(FakeProblem(s), steps=3, dt=0.1) for s in (2, 7, 3)]
    srv, be = _failing_server(10, bad_open=7)
    res = srv.run(reqs)
    assert "open failed" in res[1].error and res[1].flux is None
    assert res[0].error is None and res[2].error is None
    assert res[0].flux[0] == 3 and res[2].flux[0] == 3
    assert max(used for _, used in be.calls) == 5      # the failed open charged no memory
    assert not be.open_sizes                          # everything opened was closed


def test_a_failing_step_retires_its_request_and_the_others_finish():
    reqs = [Request(FakeProblem(s), steps=6, dt=0.1) for s in (2, 4, 3)]
    srv, be = _failing_server(9, bad_step=4, after=2)
    res = srv.run(reqs)
    assert res[1].error == "not converged" and res[1].flux is None
    assert res[0].flux[0] == 6 and res[2].flux[0] == 6
    # the failed problem left after its third step call; the others went on without it
    assert all(len(h) == 2 for h, _ in be.calls[3:]) and len(be.calls) == 6
    assert not be.open_sizes


def test_an_escaping_error_still_closes_every_context():
    class Boom(FailingBackend):
        def step(self, handles, dts):
            raise ValueError("bad batch")
    clk, be = FakeClock(), Boom()
    srv = Server(10, backend=be, clock=clk, sleep=clk.sleep, estimate=lambda p, mixed: p.size, open_workers=0)
    import pytest
    with pytest.raises(ValueError):
        srv.run([Request(FakeProblem(1), steps=2, dt=0.1), Request(FakeProblem(2), steps=2, dt=0.1)])
    assert len(be.closed) == 2 and not be.open_sizes


def test_serves_a_poisson_stream_under_the_estimated_budget():
    import mlpg_inputs as mi
    from paper_2008_02205_gb300.serving import estimate_bytes

    class SizedBackend(FakeBackend):
        def open(self, req):
            h = id(req)
            self.open_sizes[h] = estimate_bytes(req.problem, True)
            self.steps[h] = 0
            return h

    stream = mi.serving_stream(count=30, rate=50.0, seed=5200, n_range=(64, 2048))
    reqs = [Request(p, p.steps, p.dt, arrival=t, options={"precision": 1}) for p, t in stream]
    est = [estimate_bytes(p, True) for p, _ in stream]
    budget = 3 * max(est)
    clk, be = FakeClock(), SizedBackend()
    srv = Server(budget, max_active=8, backend=be, clock=clk, sleep=clk.sleep)
    res = srv.run(reqs)
    assert all(r.error is None and r.flux[0] == r.request.steps for r in res)
    assert max(used for _, used in be.calls) <= budget
    assert srv.peak_active >= 2
    admitted = [r.admitted for r in sorted(res, key=lambda r: r.request.arrival)]
    assert admitted == sorted(admitted)


def test_device_memory_is_recorded_when_the_backend_reports_it():
    class Measured(FakeBackend):
        def device_bytes(self, h):
            return 1000 + self.steps[h]

    clk, be = FakeClock(), Measured()
    srv = Server(10, backend=be, clock=clk, sleep=clk.sleep, estimate=lambda p, mixed: p.size, open_workers=0)
    res = srv.run([Request(FakeProblem(2), steps=3, dt=0.1), Request(FakeProblem(1), steps=5, dt=0.1)])
    assert [r.device_bytes for r in res] == [1003, 1005]     # taken after each problem's last step
    res = _server(10)[0].run([Request(FakeProblem(1), steps=1, dt=0.1)])
    assert res[0].device_bytes is None                       # a backend without the counter


class SlowOpenBackend(FakeBackend):
    """Set-up of the second request blocks until the first has taken three
    steps: with background set-up the first keeps stepping meanwhile."""

    def __init__(self):
        super().__init__()
        import threading
        self.gate = threading.Event()

    def open(self, req):
        if req.problem.size == 2:
            assert self.gate.wait(timeout=10.0)
        return super().open(req)

    def step(self, handles, dts):
        import time
        super().step(handles, dts)
        if any(self.steps[h] >= 3 for h in handles):
            self.gate.set()
        time.sleep(0.002)                      # a step takes time: the set-up thread catches up


def test_setup_runs_beside_the_resident_batch():
    be = SlowOpenBackend()
    reqs = [Request(FakeProblem(1), steps=200, dt=0.1, arrival=0.0),
            Request(FakeProblem(2), steps=2, dt=0.1, arrival=0.0)]
    srv = Server(10, backend=be, estimate=lambda p, mixed: p.size, open_workers=1)
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    assert res[0].flux[0] == 200 and res[1].flux[0] == 2
    assert srv.steps_during_open >= 3          # the first problem stepped while the second was set up
    assert any(len(h) == 2 for h, _ in be.calls)


def test_background_setup_failure_stays_with_its_request():
    class Bad(FakeBackend):
        def open(self, req):
            if req.problem.size == 3:
                raise RuntimeError("geometry")
            return super().open(req)
    be = Bad()
    reqs = [Request(FakeProblem(1), steps=3, dt=0.1), Request(FakeProblem(3), steps=3, dt=0.1),
            Request(FakeProblem(2), steps=3, dt=0.1)]
    res = Server(10, backend=be, estimate=lambda p, mixed: p.size, open_workers=2).run(reqs)
    assert res[1].error.startswith("open failed") and res[1].flux is None
    assert res[0].flux[0] == 3 and res[2].flux[0] == 3
    assert be.open_sizes == {}
