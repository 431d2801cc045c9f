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
                 estimate=lambda p, mixed: p.size)
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
