"""The serving loop on the GPU: problems of different sizes, dimensions and
quadratures arrive over time, are admitted under a memory budget that forces
some of them to wait, and are stepped together; every served result equals
the same problem solved alone, within the mixed-precision tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402
from paper_2008_02205_gb300.serving import Request, Server, estimate_bytes, latency_percentiles  # noqa: E402


def test_served_results_equal_alone_results():
    probs = mi.batched_2d(3, seed=4200, n_range=(64, 300), steps=3) + \
        [mi.lognormal_3d(6, sn=4, seed=3002, steps=3, dt=0.02)]
    opts = dict(precision=pkg.MLPG_MIXED, refine_tol=1e-12)
    # the first two arrive together (the budget below admits any two, so they
    # overlap on the device whatever the timing); the others join later
    arrivals = [0.0, 0.0, 0.02, 0.04]
    reqs = [Request(p, p.steps, p.dt, arrival=t, options=opts) for p, t in zip(probs, arrivals)]
    alone = []
    for r in reqs:
        with pkg.TransportProblem.from_problem(r.problem, **r.options) as tp:
            tp.integrate().assemble()
            alone.append(tp.run(r.dt, r.steps))
    est = sorted(estimate_bytes(p, True) for p in probs)
    server = Server(hbm_budget_bytes=est[-1] + est[-2], max_active=3)
    res = server.run(reqs)
    for r, a in zip(res, alone):
        assert r.error is None
        assert np.linalg.norm(r.flux - a) / np.linalg.norm(a) < 1e-9
    assert server.peak_active >= 2
    lat = latency_percentiles(res)
    assert 0 < lat["p50"] <= lat["p99"]


def test_failed_requests_leave_alone_and_the_rest_are_served():
    """One request hits an iteration cap in its first step and one cannot be
    created (a point outside the box): each fails with its own error, and the
    two healthy problems stepped in the same batches equal their solo runs."""
    good = mi.batched_2d(2, seed=4300, n_range=(64, 200), steps=3)
    capped = mi.batched_2d(1, seed=4310, n_range=(64, 100), steps=3)[0]
    outside = mi.batched_2d(1, seed=4320, n_range=(64, 100), steps=3)[0]
    outside.x = outside.x.copy()
    outside.x[0, 0] = 1.5
    mixed = dict(precision=pkg.MLPG_MIXED, refine_tol=1e-12)
    reqs = [Request(good[0], 3, good[0].dt, options=mixed),
            Request(capped, 3, capped.dt, options=dict(max_inner=1, inner_restart=2)),
            Request(outside, 3, outside.dt, options=mixed),
            Request(good[1], 3, good[1].dt, options=mixed)]
    alone = []
    for p in good:
        with pkg.TransportProblem.from_problem(p, **mixed) as tp:
            tp.integrate().assemble()
            alone.append(tp.run(p.dt, 3))
    res = Server(hbm_budget_bytes=1 << 34, max_active=4).run(reqs)
    assert res[1].flux is None and "status -7" in res[1].error
    assert res[2].flux is None and res[2].error.startswith("open failed")
    for r, a in zip((res[0], res[3]), alone):
        assert r.error is None
        assert np.linalg.norm(r.flux - a) / np.linalg.norm(a) < 1e-9
