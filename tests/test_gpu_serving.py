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
