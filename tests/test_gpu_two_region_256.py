"""The benchmark workload itself against the oracle's solve of it.

2D unit square, 256x256 jittered points, S8 (40 directions), two-region
sigma_t (100 in [0.4, 0.6]^2, 1 elsewhere), scattering ratio 0.9, q = 1 for
x < 0.5, vacuum, 20 backward-Euler steps of dt = 0.005 (Sec. 4.1-4.2), in
the benchmark's launch configuration.  The expected scalar flux after steps
1, 10 and 20 was written by tests/golden/make_two_region_256_golden.py, which
runs only the FP64 oracle (exact inner solves, outer GMRES to 1e-13).

Bars (relative L2 over all points): 1e-9 for the FP64 path, 1e-8 for the
mixed-precision path (FP32 operator streams and Krylov vectors, FP64
refinement of every step to a 1e-11 step residual)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import mlpg_inputs as mi  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "two_region_256_phi.npz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def golden():
    g = np.load(GOLDEN)
    assert int(g["n_per_dim"]) == 256 and int(g["steps"]) == 20
    return g


@pytest.mark.parametrize("precision,bar", [(pkg.MLPG_MIXED, 1e-8), (pkg.MLPG_FP64, 1e-9)])
def test_two_region_256_matches_oracle(golden, precision, bar):
    prob = mi.two_region_2d()
    errs = {}
    with pkg.TransportProblem.from_problem(prob, precision=precision) as tp:
        tp.integrate().assemble()
        for k in range(1, prob.steps + 1):
            tp.step(prob.dt)
            if f"phi_{k}" in golden:
                errs[k] = _rel(tp.scalar_flux(), golden[f"phi_{k}"])
        st = tp.stats()
    print(f"precision {precision}: rel. L2 vs oracle by step {errs}; last step outer {st['last_outer_iters']}, "
          f"oracle outer by step {golden['outer_iterations'].tolist()}")
    assert set(errs) == {1, 10, 20}
    for k, e in errs.items():
        assert e < bar, (k, e)
