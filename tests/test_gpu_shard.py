"""Direction shards on the GPU: one problem split over two and three contexts
(subsets of the ordinates, Sec. 4.2: L^-1 is block-diagonal in angle), each
stepped by its own host thread on this device, exchanging only the angular
reduction D and the residual norms through the cross-shard sum callback.
The outer solve is replicated on identical data, so the split problem must
give the unsplit problem's scalar flux and angular flux: to 1e-12 relative
L2 in FP64 (the same arithmetic, summed in another order), to the refinement
tolerance in mixed precision; and the oracle's flux within the usual bars."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import oracle.mlpg_oracle as O  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402
from paper_2008_02205_gb300.shard import ShardedProblem  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,shards,bar", [(pkg.MLPG_FP64, 2, 1e-12), (pkg.MLPG_FP64, 3, 1e-12),
                                                  (pkg.MLPG_MIXED, 2, 1e-10)])
def test_sharded_solve_equals_the_unsplit_solve(precision, shards, bar):
    prob = mi.two_region_2d(14, sn=8, steps=3, seed=2414)
    opts = dict(precision=precision, inner_tol=1e-13, outer_tol=1e-13, refine_tol=1e-12)
    with pkg.TransportProblem.from_problem(prob, **opts) as tp:
        tp.integrate().assemble()
        whole = tp.run(prob.dt, prob.steps)
        psi = tp.state()
    with ShardedProblem(prob, shards, **opts) as sp:
        split = sp.run(prob.dt, prob.steps)
        psi_s = sp.state()
    assert _rel(split, whole) < bar
    assert _rel(psi_s, psi) < 10 * bar
    ref = O.solve_problem(prob)
    assert _rel(split, ref) < (1e-9 if precision == pkg.MLPG_FP64 else 1e-8)


def test_sharded_3d_with_inflow():
    prob = mi.lognormal_3d(5, sn=4, seed=3005, steps=2, dt=0.02)
    opts = dict(inner_tol=1e-13, outer_tol=1e-13)
    with pkg.TransportProblem.from_problem(prob, **opts) as tp:
        tp.integrate().assemble()
        whole = tp.run(prob.dt, prob.steps)
    with ShardedProblem(prob, 2, **opts) as sp:
        split = sp.run(prob.dt, prob.steps)
    assert _rel(split, whole) < 1e-12
