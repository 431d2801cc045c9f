"""GPU parity of the tiled FP32 transport-operator apply (Sec. 4.2, operator L).

The row-tile kernel stages each tile's neighbour rows of X in shared memory
and combines the direction-independent arrays per direction in registers.  It
is checked against the oracle's assembled L_m (FP64, one sparse product per
direction) and against the row-team kernel on the same context's operators,
for every direction count the kernel handles differently: 4 or 8 directions
per thread, one or several direction chunks per tile, 2D and 3D, tiles cut
short by the point count (ragged last tile), several tiles per problem.
Tolerance: FP32 arithmetic over about 50 (2D) or 240 (3D) entries per row
with values of both signs, 3e-6 relative L2 against FP64, as for the
row-team kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import oracle.mlpg_oracle as O  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _apply(prob, X, kernel, dt, **opts):
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED, apply_kernel=kernel, **opts) as tp:
        tp.integrate().assemble()
        Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
        Yd = torch.full_like(Xd, float("nan"))
        pkg.mlpg_apply_L_dev(tp.ctx, dt, pkg.MLPG_MIXED, Xd.data_ptr(), Yd.data_ptr())
        torch.cuda.synchronize()
        st = tp.stats()
        return Yd.double().cpu().numpy(), st


CASES = [
    # (dim, points per side, S_N or refined set, expected directions per CTA or None)
    (2, 13, 4, None),     # m = 12: 4 directions per thread, 169 points: three tiles, the last ragged
    (2, 30, 6, None),     # m = 24: 8 per thread
    (2, 30, 8, None),     # m = 40: the benchmark's angular set
    (2, 17, 10, None),    # m = 60: 4 per thread
    (2, 17, 12, 28),      # m = 84: three direction chunks of 28
    (3, 6, 4, None),      # 3D, m = 24
    (3, 7, 8, None),      # 3D, m = 80, several chunks
    (3, 5, "refined", None),  # 3D, Alg. 2 set (m = 48 with levels 0 -> 2)
]


MMA_CASES = [
    (2, 30, 6, 24),       # m = 24: one chunk of three n-tiles
    (2, 30, 8, 40),       # m = 40: two n-tile pairs and a single n-tile
    (3, 6, 4, 24),        # 3D, m = 24: two k-steps (ten base arrays)
    (3, 7, 8, None),      # 3D, m = 80: several chunks (the halo of a 7^3 tile limits the chunk)
    (3, 5, "refined", 32),  # 3D, Alg. 2 set (m = 32)
]


@pytest.mark.parametrize("dim,side,sn,chunk", MMA_CASES)
def test_tensor_core_tiles_match_oracle_and_row_teams(dim, side, sn, chunk):
    """apply_kernel 3: the base arrays combined by mma.m16n8k8 on TF32 high
    and low parts; FP32 accuracy, checked as the CUDA-core tiles are."""
    if dim == 2:
        prob = mi.two_region_2d(n_per_dim=side, sn=sn, seed=2100 + side)
    elif sn == "refined":
        prob = mi.lognormal_3d(side, seed=3100 + side, refine=(0, 2, 30.0))
    else:
        prob = mi.lognormal_3d(side, sn=sn, seed=3100 + side)
    rng = np.random.default_rng(13)
    X = rng.uniform(-1.0, 1.0, (prob.n, prob.m))
    Yt, st = _apply(prob, X, 3, prob.dt)
    assert st["apply_kernel"] == 3 and st["tile_chunk"] % 8 == 0 and prob.m % st["tile_chunk"] == 0
    if chunk is not None:
        assert st["tile_chunk"] == chunk
    Yr, _ = _apply(prob, X, 1, prob.dt)
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w)
    ref = np.stack([tr.L_matrix(m, 1.0 / prob.dt) @ X[:, m] for m in range(prob.m)], axis=1)
    assert np.all(np.isfinite(Yt))
    assert _rel(Yt, ref) < 3e-6
    assert _rel(Yt, Yr) < 3e-6


def test_mixed_run_through_tensor_core_tiles_matches_oracle():
    prob = mi.two_region_2d(n_per_dim=18, sn=8, seed=2218, steps=3)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED, apply_kernel=3) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert tp.stats()["apply_kernel"] == 3
    ref = O.solve_problem(prob)
    assert _rel(phi, ref) < 1e-8


@pytest.mark.parametrize("dim,side,sn,chunk", CASES)
def test_tiled_apply_matches_oracle_and_row_teams(dim, side, sn, chunk):
    if dim == 2:
        prob = mi.two_region_2d(n_per_dim=side, sn=sn, seed=2100 + side)
    elif sn == "refined":
        prob = mi.lognormal_3d(side, seed=3100 + side, refine=(0, 2, 30.0))
    else:
        prob = mi.lognormal_3d(side, sn=sn, seed=3100 + side)
    assert prob.m % 4 == 0
    rng = np.random.default_rng(11)
    X = rng.uniform(-1.0, 1.0, (prob.n, prob.m))
    Yt, st = _apply(prob, X, 2, prob.dt)
    assert st["apply_kernel"] == 2
    if chunk is not None:
        assert st["tile_chunk"] == chunk
    Yr, st1 = _apply(prob, X, 1, prob.dt)
    assert st1["apply_kernel"] == 1
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w)
    ref = np.stack([tr.L_matrix(m, 1.0 / prob.dt) @ X[:, m] for m in range(prob.m)], axis=1)
    assert np.all(np.isfinite(Yt))
    assert _rel(Yt, ref) < 3e-6
    assert _rel(Yt, Yr) < 3e-6


def test_tiled_apply_is_the_automatic_choice_for_the_benchmark_set():
    prob = mi.two_region_2d(n_per_dim=40)
    X = np.random.default_rng(5).uniform(-1.0, 1.0, (prob.n, prob.m))
    _, st = _apply(prob, X, 0, prob.dt)
    assert st["apply_kernel"] == 2 and st["tile_chunk"] == 40


def test_mixed_run_through_tiles_matches_oracle():
    """A whole mixed-precision run (residual form Y = B - L X inside GMRES and
    the FP64 refinement) on the tiled kernel: the flux within 1e-8 of the
    oracle's FP64 solve."""
    prob = mi.two_region_2d(n_per_dim=18, sn=8, seed=2218, steps=3)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED, apply_kernel=2) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert tp.stats()["apply_kernel"] == 2
    ref = O.solve_problem(prob)
    assert _rel(phi, ref) < 1e-8


GATHER_CASES = [
    # (dim, points per side, S_N or refined set, rows per tile, directions per thread, expected chunk)
    (2, 13, 4, 8, 4, 12),      # m = 12, 169 points: 22 tiles of 8 rows, the last ragged
    (2, 30, 8, 32, 8, 40),     # the benchmark's angular set
    (2, 17, 12, 16, 4, 44),    # m = 84: two chunks of 44 and 40 (the last chunk's spare lanes read nothing)
    (2, 17, 12, 32, 4, 28),    # m = 84 on 32-row tiles: three chunks (at most 320 threads per CTA)
    (3, 6, 4, 16, 8, 24),      # 3D, m = 24
    (3, 7, 8, 8, 8, 80),       # 3D, m = 80 in one chunk (the staged-halo tiles need several)
    (3, 7, 8, 4, 4, 80),       # 3D, 4-row tiles
    (3, 5, "refined", 0, 0, None),  # 3D, Alg. 2 set, automatic tile shape
]


@pytest.mark.parametrize("dim,side,sn,rows,dpt,chunk", GATHER_CASES)
def test_gather_tiles_match_oracle_and_row_teams(dim, side, sn, rows, dpt, chunk):
    """apply_kernel 4: the tile's records staged in shared memory, X read from
    global memory; the same arithmetic as the staged-halo tiles."""
    if dim == 2:
        prob = mi.two_region_2d(n_per_dim=side, sn=sn, seed=2100 + side)
    elif sn == "refined":
        prob = mi.lognormal_3d(side, seed=3100 + side, refine=(0, 2, 30.0))
    else:
        prob = mi.lognormal_3d(side, sn=sn, seed=3100 + side)
    rng = np.random.default_rng(17)
    X = rng.uniform(-1.0, 1.0, (prob.n, prob.m))
    Yt, st = _apply(prob, X, 4, prob.dt, tile_rows=rows, tile_dpt=dpt)
    assert st["apply_kernel"] == 4
    if chunk is not None:
        assert st["tile_chunk"] == chunk
    Yr, _ = _apply(prob, X, 1, prob.dt)
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w)
    ref = np.stack([tr.L_matrix(m, 1.0 / prob.dt) @ X[:, m] for m in range(prob.m)], axis=1)
    assert np.all(np.isfinite(Yt))
    assert _rel(Yt, ref) < 3e-6
    assert _rel(Yt, Yr) < 3e-6


def test_gather_tiles_at_the_3d_configuration_size():
    """40^3 points, 272 directions (the refined 3D set): the automatic choice
    is gather mode with all directions in one chunk of 4-row tiles; against
    the row-team kernel on the same operators (both FP32, parity-tested
    against the oracle above)."""
    prob = mi.lognormal_3d(refine=(1, 5, 15.0))
    X = np.random.default_rng(19).uniform(-1.0, 1.0, (prob.n, prob.m))
    Yt, st = _apply(prob, X, 0, prob.dt)   # the automatic choice at this size
    assert st["apply_kernel"] == 4 and st["tile_chunk"] == 272
    Yr, _ = _apply(prob, X, 1, prob.dt)
    assert np.all(np.isfinite(Yt))
    assert _rel(Yt, Yr) < 3e-6


def test_mixed_run_through_gather_tiles_matches_oracle():
    prob = mi.two_region_2d(n_per_dim=18, sn=8, seed=2218, steps=3)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED, apply_kernel=4) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert tp.stats()["apply_kernel"] == 4
    ref = O.solve_problem(prob)
    assert _rel(phi, ref) < 1e-8


def test_apply_rejects_misaligned_and_overlapping_vectors():
    prob = mi.two_region_2d(n_per_dim=10, sn=4, seed=2210)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED) as tp:
        tp.integrate().assemble()
        buf = torch.zeros(3 * prob.n * prob.m + 8, dtype=torch.float32, device="cuda")
        x = buf.data_ptr()
        y = x + 4 * (prob.n * prob.m + 4)
        for bad_x, bad_y in ((x + 4, y), (x, y + 8), (x, x + 16)):
            with pytest.raises(pkg.MlpgError):
                pkg.mlpg_apply_L_dev(tp.ctx, prob.dt, pkg.MLPG_MIXED, bad_x, bad_y)
        pkg.mlpg_apply_L_dev(tp.ctx, prob.dt, pkg.MLPG_MIXED, x, y)
        torch.cuda.synchronize()
