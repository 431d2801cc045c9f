"""Seeded synthetic inputs for the MLPG/RK discrete-ordinates transport solve.

This module is shared by the tests, the benchmark and the CPU oracle.  It holds
only input generation: point clouds, angular quadrature sets, per-point material
data.  None of the discretisation arithmetic (kernels, RK corrections, cells,
quadrature over cells, assembly, solvers) lives here.

Point sets follow the perturbed-lattice recipe of Sec. 5 ("Manufactured
problems"): a uniform lattice whose coordinates are each displaced by
gamma * spacing with gamma uniform in [-0.2, 0.2], independently per point and
dimension.  Lattice points are cell-centred in the unit box.

Angular sets are level-symmetric S_N quadratures built here by even-moment
matching (the paper's own LDFE sets are only cited, Sec. 4.3).  In 2D the
directions of the upper hemisphere (Omega_z > 0) are kept with doubled weights,
so that sum(w) = 4*pi as in the 3D transport equation (Eq. transport-equation,
Sec. 4.1).
"""
from __future__ import annotations

import functools
import itertools
import math
from dataclasses import dataclass, field

import numpy as np

FOUR_PI = 4.0 * math.pi


# --------------------------------------------------------------------------
# point sets
# --------------------------------------------------------------------------
def jittered_lattice(n_per_dim: int, dim: int, seed: int, lo: float = 0.0,
                     hi: float = 1.0, jitter: float = 0.2):
    """Cell-centred lattice of n_per_dim**dim points in [lo, hi]^dim.

    Each coordinate is moved by spacing * gamma, gamma ~ U[-jitter, jitter]
    (numpy PCG64(seed)), as in Sec. 5.  Returns (x[n, dim], spacing).
    Point order: the last coordinate varies slowest (row-major over (z, y, x)).
    """
    h = (hi - lo) / n_per_dim
    axes = [lo + (np.arange(n_per_dim) + 0.5) * h for _ in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # x fastest
    x = np.stack([g.reshape(-1) for g in grids], axis=1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        x = x + h * rng.uniform(-jitter, jitter, size=x.shape)
    return np.ascontiguousarray(x), h


# --------------------------------------------------------------------------
# level-symmetric angular quadrature by even-moment matching
# --------------------------------------------------------------------------
def _octant_points(n_levels: int):
    """Index triples (a, b, c), 1-based levels with a + b + c = n_levels + 2."""
    pts = []
    for a in range(1, n_levels + 1):
        for b in range(1, n_levels + 1):
            c = n_levels + 2 - a - b
            if c >= 1:
                pts.append((a, b, c))
    return pts


def _ls_weights(order: int, mu1: float):
    """Per-class weights matching the even moments for a given mu1.

    Returns (mu levels, points, class of each point, class weights) with the
    octant normalised to 4*pi/8.  Moments used: k = 0 and k = 2..n_classes
    (k = 1 holds for every symmetric set and adds no equation).
    """
    n = order // 2
    if n == 1:
        mu = np.array([math.sqrt(1.0 / 3.0)])
    else:
        delta = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (order - 2)
        mu2 = mu1 * mu1 + delta * np.arange(n)
        if np.any(mu2 <= 0.0):
            return None
        mu = np.sqrt(mu2)
    pts = _octant_points(n)
    classes = sorted({tuple(sorted(p)) for p in pts})
    cls_of = [classes.index(tuple(sorted(p))) for p in pts]
    ncls = len(classes)
    ks = [0] + list(range(2, ncls + 1))
    A = np.zeros((ncls, ncls))
    rhs = np.zeros(ncls)
    for r, k in enumerate(ks):
        for p, c in zip(pts, cls_of):
            A[r, c] += mu[p[0] - 1] ** (2 * k)
        rhs[r] = FOUR_PI / 8.0 / (2 * k + 1)
    try:
        wc = np.linalg.solve(A, rhs)
    except np.linalg.LinAlgError:
        return None
    return mu, pts, cls_of, wc


def _next_moment_residual(order: int, mu1: float):
    got = _ls_weights(order, mu1)
    if got is None:
        return None, None
    mu, pts, cls_of, wc = got
    k = len(wc) + 1
    s = sum(wc[c] * mu[p[0] - 1] ** (2 * k) for p, c in zip(pts, cls_of))
    return s - FOUR_PI / 8.0 / (2 * k + 1), wc


def level_symmetric(order: int, dim: int):
    """Level-symmetric S_N set: (omega[M, 3], w[M]) with sum(w) = 4*pi.
    Built once per (order, dim); every call returns fresh copies.

    mu1 is the root, in (0, 1/sqrt(3)), of the first even moment not used for
    the weights, taken among roots with all class weights positive (the root
    with the largest mu1 when several exist).  3D: N(N+2) directions; 2D: the
    N(N+2)/2 directions with Omega_z > 0, weights doubled.
    """
    om, w = _level_symmetric_cached(int(order), int(dim))
    return om.copy(), w.copy()


@functools.lru_cache(maxsize=None)
def _level_symmetric_cached(order: int, dim: int):
    if order < 2 or order % 2:
        raise ValueError("S_N order must be even and >= 2")
    n = order // 2
    if n == 1:
        mu1 = math.sqrt(1.0 / 3.0)
    else:
        grid = np.linspace(1e-4, math.sqrt(1.0 / 3.0) - 1e-6, 4000)
        roots = []
        prev = None
        for g in grid:
            res, wc = _next_moment_residual(order, g)
            if res is not None and prev is not None and prev[0] is not None \
                    and np.sign(res) != np.sign(prev[0]):
                a, b = prev[1], g
                fa = prev[0]
                for _ in range(200):
                    mid = 0.5 * (a + b)
                    fm, _ = _next_moment_residual(order, mid)
                    if fm is None:
                        break
                    if np.sign(fm) == np.sign(fa):
                        a, fa = mid, fm
                    else:
                        b = mid
                r = 0.5 * (a + b)
                _, wr = _next_moment_residual(order, r)
                if wr is not None and np.all(wr > 0):
                    roots.append(r)
            prev = (res, g)
        if roots:
            mu1 = max(roots)
        else:  # no moment root with positive weights: smallest residual
            best = None
            for g in grid:
                res, wc = _next_moment_residual(order, g)
                if res is None or not np.all(wc > 0):
                    continue
                if best is None or abs(res) < best[0]:
                    best = (abs(res), g)
            if best is None:
                raise ValueError(f"no positive level-symmetric S{order} set")
            mu1 = best[1]
    mu, pts, cls_of, wc = _ls_weights(order, mu1)
    dirs, wts = [], []
    for sx, sy, sz in itertools.product((1.0, -1.0), repeat=3):
        if dim == 2 and sz < 0:
            continue
        for p, c in zip(pts, cls_of):
            dirs.append((sx * mu[p[0] - 1], sy * mu[p[1] - 1], sz * mu[p[2] - 1]))
            wts.append(wc[c] * (2.0 if dim == 2 else 1.0))
    omega = np.asarray(dirs, dtype=np.float64)
    w = np.asarray(wts, dtype=np.float64)
    w *= FOUR_PI / w.sum()
    return np.ascontiguousarray(omega), np.ascontiguousarray(w)


# --------------------------------------------------------------------------
# problem descriptions
# --------------------------------------------------------------------------
@dataclass
class Problem:
    """One transport problem: points, extents, angular set, materials, steps."""
    name: str
    dim: int
    x: np.ndarray            # [n, dim]
    R: np.ndarray            # [n] kernel support radius (2 * spacing)
    omega: np.ndarray        # [m, 3]
    w: np.ndarray            # [m]
    sigma_t: np.ndarray      # [n]
    sigma_s: np.ndarray      # [n]
    q: np.ndarray            # [n] isotropic source per steradian
    dt: float
    steps: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    inflow: dict = field(default_factory=dict)   # face -> psi_b
    spacing: float = 0.0

    @property
    def n(self):
        return self.x.shape[0]

    @property
    def m(self):
        return self.omega.shape[0]


def make_problem(name: str, n_per_dim: int, dim: int, sn: int, seed: int,
                 sigma_t, sigma_s, q, dt: float, steps: int,
                 inflow=None, support: float = 2.0, jitter: float = 0.2):
    """Build a Problem on a jittered unit-box lattice.

    sigma_t / sigma_s / q are scalars or callables f(x[n, dim], rng) -> [n]
    evaluated at the points (constant over each point's cell).
    """
    x, h = jittered_lattice(n_per_dim, dim, seed, jitter=jitter)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    def ev(v, *extra):
        if callable(v):
            return np.ascontiguousarray(np.asarray(v(x, rng, *extra), dtype=np.float64))
        return np.full(x.shape[0], float(v))
    st = ev(sigma_t)
    ss = ev(sigma_s, st) if callable(sigma_s) else np.full(x.shape[0], float(sigma_s))
    qq = ev(q)
    omega, w = level_symmetric(sn, dim)
    return Problem(name=name, dim=dim, x=x, R=np.full(x.shape[0], support * h),
                   omega=omega, w=w, sigma_t=st, sigma_s=ss, q=qq, dt=dt,
                   steps=steps, inflow=dict(inflow or {}), spacing=h)


def small_2d(n_per_dim: int = 32, sn: int = 4, seed: int = 1000, steps: int = 10,
             dt: float = 0.01, sigma_t: float = 1.0, sigma_s: float = 0.5,
             q: float = 1.0, jitter: float = 0.2):
    """2D unit square, n_per_dim^2 jittered points, support 2h, linear RK,
    level-symmetric S_sn, uniform sigma_t / sigma_s / q, vacuum boundaries,
    c = 1, backward Euler.  Defaults: 32x32 points, S4 (12 directions),
    sigma_t = 1, sigma_s = 0.5, q = 1, dt = 0.01, 10 steps."""
    return make_problem(f"2d-{n_per_dim}x{n_per_dim}-S{sn}", n_per_dim, 2, sn, seed,
                        sigma_t, sigma_s, q, dt, steps, jitter=jitter)


def two_region_2d(n_per_dim: int = 256, sn: int = 8, seed: int = 2000, steps: int = 20,
                  dt: float = 0.005, ratio: float = 0.9):
    """2D unit square, jittered lattice, S_sn, sigma_t = 100 for points in the
    centred square [0.4, 0.6]^2 and 1 elsewhere, sigma_s = ratio * sigma_t,
    q = 1 for points with x < 0.5 and 0 elsewhere, vacuum boundaries.
    Defaults: 256x256 points, S8 (40 directions), 20 steps of dt = 0.005."""
    def st(x, rng):
        inside = np.all((x >= 0.4) & (x <= 0.6), axis=1)
        return np.where(inside, 100.0, 1.0)

    def ss(x, rng, sig_t):
        return ratio * sig_t

    def qq(x, rng):
        return np.where(x[:, 0] < 0.5, 1.0, 0.0)
    return make_problem(f"2d-two-region-{n_per_dim}x{n_per_dim}-S{sn}", n_per_dim, 2, sn,
                        seed, st, ss, qq, dt, steps)


def lognormal_3d(n_per_dim: int = 40, sn: int = 8, seed: int = 3000, steps: int = 10,
                 dt: float = 0.01, refine=None):
    """3D unit cube, jittered lattice, S_sn, sigma_t ~ lognormal(0, 1) per point,
    sigma_s = 0.8 sigma_t, no volume source, isotropic inflow psi_b = 1 on the
    x = 0 face.  Defaults: 40^3 points, S8 (80 directions), 10 steps of 0.01.
    refine = (min_level, goal_level, cone_deg) replaces S_sn by the selectively
    refined hierarchical quadrature of Alg. 2 around +x (the configuration's
    refinement within 15 degrees of +x: (1, 5, 15.0), 272 directions)."""
    def st(x, rng):
        return rng.lognormal(0.0, 1.0, size=x.shape[0])

    def ss(x, rng, sig_t):
        return 0.8 * sig_t
    p = make_problem(f"3d-lognormal-{n_per_dim}^3-S{sn}", n_per_dim, 3, sn, seed,
                     st, ss, 0.0, dt, steps, inflow={0: 1.0})
    if refine is not None:
        lo, goal, cone = refine
        p.omega, p.w = refined_quadrature(lo, goal, cone_hits((1.0, 0.0, 0.0), cone))
        p.name = f"3d-lognormal-{n_per_dim}^3-refined{lo}-{goal}-{cone:g}deg"
    return p


def batched_2d(count: int = 64, seed: int = 4000, n_range=(1024, 65536),
               sn_choices=(4, 6, 8, 10, 12), steps: int = 10, dt: float = 0.01):
    """Independent 2D problems for batched runs: per problem the point count is
    log-uniform in n_range (rounded to a k x k lattice), S_N is drawn from
    sn_choices, sigma_t is uniform in [0.1, 10] and the scattering ratio
    uniform in [0, 0.99] (both constant over the problem), q = 1, vacuum
    boundaries.  Problem b uses lattice seed seed + b; the draws come from
    numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(count):
        npts = np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))
        k = max(2, int(round(np.sqrt(npts))))
        sn = int(rng.choice(np.asarray(sn_choices)))
        sig_t = float(rng.uniform(0.1, 10.0))
        ratio = float(rng.uniform(0.0, 0.99))
        out.append(make_problem(f"2d-batch{b}-{k}x{k}-S{sn}", k, 2, sn, seed + b,
                                sig_t, ratio * sig_t, 1.0, dt, steps))
    return out


# ---------------------------------------------------------------------------
# hierarchical octant quadrature and selective refinement (Sec. 4.3, Alg. 2)
# ---------------------------------------------------------------------------
def _octant_triangles(level: int):
    """Spherical triangles of the unit sphere at a refinement level: the eight
    octants, each split `level` times into four by its normalised edge
    midpoints.  Children of triangle t are 4t .. 4t + 3, so the level-G
    descendants of a level-l triangle t are t 4^(G-l) .. (t + 1) 4^(G-l) - 1."""
    tris = []
    for sx in (1.0, -1.0):
        for sy in (1.0, -1.0):
            for sz in (1.0, -1.0):
                tris.append((np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, sz])))
    for _ in range(level):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (v / np.linalg.norm(v) for v in (a + b, b + c, c + a))
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nxt
    return tris


def _tri_ordinates(tris):
    """Ordinate (normalised vertex centroid) and weight (spherical area, by the
    Van Oosterom-Strackee formula) of each spherical triangle."""
    om = np.array([(a + b + c) / np.linalg.norm(a + b + c) for a, b, c in tris])
    w = np.array([2.0 * np.arctan2(abs(a @ np.cross(b, c)), 1.0 + a @ b + b @ c + c @ a) for a, b, c in tris])
    return om, w


def refined_quadrature(min_level: int, goal_level: int, hits):
    """Selective refinement of the hierarchical octant quadrature (Alg. 2):
    start from the goal level; for each coarser level from min_level up, an
    ordinate whose goal-level descendants all miss the object (hits(omega)
    False for each) and are all still unmerged replaces them; the goal
    ordinates left are kept.  Weights are exact spherical areas, so they sum
    to 4 pi.  Returns (omega[M, 3], w[M])."""
    G = goal_level
    gom, gw = _tri_ordinates(_octant_triangles(G))
    hit = np.array([bool(hits(o)) for o in gom])
    present = np.ones(len(gom), bool)
    om_out, w_out = [], []
    for lev in range(min_level, G):
        lom, lw = _tri_ordinates(_octant_triangles(lev))
        span = 4 ** (G - lev)
        for t in range(len(lom)):
            d = slice(t * span, (t + 1) * span)
            if present[d].all() and not hit[d].any():
                om_out.append(lom[t])
                w_out.append(lw[t])
                present[d] = False
    om_out += list(gom[present])
    w_out += list(gw[present])
    return np.array(om_out), np.array(w_out)


def cone_hits(axis=(1.0, 0.0, 0.0), half_angle_deg: float = 15.0):
    """Directions within half_angle_deg of axis."""
    ax = np.asarray(axis, float) / np.linalg.norm(axis)
    c = np.cos(np.radians(half_angle_deg))
    return lambda o: float(np.asarray(o) @ ax) >= c


# ---------------------------------------------------------------------------
# line source and absorbing disk (the asteroid problem, Sec. 5.4, scaled down)
# ---------------------------------------------------------------------------
def polar_product_quadrature(n_azimuth: int, n_polar: int):
    """Product set for line-source problems: in-plane lengths mu_k (the cosine
    of the angle to the x-y plane) at the Gauss-Legendre nodes of [0, 1] with
    weights a_k, times n_azimuth equally spaced azimuths (offset by half a
    spacing); Omega = (mu cos theta, mu sin theta, sqrt(1 - mu^2)).  The weight
    of an ordinate is 2 pi mu_k a_k / n_azimuth: with the azimuths resolved,
    the scalar flux of a unit line source is then sum_k a_k exp(-omega / mu_k) / r,
    the polar quadrature of the mu integral in App. B (which integrates over mu
    with unit measure).  Returns (omega[M, 3], w[M], mu[K], a[K])."""
    t, a = np.polynomial.legendre.leggauss(n_polar)
    mu, a = 0.5 * (t + 1.0), 0.5 * a
    th = (np.arange(n_azimuth) + 0.5) * (2.0 * math.pi / n_azimuth)
    om = np.array([[m * math.cos(p), m * math.sin(p), math.sqrt(1.0 - m * m)] for m in mu for p in th])
    w = np.repeat(2.0 * math.pi * mu * a / n_azimuth, n_azimuth)
    return om, w, mu, a


def asteroid_2d(n_per_dim: int = 32, n_azimuth: int = 64, n_polar: int = 2,
                sigma_background: float = 0.5, sigma_asteroid: float = 10.0,
                radius: float = 0.35, centre=(0.35, 0.0), source=(-0.55, 0.0),
                source_width: float = 0.1):
    """A scaled-down 2D asteroid problem on [-1, 1]^2: a disk of radius
    `radius` at `centre` with sigma_t = sigma_asteroid for the points inside it
    and sigma_background elsewhere, no scattering, an isotropic source
    q = exp(-|x - source|^2 / (2 source_width^2)) per point, cut to zero beyond
    three widths,
    vacuum boundaries, one steady step, the product set of
    polar_product_quadrature.  Regular lattice (no jitter), so every interior
    cell is an h x h square and a source point j carries q_j h^2.  Defaults:
    32x32 points, 64 azimuths x 2 polar levels, sigma 0.5 / 10, a disk 7 mean
    free paths across at 0.55 from a source of width 0.1.  The paper's problem
    (radius 35, source 70 from the surface, sigma 0.001 / 10, a shell with
    variable spacing and a refined 4,096-ordinate set) is not reproduced."""
    x, h = jittered_lattice(n_per_dim, 2, 0, lo=-1.0, hi=1.0, jitter=0.0)
    inside = np.linalg.norm(x - np.asarray(centre, np.float64), axis=1) < radius
    st = np.where(inside, float(sigma_asteroid), float(sigma_background))
    d2 = np.sum((x - np.asarray(source, np.float64)) ** 2, axis=1) / source_width ** 2
    q = np.where(d2 <= 9.0, np.exp(-0.5 * d2), 0.0)
    omega, w, _, _ = polar_product_quadrature(n_azimuth, n_polar)
    return Problem(name=f"2d-asteroid-{n_per_dim}x{n_per_dim}-A{n_azimuth}P{n_polar}", dim=2, x=x,
                   R=np.full(len(x), 2.0 * h), omega=omega, w=w, sigma_t=st, sigma_s=np.zeros(len(x)),
                   q=q, dt=math.inf, steps=1, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), spacing=h)


# ---------------------------------------------------------------------------
# request stream of the serving configuration
# ---------------------------------------------------------------------------
def serving_stream(count: int = 64, rate: float = 2.0, seed: int = 5000, n_range=(4096, 250000),
                   p3d: float = 0.25, sn_2d=(4, 6, 8, 10, 12), sn_3d=(4, 8, 12), p_refined: float = 0.25,
                   steps_range=(5, 50), dt: float = 0.01):
    """Arriving transport problems: a list of (Problem, arrival time).

    Arrivals are a Poisson process of the given rate (exponential gaps, the
    first one after a gap from time 0).  Per request, drawn from numpy
    PCG64(seed): dimension 3 with probability p3d, else 2; a point count
    log-uniform in n_range, rounded to a k^dim lattice; in 2D S_N from sn_2d
    (12 to 84 directions), in 3D the selectively refined set of Alg. 2 within
    15 degrees of +x (272 directions) with probability p_refined, else S_N from
    sn_3d (24 to 168); two regions, the centred box [0.4, 0.6]^dim and the
    rest, each with sigma_t log-uniform in [0.1, 100]; one scattering ratio
    uniform in [0, 0.99]; q = 1 for x_0 < 0.5; vacuum boundaries; steps
    uniform in steps_range (inclusive); backward-Euler step dt.  Problem b uses
    lattice seed seed + 1 + b."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    t = 0.0
    refined_set = None
    for b in range(count):
        t += rng.exponential(1.0 / rate)
        dim = 3 if rng.uniform() < p3d else 2
        npts = math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))
        k = max(2, int(round(npts ** (1.0 / dim))))
        refined = dim == 3 and rng.uniform() < p_refined
        sn = int(rng.choice(np.asarray(sn_2d if dim == 2 else sn_3d)))
        s_in, s_out = np.exp(rng.uniform(math.log(0.1), math.log(100.0), 2))
        ratio = float(rng.uniform(0.0, 0.99))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))

        def st(x, r, s_in=s_in, s_out=s_out):
            inside = np.all((x >= 0.4) & (x <= 0.6), axis=1)
            return np.where(inside, s_in, s_out)

        def ss(x, r, sig_t, ratio=ratio):
            return ratio * sig_t

        def qq(x, r):
            return np.where(x[:, 0] < 0.5, 1.0, 0.0)
        p = make_problem(f"serve{b}-{dim}d-{k}^{dim}", k, dim, sn, seed + 1 + b, st, ss, qq, dt, steps)
        if refined:
            if refined_set is None:
                refined_set = refined_quadrature(1, 5, cone_hits((1.0, 0.0, 0.0), 15.0))
            p.omega, p.w = refined_set[0].copy(), refined_set[1].copy()
            p.name += "-refined"
        out.append((p, t))
    return out
