"""GB300 (sm_103a) library for the time-dependent discrete-ordinates transport
solve on a meshless MLPG / reproducing-kernel / Voronoi-cell discretisation
(Bassett & Owen, arXiv 2008.02205).

The compute lives in ``libmlpg.so`` (hand-written CUDA behind the C ABI of
``include/mlpg.h``).  This module only marshals arguments: the functions
``mlpg_*`` below have the names and arguments of the C entry points, and
``TransportProblem`` is a small convenience wrapper over them.  There is no
CPU fallback: importing the binding without a built library, or calling it
without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlpg.so")

MLPG_OK = 0
STATUS = {0: "MLPG_OK", -1: "MLPG_ERR_ARG", -2: "MLPG_ERR_STATE", -3: "MLPG_ERR_OOM", -4: "MLPG_ERR_CUDA",
          -5: "MLPG_ERR_GEOMETRY", -6: "MLPG_ERR_RK_SINGULAR", -7: "MLPG_ERR_NOT_CONVERGED"}
(MLPG_ERR_ARG, MLPG_ERR_STATE, MLPG_ERR_OOM, MLPG_ERR_CUDA, MLPG_ERR_GEOMETRY, MLPG_ERR_RK_SINGULAR,
 MLPG_ERR_NOT_CONVERGED) = range(-1, -8, -1)
MLPG_FP64 = 0
MLPG_MIXED = 1


class MlpgError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


class Options(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("tau_factor", ctypes.c_double), ("c", ctypes.c_double), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("outer_tol", ctypes.c_double),
                ("inner_restart", ctypes.c_int), ("outer_restart", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("mixed_inner_tol", ctypes.c_double), ("check_every", ctypes.c_int),
                ("mixed_restart", ctypes.c_int), ("mixed_reorth", ctypes.c_int),
                ("mixed_half_prec", ctypes.c_int), ("outer_method", ctypes.c_int), ("rk_order", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("apply_kernel", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("tile_dpt", ctypes.c_int), ("outer_precond", ctypes.c_int),
                ("dsa_tol", ctypes.c_double), ("dsa_max", ctypes.c_int), ("cells_3d", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("m", ctypes.c_int32),
                ("n_volume_qp", ctypes.c_int64), ("n_boundary_qp", ctypes.c_int64),
                ("steps", ctypes.c_int32), ("last_outer_iters", ctypes.c_int32),
                ("last_inner_iters", ctypes.c_int64), ("last_inner_solves", ctypes.c_int32),
                ("last_refinements", ctypes.c_int32), ("last_residual", ctypes.c_double),
                ("total_outer_iters", ctypes.c_int64), ("total_inner_iters", ctypes.c_int64),
                ("spmm_launches", ctypes.c_int64), ("spmm_ms", ctypes.c_double),
                ("spmm_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("apply_kernel", ctypes.c_int32), ("tile_chunk", ctypes.c_int32),
                ("tile_max_halo", ctypes.c_int64), ("last_dsa_iters", ctypes.c_int64),
                ("total_dsa_iters", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p


def load_library(path: str = LIB_PATH):
    """Load libmlpg.so (built by ``paper_2008_02205_gb300.build``).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2008_02205_gb300.build` "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "mlpg_default_options": (None, [_P]),
        "mlpg_create": (i32, [_P, i64, _P, _P, i32, _P, _P, _P, _P, _P, _P]),
        "mlpg_create_dev": (i32, [_P, i64, _P, _P, i32, _P, _P, _P, _P, _P, _P]),
        "mlpg_set_inflow": (i32, [_P, ctypes.c_int, dbl]),
        "mlpg_set_initial": (i32, [_P, _P]),
        "mlpg_integrate": (i32, [_P]),
        "mlpg_assemble": (i32, [_P]),
        "mlpg_step": (i32, [_P, dbl]),
        "mlpg_step_batch": (i32, [_P, _P, ctypes.c_int, _P]),
        "mlpg_scalar_flux": (i32, [_P, _P, ctypes.c_int]),
        "mlpg_scalar_flux_dev": (i32, [_P, _P, ctypes.c_int]),
        "mlpg_get_state": (i32, [_P, _P]),
        "mlpg_set_state": (i32, [_P, _P]),
        "mlpg_get_stats": (i32, [_P, _P]),
        "mlpg_enable_timing": (i32, [_P, ctypes.c_int]),
        "mlpg_get_neighbors": (i32, [_P, _P, _P]),
        "mlpg_get_volumes": (i32, [_P, _P]),
        "mlpg_n_matrices": (ctypes.c_int, [ctypes.c_int]),
        "mlpg_n_vectors": (ctypes.c_int, [ctypes.c_int]),
        "mlpg_get_forms": (i32, [_P, _P, _P]),
        "mlpg_apply_L_dev": (i32, [_P, dbl, ctypes.c_int, _P, _P]),
        "mlpg_overlap_counts_noalloc": (i32, [ctypes.c_int, i64, _P, _P, _P, _P, _P, _P]),
        "mlpg_set_reduce": (i32, [_P, _P, _P]),
        "mlpg_last_error": (ctypes.c_char_p, [_P]),
        "mlpg_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


def _arr(a, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _check(ctx, status):
    if status != MLPG_OK:
        msg = load_library().mlpg_last_error(ctx) if ctx else b""
        raise MlpgError(status, (msg or b"").decode())


# ---- thin wrappers with the C names (marshalling only) --------------------
def mlpg_default_options(**overrides) -> Options:
    o = Options()
    load_library().mlpg_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k in ("lo", "hi"):
            getattr(o, k)[:] = list(v) + [0.0] * (3 - len(v))
        else:
            setattr(o, k, v)
    return o


def _check_shapes(dim, x, R, om, ww, st, ss, qq):
    """The C side reads n * dim, n, 3 m and m values from these pointers."""
    if x.ndim != 2 or x.shape[1] != dim:
        raise ValueError(f"points must be [n, {dim}], got {x.shape}")
    if om.ndim != 2 or om.shape[1] != 3:
        raise ValueError(f"omega must be [m, 3], got {om.shape}")
    n, m = x.shape[0], om.shape[0]
    for name, a, k in (("kernel_extent", R, n), ("w", ww, m), ("sigma_t", st, n), ("sigma_s", ss, n), ("q", qq, n)):
        if a.shape != (k,):
            raise ValueError(f"{name} must have shape ({k},), got {a.shape}")


def _state_size(ctx):
    s = mlpg_get_stats(ctx)
    return s["n"] * s["m"]


def mlpg_create(opt: Options, points, kernel_extent, omega, w, sigma_t, sigma_s, q):
    x, R, om, ww, st, ss, qq = (_arr(a) for a in (points, kernel_extent, omega, w, sigma_t, sigma_s, q))
    _check_shapes(opt.dim, x, R, om, ww, st, ss, qq)
    ctx = _P()
    s = load_library().mlpg_create(ctypes.byref(opt), x.shape[0], _ptr(x), _ptr(R), om.shape[0], _ptr(om),
                                   _ptr(ww), _ptr(st), _ptr(ss), _ptr(qq), ctypes.byref(ctx))
    if s != MLPG_OK:
        if ctx:
            msg = load_library().mlpg_last_error(ctx)
            load_library().mlpg_destroy(ctx)
            raise MlpgError(s, (msg or b"").decode())
        raise MlpgError(s, "create failed")
    return ctx


def mlpg_create_dev(opt: Options, n, m, points_ptr, extent_ptr, omega_ptr, w_ptr, st_ptr, ss_ptr, q_ptr):
    """Device-pointer create: every *_ptr is an integer device address (e.g. tensor.data_ptr())."""
    ctx = _P()
    s = load_library().mlpg_create_dev(ctypes.byref(opt), n, points_ptr, extent_ptr, m, omega_ptr, w_ptr,
                                       st_ptr, ss_ptr, q_ptr, ctypes.byref(ctx))
    if s != MLPG_OK:
        if ctx:
            msg = load_library().mlpg_last_error(ctx)
            load_library().mlpg_destroy(ctx)
            raise MlpgError(s, (msg or b"").decode())
        raise MlpgError(s, "create failed")
    return ctx


def mlpg_set_inflow(ctx, face, psi_b):
    _check(ctx, load_library().mlpg_set_inflow(ctx, face, psi_b))


def mlpg_set_initial(ctx, psi0=None):
    a = None if psi0 is None else _arr(psi0)
    if a is not None and a.size != _state_size(ctx):
        raise ValueError(f"psi0 must hold n * m = {_state_size(ctx)} values, got {a.size}")
    _check(ctx, load_library().mlpg_set_initial(ctx, _ptr(a)))


def mlpg_integrate(ctx):
    _check(ctx, load_library().mlpg_integrate(ctx))


def mlpg_assemble(ctx):
    _check(ctx, load_library().mlpg_assemble(ctx))


def mlpg_step(ctx, dt):
    _check(ctx, load_library().mlpg_step(ctx, dt))


def mlpg_step_batch(ctxs, dts, raise_on_error=True):
    """One step of each context, run concurrently (distinct contexts and
    streams).  Returns every context's own status (0 = done); a failure raises
    MlpgError naming the failed contexts unless raise_on_error is False.  An
    argument error of the whole call (no step taken) always raises."""
    k = len(ctxs)
    arr = (_P * max(k, 1))(*ctxs)
    d = _arr(np.broadcast_to(np.asarray(dts, dtype=np.float64), (k,)))
    unwritten = 1                                   # not a status value
    out = (ctypes.c_int * max(k, 1))(*([unwritten] * max(k, 1)))
    st = load_library().mlpg_step_batch(arr, _ptr(d), k, out)
    each = [int(out[i]) for i in range(k)]
    if st != MLPG_OK and (k == 0 or each[0] == unwritten):
        raise MlpgError(st, "; ".join(m for m in (mlpg_last_error(c) for c in ctxs if c) if m) or "bad batch")
    if st != MLPG_OK and raise_on_error:
        raise MlpgError(st, "; ".join(f"[{i}] {mlpg_last_error(c)}" for i, (c, s) in enumerate(zip(ctxs, each)) if s))
    return each


def mlpg_scalar_flux(ctx, n, kind=0):
    out = np.zeros(n)
    _check(ctx, load_library().mlpg_scalar_flux(ctx, _ptr(out), kind))
    return out


def mlpg_scalar_flux_dev(ctx, out_ptr, kind=0):
    _check(ctx, load_library().mlpg_scalar_flux_dev(ctx, out_ptr, kind))


def mlpg_get_state(ctx, n, m):
    out = np.zeros((n, m))
    _check(ctx, load_library().mlpg_get_state(ctx, _ptr(out)))
    return out


def mlpg_set_state(ctx, psi):
    a = _arr(psi)
    if a.size != _state_size(ctx):
        raise ValueError(f"psi must hold n * m = {_state_size(ctx)} values, got {a.size}")
    _check(ctx, load_library().mlpg_set_state(ctx, _ptr(a)))


def mlpg_get_stats(ctx) -> dict:
    st = Stats()
    _check(ctx, load_library().mlpg_get_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def mlpg_enable_timing(ctx, on=True):
    _check(ctx, load_library().mlpg_enable_timing(ctx, int(on)))


def mlpg_get_neighbors(ctx, n, nnz):
    rowptr = np.zeros(n + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    _check(ctx, load_library().mlpg_get_neighbors(ctx, _ptr(rowptr), _ptr(col)))
    return rowptr, col


def mlpg_get_volumes(ctx, n):
    out = np.zeros(n)
    _check(ctx, load_library().mlpg_get_volumes(ctx, _ptr(out)))
    return out


def mlpg_n_matrices(dim=2):
    return load_library().mlpg_n_matrices(dim)


def mlpg_n_vectors(dim=2):
    return load_library().mlpg_n_vectors(dim)


def mlpg_get_forms(ctx, n, nnz, dim=2):
    mats = np.zeros((mlpg_n_matrices(dim), nnz))
    vecs = np.zeros((mlpg_n_vectors(dim), n))
    _check(ctx, load_library().mlpg_get_forms(ctx, _ptr(mats), _ptr(vecs)))
    return mats, vecs


def mlpg_apply_L_dev(ctx, dt, precision, x_ptr, y_ptr):
    _check(ctx, load_library().mlpg_apply_L_dev(ctx, dt, precision, x_ptr, y_ptr))


def mlpg_overlap_counts_noalloc(dim, n, points_ptr, extent_ptr, lo, hi, counts_ptr, stream=None):
    """Row sizes of the overlap pattern into a device int32 buffer, without any
    device allocation (device pointers in and out; lo/hi are host sequences).
    Returns the status code (0 on success); the work is queued on `stream`."""
    lo_a = _arr(list(lo)[:dim])
    hi_a = _arr(list(hi)[:dim])
    return load_library().mlpg_overlap_counts_noalloc(dim, n, points_ptr, extent_ptr, _ptr(lo_a), _ptr(hi_a),
                                                      counts_ptr, stream)


# cross-shard sum callback: int fn(double *buf, int64_t count, void *user)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p)


def mlpg_set_reduce(ctx, fn):
    """Install a cross-shard sum (a REDUCE_FN object, kept alive by the
    caller) or remove it (None)."""
    ptr = ctypes.cast(fn, _P) if fn is not None else None
    _check(ctx, load_library().mlpg_set_reduce(ctx, ptr, None))


def mlpg_last_error(ctx):
    return (load_library().mlpg_last_error(ctx) or b"").decode()


def mlpg_destroy(ctx):
    if ctx:
        load_library().mlpg_destroy(ctx)


class TransportProblem:
    """Owns one context: create -> integrate -> assemble -> step* -> flux."""

    def __init__(self, points, kernel_extent, omega, w, sigma_t, sigma_s, q, inflow=None, **options):
        self.n, self.dim = (int(v) for v in np.asarray(points).shape)
        self.m = int(np.asarray(omega).shape[0])
        options.setdefault("dim", self.dim)
        self.opt = mlpg_default_options(**options)
        self.ctx = mlpg_create(self.opt, points, kernel_extent, omega, w, sigma_t, sigma_s, q)
        for f, v in (inflow or {}).items():
            mlpg_set_inflow(self.ctx, int(f), float(v))

    @classmethod
    def from_problem(cls, prob, **options):
        """From an ``mlpg_inputs.Problem`` (its box unless lo / hi are given)."""
        for key in ("lo", "hi"):
            if getattr(prob, key, None) is not None:
                options.setdefault(key, tuple(getattr(prob, key)))
        return cls(prob.x, prob.R, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q,
                   inflow=prob.inflow, **options)

    def integrate(self):
        mlpg_integrate(self.ctx)
        self.nnz = self.stats()["nnz"]
        return self

    def assemble(self):
        mlpg_assemble(self.ctx)
        return self

    def step(self, dt):
        mlpg_step(self.ctx, dt)

    def run(self, dt, steps):
        for _ in range(steps):
            mlpg_step(self.ctx, dt)
        return self.scalar_flux()

    @staticmethod
    def step_batch(problems, dt):
        """One step of each TransportProblem, concurrently on their own streams."""
        mlpg_step_batch([p.ctx for p in problems], dt)

    def scalar_flux(self, kind=0):
        return mlpg_scalar_flux(self.ctx, self.n, kind)

    def state(self):
        return mlpg_get_state(self.ctx, self.n, self.m)

    def set_state(self, psi):
        mlpg_set_state(self.ctx, psi)

    def stats(self):
        return mlpg_get_stats(self.ctx)

    def neighbors(self):
        return mlpg_get_neighbors(self.ctx, self.n, self.stats()["nnz"])

    def volumes(self):
        return mlpg_get_volumes(self.ctx, self.n)

    def forms(self):
        return mlpg_get_forms(self.ctx, self.n, self.stats()["nnz"], self.dim)

    def close(self):
        if self.ctx:
            mlpg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


FOUR_PI = 4.0 * math.pi
