"""Autotuner for the tile shape of the batched FP32 transport-operator apply.

The tiled L-apply (Sec. 4.2, operator L for all directions at once) has two
shape parameters: rows per tile (32 or 64) and directions per thread (4 or 8,
dividing m); its tensor-core variant (m % 8 == 0) has the rows per tile; the
row-team kernel is the alternative for any m.  Which is
fastest depends on the dimension (stencil size, halo) and on the number of
directions m, so this module times every candidate on the problem's own
operators (CUDA events on the library stream, inputs resident, after warm-up)
and keeps the fastest per (dim, m) in a JSON cache:

    choice = tuned_options(prob)          # {"apply_kernel": ..., "tile_rows": ..., "tile_dpt": ...}
    TransportProblem.from_problem(prob, precision=MLPG_MIXED, **choice)

The cache file is $MLPG_TUNE_CACHE, else ~/.cache/mlpg/apply_tiles.json.
Every timing goes through the C ABI (mlpg_apply_L_dev); nothing here
computes the operator.
"""
from __future__ import annotations

import json
import os
import statistics

from . import MLPG_ERR_ARG, MLPG_MIXED, MlpgError, TransportProblem, mlpg_apply_L_dev


def cache_path() -> str:
    return os.environ.get("MLPG_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "mlpg",
                                                            "apply_tiles.json")


def candidates(m: int):
    """Every apply configuration the library accepts for m directions."""
    out = [{"apply_kernel": 1, "tile_rows": 0, "tile_dpt": 0}]
    if m % 8 == 0:
        for rows in (64, 32):
            out.append({"apply_kernel": 3, "tile_rows": rows, "tile_dpt": 0})
    if m % 4 == 0:
        for dpt in (8, 4):
            if m % dpt:
                continue
            for rows in (64, 32):
                out.append({"apply_kernel": 2, "tile_rows": rows, "tile_dpt": dpt})
            for rows in (32, 16, 8, 4):
                out.append({"apply_kernel": 4, "tile_rows": rows, "tile_dpt": dpt})
    return out


def _key(dim: int, m: int) -> str:
    return f"dim{dim}-m{m}"


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, entry: dict) -> None:
    c = load_cache()
    c[key] = entry
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_apply(prob, options: dict, reps: int = 20, warmup: int = 5, stream=None):
    """Median device time (us) of one batched FP32 L-apply of `prob` with
    `options`, and the statistics the library reports for that context."""
    import torch
    if stream is None or stream.cuda_stream == 0:
        # the library runs on the stream it is given, or on its own when given the null stream:
        # time on a stream of ours so that the events bracket its kernels
        stream = torch.cuda.Stream()
    with TransportProblem.from_problem(prob, precision=MLPG_MIXED, stream=stream.cuda_stream, **options) as tp:
        tp.integrate().assemble()
        X = torch.rand(prob.n, prob.m, device=stream.device, dtype=torch.float32)
        Y = torch.empty_like(X)
        torch.cuda.synchronize()   # X is written on the current stream, read on `stream`
        for _ in range(warmup):
            mlpg_apply_L_dev(tp.ctx, prob.dt, MLPG_MIXED, X.data_ptr(), Y.data_ptr())
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mlpg_apply_L_dev(tp.ctx, prob.dt, MLPG_MIXED, X.data_ptr(), Y.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(1e3 * e0.elapsed_time(e1))
        return statistics.median(times), tp.stats()


def tune(prob, reps: int = 20, warmup: int = 5, stream=None, store: bool = True, cands=None):
    """Time every candidate on `prob`; returns (best options, table of
    {config, us, apply_kernel used, chunk, max halo}).  A candidate the
    library turns down is skipped: a tile shape whose context falls back to
    the row-team kernel, or one the apply refuses with MLPG_ERR_ARG (no
    direction chunk fits shared memory)."""
    table = []
    for opt in (cands if cands is not None else candidates(prob.m)):
        try:
            us, st = time_apply(prob, opt, reps, warmup, stream)
        except MlpgError as e:
            if e.status != MLPG_ERR_ARG:   # only a shape the library turns down is skipped
                raise
            continue
        if opt["apply_kernel"] >= 2 and st["apply_kernel"] != opt["apply_kernel"]:
            continue
        table.append({**opt, "us": us, "tile_chunk": st["tile_chunk"], "tile_max_halo": st["tile_max_halo"]})
    best = min(table, key=lambda r: r["us"])
    choice = {k: best[k] for k in ("apply_kernel", "tile_rows", "tile_dpt")}
    if store:
        _store(_key(prob.dim, prob.m), {"choice": choice, "n": int(prob.n), "table": table})
    return choice, table


def tuned_options(prob, **kw) -> dict:
    """The cached choice for (prob.dim, prob.m); tunes on `prob` first when
    the cache has none."""
    hit = load_cache().get(_key(prob.dim, prob.m))
    if hit:
        return dict(hit["choice"])
    return tune(prob, **kw)[0]


def problem_key(prob) -> str:
    return _key(prob.dim, prob.m)


__all__ = ["candidates", "tune", "tuned_options", "time_apply", "cache_path", "load_cache", "problem_key"]
