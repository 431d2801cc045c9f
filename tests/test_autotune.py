"""The apply autotuner's host logic on the CPU, with a fake timer in place of
the GPU: which shapes it tries for a direction count, that it keeps the
fastest, that it skips shapes the library turns down (a context that falls
back to row teams, an apply refused with MLPG_ERR_ARG) and re-raises any
other error, and that its cache round-trips through the file it names."""
import types

import pytest

import paper_2008_02205_gb300 as pkg
from paper_2008_02205_gb300 import autotune


def test_candidates_follow_the_divisibility_of_m():
    assert autotune.candidates(42) == [{"apply_kernel": 1, "tile_rows": 0, "tile_dpt": 0}]
    c12 = autotune.candidates(12)   # m % 4 == 0 only: CUDA-core tiles with 4 directions per thread
    assert {(o["apply_kernel"], o["tile_dpt"]) for o in c12} == {(1, 0), (2, 4), (4, 4)}
    c40 = autotune.candidates(40)   # m % 8 == 0: tensor-core tiles and both thread widths
    kinds = {(o["apply_kernel"], o["tile_rows"], o["tile_dpt"]) for o in c40}
    gather = {(4, r, d) for r in (32, 16, 8, 4) for d in (8, 4)}
    assert {(3, 64, 0), (3, 32, 0), (2, 64, 8), (2, 32, 8), (2, 64, 4), (2, 32, 4), (1, 0, 0)} | gather == kinds


def _fake(times, refuse=(), fallback=(), other=()):
    def time_apply(prob, opt, reps, warmup, stream):
        key = (opt["apply_kernel"], opt["tile_rows"], opt["tile_dpt"])
        if key in refuse:
            raise pkg.MlpgError(pkg.MLPG_ERR_ARG, "no direction chunk fits shared memory")
        if key in other:
            raise pkg.MlpgError(pkg.MLPG_ERR_CUDA, "launch failed")
        used = 1 if key in fallback else opt["apply_kernel"]
        return times[key], {"apply_kernel": used, "tile_chunk": 40, "tile_max_halo": 100}
    return time_apply


def test_tune_keeps_the_fastest_and_skips_what_the_library_turns_down(monkeypatch, tmp_path):
    monkeypatch.setenv("MLPG_TUNE_CACHE", str(tmp_path / "tune.json"))
    times = {(1, 0, 0): 100.0, (3, 64, 0): 50.0, (3, 32, 0): 60.0, (2, 64, 8): 70.0, (2, 32, 8): 65.0,
             (2, 64, 4): 80.0, (2, 32, 4): 75.0}
    times.update({(4, r, d): 90.0 + r / 8 + d for r in (32, 16, 8, 4) for d in (8, 4)})
    prob = types.SimpleNamespace(m=40, dim=3, n=64000)
    # the fastest shape (3, 64) is refused, the next (3, 32) falls back to row teams
    monkeypatch.setattr(autotune, "time_apply", _fake(times, refuse={(3, 64, 0)}, fallback={(3, 32, 0)}))
    choice, table = autotune.tune(prob)
    assert choice == {"apply_kernel": 2, "tile_rows": 32, "tile_dpt": 8}
    assert {(r["apply_kernel"], r["tile_rows"], r["tile_dpt"]) for r in table} == \
        {(1, 0, 0), (2, 64, 8), (2, 32, 8), (2, 64, 4), (2, 32, 4)} | {(4, r, d) for r in (32, 16, 8, 4) for d in (8, 4)}
    cached = autotune.load_cache()["dim3-m40"]
    assert cached["choice"] == choice and cached["n"] == 64000


def test_tune_reraises_errors_other_than_a_refused_shape(monkeypatch, tmp_path):
    monkeypatch.setenv("MLPG_TUNE_CACHE", str(tmp_path / "tune.json"))
    times = {(1, 0, 0): 100.0, (2, 64, 4): 80.0, (2, 32, 4): 75.0, (4, 32, 4): 90.0, (4, 16, 4): 91.0,
             (4, 8, 4): 92.0, (4, 4, 4): 93.0}
    prob = types.SimpleNamespace(m=12, dim=2, n=4096)
    monkeypatch.setattr(autotune, "time_apply", _fake(times, other={(2, 32, 4)}))
    with pytest.raises(pkg.MlpgError):
        autotune.tune(prob)
