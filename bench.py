"""Benchmark: time-dependent discrete-ordinates solves per second on one GB300.

One bench step is one whole solve of the two-region problem through the C ABI:
create (inputs already in HBM) -> integrate (neighbours, cells, quadrature,
RK interpolation) -> assemble (all forms) -> 20 backward-Euler steps (nested
GMRES, mixed precision with FP64 refinement by default) -> scalar flux.

Workload: 2D unit square, 256x256 jittered points (support 2h, linear RK),
level-symmetric S8 (40 directions), sigma_t = 100 in [0.4,0.6]^2 and 1
elsewhere, sigma_s = 0.9 sigma_t, q = 1 for x < 0.5, vacuum boundaries,
dt = 0.005, 20 steps.  Synthetic, seeded inputs (numpy PCG64).

Prints one JSON line.  `--impl reference` times the CPU oracle instead, on a
bounded sample of the same workload (see `_reference`).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "2d-two-region-256x256-S8-20steps"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=256, help="points per side (default: the 256x256 workload)")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-pointer end-to-end solves")
    ap.add_argument("--mode", default="solve", choices=["solve", "apply", "apply3d"],
                    help="solve: whole solves (the benchmark); apply: only the batched L-apply of the "
                         "workload, timed per launch (used for kernel profiles); apply3d: the same for the "
                         "3D configuration (lognormal sigma, the Alg. 2 set refined within 15 degrees of +x)")
    ap.add_argument("--side3", type=int, default=40, help="apply3d: points per side (default 40)")
    ap.add_argument("--be-steps", type=int, default=None,
                    help="backward-Euler steps per solve (default: the workload's 20; profiling runs use fewer)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra measurements (3D apply, serving stream, batched problems)")
    ap.add_argument("--no-tune", action="store_true", help="default tile shape instead of the autotuned one")
    return ap.parse_args()


def _max_over_ranks(x, world, device=None):
    """The largest x over all ranks (a job takes as long as its slowest rank);
    x itself when there is one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(world, solves_per_rank, seconds):
    """Whole-job solves/s: every rank solved solves_per_rank problems of its own
    (weak scaling) in `seconds`, the slowest rank's time."""
    return world * solves_per_rank / seconds


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = []
        reasons = set()
        smax = None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


PROFILE = os.path.join(ROOT, "profiles", "k_spmm32_tile-2d-two-region-256x256-S8.md")
APPLY_KERNELS = {1: "k_spmm32 (row teams)", 2: "k_spmm32_tile (row tiles, TMA-staged)",
                 3: "k_spmm32_mma (row tiles, tensor cores)",
                 4: "k_spmm32_tile (row tiles, gather mode)"}
KERNEL_SRC = os.path.join(ROOT, "paper_2008_02205_gb300", "csrc", "operators.cu")
# FP32 FMA peak of the GB300 (TFMA/s): 152 SMs x 128 FP32 lanes x 2.07 GHz maximum SM clock
FP32_FMA_PEAK_T = 152 * 128 * 2.07e9 / 1e12


def _traffic():
    """DRAM bytes per launch of the FP32 L-apply from the committed ncu summary,
    or None when the kernel source changed since that capture."""
    import hashlib
    try:
        txt = open(PROFILE).read()
        src = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().lstrip("-* ").startswith(("traffic_bytes_per_launch", "source_sha256")):
            k, v = line.split(":", 1)
            vals[k.strip(" -`*")] = v.strip(" `*")
    if vals.get("source_sha256") != src:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


SAMPLE_SIDE = 48


def _oracle_sample(reps=1):
    """CPU oracle on a bounded sample of the workload: the same two-region S8
    recipe at 48x48 points (about 28x fewer unknowns), one whole 20-step solve,
    as it stands (exact sparse-LU inner solves, unpreconditioned outer GMRES).
    solves/s is scaled to the 256x256 workload by the ratio of unknowns."""
    import oracle.mlpg_oracle as O
    import mlpg_inputs as mi
    prob = mi.two_region_2d(n_per_dim=SAMPLE_SIDE)
    times = []
    cpu = 0.0
    for _ in range(max(reps, 1)):
        c0, t0 = time.process_time(), time.perf_counter()
        O.solve_problem(prob, outer_tol=1e-12)
        times.append(time.perf_counter() - t0)
        cpu += time.process_time() - c0
    scale = (SAMPLE_SIDE * SAMPLE_SIDE) / (256 * 256)
    sample_s = statistics.median(times)
    value = scale / sample_s
    # threads the oracle kept busy: process CPU time over wall time (its sparse
    # LU and sparse products run on one thread; BLAS pools may hold more idle)
    cores = max(1, round(cpu / sum(times)))
    return {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{SAMPLE_SIDE}x{SAMPLE_SIDE} points, same recipe, full 20-step solve, "
                      f"{sample_s:.2f} s each, {cpu / sum(times):.2f} cores busy on average; "
                      f"scaled by unknowns {SAMPLE_SIDE**2}/65536"}


def _reference(args):
    cb = _oracle_sample(args.steps)
    value = cb["value"]
    line = {"metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": 0, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": f"{SAMPLE_SIDE}x{SAMPLE_SIDE}"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _apply_mode(args, pkg, prob, prec, opts, dv, stream, world, rank, workload=WORKLOAD):
    """Time the batched L-apply alone on the workload's operators (one launch
    per step, CUDA events on the library stream); used for kernel profiles.
    3D: reported against the FP32 FMA peak (ten FMAs per entry and direction),
    with the HBM figures beside it."""
    import torch
    o = pkg.mlpg_default_options(**opts)
    ctx = pkg.mlpg_create_dev(o, prob.n, prob.m, dv["x"].data_ptr(), dv["R"].data_ptr(), dv["om"].data_ptr(),
                              dv["w"].data_ptr(), dv["st"].data_ptr(), dv["ss"].data_ptr(), dv["q"].data_ptr())
    try:
        pkg.mlpg_integrate(ctx)
        pkg.mlpg_assemble(ctx)
        dt = torch.float32 if prec == pkg.MLPG_MIXED else torch.float64
        X = torch.rand(prob.n, prob.m, device=stream.device, dtype=dt)
        Y = torch.empty_like(X)
        for _ in range(args.warmup):
            pkg.mlpg_apply_L_dev(ctx, prob.dt, prec, X.data_ptr(), Y.data_ptr())
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pkg.mlpg_apply_L_dev(ctx, prob.dt, prec, X.data_ptr(), Y.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        st = pkg.mlpg_get_stats(ctx)
    finally:
        pkg.mlpg_destroy(ctx)
    us = 1e3 * statistics.median(times)
    hbm, kind = _peaks()
    gbs = st["spmm_bytes"] / (us * 1e-6) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "peak_kind": kind,
            "bytes_per_launch": st["spmm_bytes"]}
    if prob.dim == 3 and prec == pkg.MLPG_MIXED:
        tfma = 10.0 * st["nnz"] * prob.m / (us * 1e-6) / 1e12
        roof = {"bound": "alu", "achieved": tfma, "peak": FP32_FMA_PEAK_T, "unit": "TFMA/s",
                "frac": tfma / FP32_FMA_PEAK_T, "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                "hbm": {"achieved_gbs": gbs, "frac": gbs / hbm, "bytes_per_launch": st["spmm_bytes"]}}
    if rank == 0:
        print(json.dumps({"metric": "batched L-apply", "value": us, "unit": "us/launch", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                          "dtype": "f32" if prec == pkg.MLPG_MIXED else "f64",
                          "config": {"workload": workload, "mode": args.mode, "points": prob.n,
                                     "directions": prob.m, "nnz": st["nnz"],
                                     "apply_kernel": st["apply_kernel"], "tile_chunk": st["tile_chunk"],
                                     "options": {k: opts.get(k) for k in ("apply_kernel", "tile_rows", "tile_dpt")}},
                          "roofline": roof}))


GOLDEN = os.path.join(ROOT, "tests", "golden", "two_region_256_phi.npz")


def _golden():
    """The oracle's scalar flux of the full workload (written by
    tests/golden/make_two_region_256_golden.py), or None."""
    try:
        return np.load(GOLDEN)
    except OSError:
        return None


def _oracle_counts(side=24, steps=2):
    """The oracle's own inner scheme (GMRES + ILUT per direction, the paper's
    Sec. 4.2 solver) on a sample of the workload: iterations per inner solve
    and outer iterations per step."""
    import oracle.mlpg_oracle as O
    import mlpg_inputs as mi
    prob = mi.two_region_2d(n_per_dim=side, steps=steps)
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
    sol = O.Solver(tr, outer_tol=1e-12, inner="ilut-gmres", inner_tol=1e-12)
    _, _, st = sol.run(np.zeros((tr.M, disc.n)), prob.dt, prob.steps)
    c = [k for k in sol.inner_counts if k > 0]
    return {"sample": f"{side}x{side} points, {steps} steps, inner GMRES(50) + ILUT(1e-4, fill 10) to 1e-12, "
                      f"outer GMRES to 1e-12",
            "inner_per_solve": float(np.mean(c)) if c else 0.0,
            "outer_per_step": float(np.mean([x.outer_iterations for x in st]))}


def _apply_3d(pkg, stream):
    """Batched FP32 L-apply of the 3D configuration (40^3 points, the Alg. 2
    set refined within 15 degrees of +x: 272 directions), automatic kernel
    choice; algorithmic bytes per launch over the median event time."""
    import mlpg_inputs as mi
    from paper_2008_02205_gb300 import autotune
    prob = mi.lognormal_3d(refine=(1, 5, 15.0))
    us, st = autotune.time_apply(prob, {}, reps=10, warmup=3, stream=stream)
    hbm, kind = _peaks()
    gbs = st["spmm_bytes"] / (us * 1e-6) / 1e9
    # FP32 FMAs: nine to combine the ten base arrays per entry and direction, one with X
    fmas = 10.0 * st["nnz"] * prob.m
    tfma = fmas / (us * 1e-6) / 1e12
    return {"workload": "3d-lognormal-40^3-refined272", "us_per_launch": us, "bytes_per_launch": st["spmm_bytes"],
            "achieved_gbs": gbs, "frac": gbs / hbm, "peak": hbm, "peak_kind": kind,
            "fma_tfma_s": tfma, "fma_frac": tfma / FP32_FMA_PEAK_T,
            "kernel": APPLY_KERNELS.get(st["apply_kernel"], "k_spmm32"),
            "tile_chunk": st["tile_chunk"], "nnz": st["nnz"]}


def _serving(pkg, count=10, rates=(2.0, 8.0)):
    """The serving configuration on a bounded sample: a Poisson stream of 2D
    and 3D requests (4k-64k points here, 12-272 directions, two-region
    sigma_t, 5-20 steps), admitted by estimated device memory, continuous
    batching; p50/p99 latency from arrival and solves/s at two arrival
    rates, against the same requests solved one after another in FP64."""
    import time as _t
    import mlpg_inputs as mi
    from paper_2008_02205_gb300.serving import Request, Server, latency_percentiles
    out = {"requests": count, "n_range": [4096, 65536], "steps_range": [5, 20], "budget_gb": 96, "rates": []}
    mixed = dict(precision=pkg.MLPG_MIXED)
    for rate in rates:
        stream = mi.serving_stream(count=count, rate=rate, seed=5000, n_range=(4096, 65536), steps_range=(5, 20))
        reqs = [Request(p, p.steps, p.dt, arrival=t, options=mixed) for p, t in stream]
        srv = Server(hbm_budget_bytes=96 << 30, max_active=8)
        t0 = _t.perf_counter()
        res = srv.run(reqs)
        wall = _t.perf_counter() - t0
        ok = [r for r in res if r.error is None]
        lat = latency_percentiles(res)
        out["rates"].append({"rate_per_s": rate, "solves_per_s": len(ok) / wall, "wall_s": wall,
                             "p50_s": lat.get("p50"), "p99_s": lat.get("p99"), "failed": len(res) - len(ok),
                             "peak_active": srv.peak_active, "steps_during_setup": srv.steps_during_open})
    # the same requests, one after another, plain FP64
    stream = mi.serving_stream(count=count, rate=rates[0], seed=5000, n_range=(4096, 65536), steps_range=(5, 20))
    t0 = _t.perf_counter()
    for p, _ in stream:
        with pkg.TransportProblem.from_problem(p, precision=pkg.MLPG_FP64) as tp:
            tp.integrate().assemble()
            tp.run(p.dt, p.steps)
    seq = _t.perf_counter() - t0
    out["fp64_sequential"] = {"solves_per_s": count / seq, "wall_s": seq}
    return out


def _batched(pkg, count=64, steps=10):
    """The batched configuration: 64 independent 2D problems (1k-64k points,
    S4-S12, sigma_t in [0.1, 10], scattering ratio in [0, 0.99]), mixed
    precision, every problem advanced by one concurrent batched step per
    time step; against the same problems stepped one after another."""
    import time as _t
    import mlpg_inputs as mi
    probs = mi.batched_2d(count, steps=steps)
    tps = []
    try:
        for p in probs:
            tps.append(pkg.TransportProblem.from_problem(p, precision=pkg.MLPG_MIXED))
            tps[-1].integrate().assemble()
        pkg.TransportProblem.step_batch(tps, probs[0].dt)          # operators formed, buffers made
        for tp in tps:
            tp.set_state(np.zeros((tp.n, tp.m)))
        t0 = _t.perf_counter()
        for _ in range(steps):
            pkg.TransportProblem.step_batch(tps, probs[0].dt)
        for tp in tps:
            tp.scalar_flux()
        batched = _t.perf_counter() - t0
        for tp in tps:
            tp.set_state(np.zeros((tp.n, tp.m)))
        t0 = _t.perf_counter()
        for tp in tps:
            for _ in range(steps):
                tp.step(probs[0].dt)
            tp.scalar_flux()
        seq = _t.perf_counter() - t0
    finally:
        for tp in tps:
            tp.close()
    return {"problems": count, "steps": steps, "points": int(sum(p.n for p in probs)),
            "solves_per_s": count / batched, "wall_s": batched,
            "sequential": {"solves_per_s": count / seq, "wall_s": seq}}


def main():
    args = _args()
    rank, world, local = _dist()
    if args.impl == "reference":
        if rank == 0:
            _reference(args)
        return
    import torch
    import mlpg_inputs as mi
    import paper_2008_02205_gb300 as pkg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # independent problems per rank (weak scaling): seed by rank
    if args.mode == "apply3d":
        prob = mi.lognormal_3d(args.side3, refine=(1, 5, 15.0), seed=3000 + rank)
    else:
        prob = mi.two_region_2d(n_per_dim=args.n, seed=2000 + rank)
    if args.be_steps is not None:
        prob.steps = args.be_steps
    prec = pkg.MLPG_MIXED if args.precision == "mixed" else pkg.MLPG_FP64
    # a dedicated stream: the library runs on it and the CUDA events below are recorded on it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    opts = dict(precision=prec, stream=stream.cuda_stream, dim=prob.dim, lo=tuple(prob.lo), hi=tuple(prob.hi))
    tuned = None
    if prec == pkg.MLPG_MIXED and not args.no_tune and args.mode != "apply3d":   # 3D: the automatic choice
        from paper_2008_02205_gb300 import autotune
        tuned = autotune.tuned_options(prob, stream=stream)   # times each tile shape once, then cached
        opts.update(tuned)
    host = dict(x=prob.x, R=prob.R, om=prob.omega, w=prob.w, st=prob.sigma_t, ss=prob.sigma_s, q=prob.q)
    dv = {k: torch.tensor(v, dtype=torch.float64, device=dev) for k, v in host.items()}
    flux = torch.empty(prob.n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    def solve_device(timing=False):
        o = pkg.mlpg_default_options(**opts)
        ctx = pkg.mlpg_create_dev(o, prob.n, prob.m, dv["x"].data_ptr(), dv["R"].data_ptr(), dv["om"].data_ptr(),
                                  dv["w"].data_ptr(), dv["st"].data_ptr(), dv["ss"].data_ptr(), dv["q"].data_ptr())
        try:
            if timing:
                pkg.mlpg_enable_timing(ctx, True)
            pkg.mlpg_integrate(ctx)
            pkg.mlpg_assemble(ctx)
            for _ in range(prob.steps):
                pkg.mlpg_step(ctx, prob.dt)
            pkg.mlpg_scalar_flux_dev(ctx, flux.data_ptr(), 0)
            return pkg.mlpg_get_stats(ctx)
        finally:
            pkg.mlpg_destroy(ctx)

    def solve_host():
        o = pkg.mlpg_default_options(**opts)
        ctx = pkg.mlpg_create(o, host["x"], host["R"], host["om"], host["w"], host["st"], host["ss"], host["q"])
        try:
            pkg.mlpg_integrate(ctx)
            pkg.mlpg_assemble(ctx)
            for _ in range(prob.steps):
                pkg.mlpg_step(ctx, prob.dt)
            return pkg.mlpg_scalar_flux(ctx, prob.n, 0)
        finally:
            pkg.mlpg_destroy(ctx)

    if args.mode == "apply":
        _apply_mode(args, pkg, prob, prec, opts, dv, stream, world, rank)
        return
    if args.mode == "apply3d":
        _apply_mode(args, pkg, prob, prec, opts, dv, stream, world, rank,
                    workload=f"3d-lognormal-{args.side3}^3-refined{prob.m}")
        return
    for _ in range(args.warmup):
        solve_device()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    per = []
    stats = None
    spmm_ms, spmm_launch, launches = 0.0, 0, 0
    for _ in range(args.steps):
        flush.zero_()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = solve_device(timing=True)
        e1.record(stream)
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1))
        spmm_ms += stats["spmm_ms"]
        spmm_launch += stats["spmm_launches"]
        launches += stats["kernel_launches"]
    clk = clocks.stop()
    tot_ms = _max_over_ranks(sum(per), world, dev)
    value = _job_rate(world, args.steps, tot_ms / 1e3)
    # end to end through the host-pointer API (copies inside the timed region)
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phi_host = solve_host()
        e2e_times.append(time.perf_counter() - t0)
    h2d = sum(v.nbytes for v in host.values())
    e2e_value = _job_rate(world, 1, _max_over_ranks(statistics.mean(e2e_times), world, dev)) if e2e_times else None
    # FP64 comparison solve (the plain FP64 GPU path) and error of this precision vs it
    fp64_info = None
    if not args.no_fp64_compare and prec == pkg.MLPG_MIXED:
        o = dict(opts)
        o["precision"] = pkg.MLPG_FP64
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with pkg.TransportProblem.from_problem(prob, **o) as tp:
            tp.integrate().assemble()
            phi64 = tp.run(prob.dt, prob.steps)
        t64 = time.perf_counter() - t0
        phi_mixed = phi_host if e2e_times else flux.cpu().numpy()
        err = float(np.linalg.norm(phi_mixed - phi64) / np.linalg.norm(phi64))
        fp64_info = {"solves_per_s": 1.0 / t64, "rel_l2_vs_fp64": err}
    # error against the oracle's solve of the same workload (stored by an oracle-only script)
    oracle_err = None
    g = _golden()
    if g is not None and args.n == 256 and prob.steps == 20:
        ref = g["phi_20"]
        phi_m = phi_host if e2e_times else flux.cpu().numpy()
        oracle_err = {"rel_l2_vs_oracle": float(np.linalg.norm(phi_m - ref) / np.linalg.norm(ref)),
                      "oracle_outer_per_step": float(np.mean(g["outer_iterations"]))}
        if fp64_info is not None:
            fp64_info["rel_l2_vs_oracle"] = float(np.linalg.norm(phi64 - ref) / np.linalg.norm(ref))
    extras = {}
    if not args.no_extras and rank == 0 and world == 1:
        for name, fn in (("apply_3d", lambda: _apply_3d(pkg, stream)), ("serving", lambda: _serving(pkg)),
                         ("batched", lambda: _batched(pkg))):
            try:
                extras[name] = fn()
            except Exception as e:      # an extra measurement never hides the main line
                extras[name] = {"error": f"{type(e).__name__}: {e}"}
    counts = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = _oracle_counts()
    hbm, peak_kind = _peaks()
    roof = None
    if spmm_launch > 0 and spmm_ms > 0:
        per_launch_s = spmm_ms / spmm_launch / 1e3
        achieved = stats["spmm_bytes"] / per_launch_s / 1e9
        roof = {"kernel": (APPLY_KERNELS.get(stats["apply_kernel"], "k_spmm32") if prec == pkg.MLPG_MIXED
                           else "k_spmm64") + ": batched L-apply",
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": _traffic() if prec == pkg.MLPG_MIXED and stats["apply_kernel"] == 2 else None,
                "peak_kind": peak_kind,
                "bytes_per_launch": stats["spmm_bytes"], "us_per_launch": per_launch_s * 1e6}
    lat = sorted(per)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    line = {"metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == pkg.MLPG_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": prob.n, "directions": prob.m, "be_steps": prob.steps,
                       "precision": args.precision, "l2": "flushed (256 MB write) between timed solves",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": p50, "p99": p99},
            "iterations": {"outer_last_step": stats["last_outer_iters"],
                           "inner_last_step": stats["last_inner_iters"],
                           "inner_solves_last_step": stats["last_inner_solves"],
                           "refinements_last_step": stats["last_refinements"],
                           "outer_total": stats["total_outer_iters"], "inner_total": stats["total_inner_iters"],
                           "gpu_inner_per_direction_solve_last_step": stats["last_inner_iters"] / max(
                               1, prob.m * stats["last_inner_solves"]),
                           "oracle_outer_per_step_full_size": (oracle_err or {}).get("oracle_outer_per_step"),
                           "oracle_ilut_gmres": counts},
            "fp64_path": fp64_info,
            "oracle": oracle_err,
            "apply_tiles": tuned,
            "extras": extras,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(prob.n * 8)},
            "roofline": roof, "clocks": clk, "gpu_launches": launches,
            "cpu_baseline": _oracle_sample(1) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
