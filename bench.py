#!/usr/bin/env python
"""Benchmark of the aMFP phonon-BTE solver on one GB300 (or N replicas).

Workload: the 2D periodic cell L = 200 nm, 256 x 256 cells, circular pore of
porosity 0.25 with diffuse walls, 30 log-spaced MFP bins 1 nm - 10 um,
48 azimuthal x 12 polar directions projected on the plane (folded to 6
polar nodes: 8640 ordinates), dT = 1 K along x.  Synthetic inputs from
paper_2106_02764_gb300.inputs (no dataset exists for this path).

One step = one full solve through the C ABI: Fourier first guess, source
iteration (Anderson-mixed, same fixed point) to the Algorithm-1 stop
(relative change of kappa below 1e-6), FP32 sweeps with FP64 moments
("mixed").  value = cell-ordinate updates per
second over the whole step; time to kappa_eff within 1e-4 of the oracle's
converged value is reported beside it, for the mixed form and for the plain
FP64 GPU sweep.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-ordinate updates/s and time to κ_eff (1e-4 rel) vs plain FP64 GPU sweep"
UNIT = "cell-ordinate updates/s"
WORKLOAD = "2d-256x256-circle-phi0.25-30bins-48x12proj (8640 folded ordinates), dT=1K"
FLOP_PER_UPDATE_2D = 7   # 1 mul + 2 fma (transport) + 1 fma (T_L moment)
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0
ACCEL = 5                # Anderson window of the outer iteration (same fixed point)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the config-3 / config-4 / sharded legs")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- oracle legs
def cpu_oracle_rate(wl, seconds, max_cores=None):
    """Algorithm-1 pass of the oracle (per-ordinate sparse LU) over a bounded
    sample of ordinates, in spawn worker processes on the host cores."""
    from oracle import bte, pool
    cores = pool.usable_cores() if max_cores is None else max_cores
    tr0 = bte.Transport(bte.Problem.from_workload(wl), cache=False)
    T_L, T_w = bte.initial_guess(tr0)
    n_ord = wl.n_ordinates
    rng = np.random.default_rng(7)
    order = rng.permutation(n_ord)
    # probe: two ordinates per worker, then size the sample to ~seconds
    with pool.PoolTransport(wl, workers=cores, chunks_per_worker=1, ordinates=order[:2 * cores]) as pt:
        t0 = time.perf_counter()
        pt.sweep(T_L, T_w)
        probe = time.perf_counter() - t0
    per_ord = probe / (2 * cores)
    n = int(min(n_ord, max(2 * cores, seconds / max(per_ord, 1e-6))))
    with pool.PoolTransport(wl, workers=cores, chunks_per_worker=1, ordinates=order[:n]) as pt:
        t0 = time.perf_counter()
        pt.sweep(T_L, T_w)
        dt = time.perf_counter() - t0
    updates = tr0.prob.mesh.nc * n
    return {"value": updates / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"one Algorithm-1 pass (per-ordinate SciPy sparse LU, no LU cache) over "
                      f"{n} of {n_ord} ordinates on the full 256x256 mesh, {dt:.1f} s"}


def reference_arm(a, rank, world):
    """--impl reference: the oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_2106_02764_gb300 import inputs as I
    wl = I.config2()
    cores = None
    vals = []
    for i in range(a.warmup + a.steps):
        r = cpu_oracle_rate(wl, seconds=max(2.0, a.cpu_seconds / 3))
        cores = r["cores"]
        if i >= a.warmup:
            vals.append(r)
    v = float(np.mean([r["value"] for r in vals]))
    ms = 1e3 * float(np.mean([r["seconds"] for r in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs re-read by fresh processes every step"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": UNIT,
                             "sample": vals[-1]["sample"] + " (each step a bounded sample of the "
                                       "config-2 pass)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm
def crossing(history, kappa_star, rtol=1e-4):
    """Iterations until kappa_n is within rtol of kappa* and stays within it."""
    h = np.array(history)
    ok = np.abs(h - kappa_star) <= rtol * abs(kappa_star)
    if not ok.any():
        return None
    last_bad = np.nonzero(~ok)[0]
    first = int(last_bad[-1]) + 1 if len(last_bad) else 0
    return first + 1 if first < len(h) else None


def time_to_kappa(stats, kappa_star, rtol=1e-4):
    """Derived from one solve's kappa history: Fourier guess + the mean
    iteration time x the crossing index (see measured_time_to_kappa)."""
    n = crossing(stats["kappa_history"], kappa_star, rtol)
    if n is None:
        return None, None
    per_it = stats["time_iter_ms"] / max(1, stats["iterations"])
    return stats["time_fourier_ms"] + n * per_it, n


def measured_time_to_kappa(run, n_iter, reps=3):
    """Device time (CUDA events on the solve stream) of a solve stopped after
    exactly n_iter iterations, the crossing index of a full solve: the
    measured time to kappa within 1e-4 (median of reps, after one warm-up)."""
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for i in range(reps + 1):
        torch.cuda.synchronize()
        e0.record(st)
        run(n_iter)
        e1.record(st)
        torch.cuda.synchronize()
        if i:
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def batch_leg(local, rtol=1e-4):
    """Config 4 (64 geometries, N = 48 ... 192): the mixed batched form against
    the plain FP64 batched form, time until every geometry with a stored
    oracle value has kappa within 1e-4 of it (measured as a batch solve
    stopped at that iteration), and the batch's update rate."""
    from paper_2106_02764_gb300 import inputs as I
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    geoms = I.config4()
    stars = {}
    for gi in range(len(geoms)):
        p = os.path.join(ROOT, "tests", "golden", f"kappa_star_cfg4_{gi}.json")
        if os.path.exists(p):
            with open(p) as f:
                stars[gi] = json.load(f)["kappa_eff"]
    if not stars:
        return None
    out = {"geometries": len(geoms), "with_oracle_value": sorted(stars),
           "updates_per_iteration": int(sum(w.n_solid * w.n_ordinates for w in geoms))}
    for prec in ("mixed", "fp64"):
        solvers = [Solver.from_workload(w, device=local) for w in geoms]
        kw = dict(precision=prec, check_every=8, accel=ACCEL, allow_not_converged=True)
        stats = solve_batch(solvers, tol=1e-6, max_iter=3000, **kw)
        ns = [crossing(stats[gi]["kappa_history"], k, rtol) for gi, k in stars.items()]
        if any(n is None for n in ns):
            out[prec] = {"time_to_kappa_1e-4_ms": None}
            continue
        n_star = max(ns)

        def run(n):
            solve_batch(solvers, tol=0.0, max_iter=n, **kw)
        t = measured_time_to_kappa(run, n_star)
        iters = max(s["iterations"] for s in stats)
        out[prec] = {"time_to_kappa_1e-4_ms": t, "iterations_to_kappa_1e-4": n_star,
                     "solve_ms": stats[0]["time_total_ms"], "iterations": iters,
                     "updates_per_s": out["updates_per_iteration"] * iters / (stats[0]["time_iter_ms"] * 1e-3)}
        for s in solvers:
            s.close()
    if out["mixed"].get("time_to_kappa_1e-4_ms") and out["fp64"].get("time_to_kappa_1e-4_ms"):
        out["speedup_time_to_kappa_vs_fp64"] = out["fp64"]["time_to_kappa_1e-4_ms"] / out["mixed"]["time_to_kappa_1e-4_ms"]
    return out


def film_leg(local):
    """Config 3 (3D film 64 x 64 x 32, 8640 ordinates): per-launch time of the 3D
    sweep over 40 iterations in each precision, with its ALU roofline (9 flop
    per solid cell-ordinate update: 2D + the z inflow)."""
    from paper_2106_02764_gb300 import inputs as I
    from paper_2106_02764_gb300.binding import Solver
    wl = I.config3()
    out = {"workload": wl.name, "n_solid": wl.n_solid, "n_ordinates": wl.n_ordinates}
    for prec in ("mixed", "fp64"):
        s = Solver.from_workload(wl, device=local)
        st = s.solve(precision=prec, tol=0.0, max_iter=40, check_every=8, profile=True,
                     allow_not_converged=True)
        ms = st["time_sweep_ms"] / max(1, st["n_sweeps"])
        flop = 9 * wl.n_solid * wl.n_ordinates
        out[prec] = {"sweep_ms": ms, "achieved_tflops": flop / (ms * 1e-3) / 1e12,
                     "updates_per_s": wl.n_solid * wl.n_ordinates / (ms * 1e-3),
                     "group_size": st["group_size"], "rows_per_thread": st["rows_per_thread"]}
        s.close()
    return out


def small_leg(local, rtol=1e-4):
    """Config 1 (2D 32^2, 8 bins x 16 directions): time to kappa within 1e-4 of
    the oracle's stored value in each precision, measured as a solve stopped at
    the crossing iteration (the same solve options as the main leg)."""
    from paper_2106_02764_gb300 import inputs as I
    from paper_2106_02764_gb300.binding import Solver
    p = os.path.join(ROOT, "tests", "golden", "kappa_star_cfg1.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        k_star = json.load(f)["kappa_eff"]
    wl = I.config1()
    out = {"workload": wl.name, "updates_per_iteration": wl.n_solid * wl.n_ordinates}
    for prec in ("fp64", "mixed"):
        s = Solver.from_workload(wl, device=local)
        kw = dict(precision=prec, check_every=8, accel=ACCEL, allow_not_converged=True)
        st = s.solve(tol=1e-6, max_iter=3000, **kw)
        n = crossing(st["kappa_history"], k_star, rtol)
        t = None
        if n is not None:
            t = measured_time_to_kappa(lambda m: s.solve(tol=0.0, max_iter=m, **kw), n)
        out[prec] = {"time_to_kappa_1e-4_ms": t, "iterations_to_kappa_1e-4": n,
                     "solve_ms": st["time_total_ms"], "iterations": st["iterations"],
                     "kappa_rel_err": abs(st["kappa_eff"] - k_star) / k_star}
        s.close()
    return out


def gradient_leg(local, reps=3):
    """Config 5 (2D 128^2, s(x) ~ U[0.5, 2], 640 ordinates): d kappa_eff / d s
    over every cell after a tight solve (Anderson(5); FP64 to a relative kappa
    change of 1e-12, mixed a fixed 600 iterations): the solve's device time,
    the gradient call's wall time (median of reps after one warm-up; record
    passes, contractions and the host copies of one obte_kappa_grad_s) and its
    error against the oracle adjoint stored with the tests."""
    import time as _time
    from paper_2106_02764_gb300 import inputs as I
    from paper_2106_02764_gb300.binding import Solver
    pj = os.path.join(ROOT, "tests", "golden", "grad_cfg5.json")
    pz = os.path.join(ROOT, "tests", "golden", "grad_cfg5.npz")
    ref = None
    if os.path.exists(pz):
        z = np.load(pz)
        ref = (z["grad"], z["coords"])
    wl = I.config5()
    out = {"workload": wl.name, "n_solid": wl.n_solid, "n_ordinates": wl.n_ordinates}
    for prec in ("mixed", "fp64"):
        s = Solver.from_workload(wl, device=local)
        if prec == "fp64":
            st = s.solve(precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=20000, check_every=16,
                         accel=ACCEL, allow_not_converged=True)
        else:
            st = s.solve(precision="mixed", tol=0.0, max_iter=600, check_every=50, accel=ACCEL,
                         allow_not_converged=True)
        ts = []
        for i in range(reps + 1):
            t0 = _time.perf_counter()
            g = s.kappa_grad_s()
            if i:
                ts.append((_time.perf_counter() - t0) * 1e3)
        e = {"solve_ms": st["time_total_ms"], "iterations": st["iterations"],
             "gradient_ms": statistics.median(ts)}
        if ref is not None:
            gr, c = ref
            gg = g[c[:, 2], c[:, 1], c[:, 0]]
            e["grad_err_rel_max"] = float(np.abs(gg - gr).max() / np.abs(gr).max())
        out[prec] = e
        s.close()
    out["reference"] = "oracle adjoint (tests/golden/grad_cfg5.npz)" if ref is not None else None
    return out


def sharded_leg(wl, local, rank, world, dist, kappa_star):
    """One config-2 solve with its ordinate groups spread over the ranks (Sec.
    3: directions over processes): per iteration each rank sweeps its share,
    the FP64 moment partials are summed by an all-reduce (NCCL under torchrun;
    nothing to sum on one rank) and every rank finalises.  Plain source
    iteration (the sharded form has no Anderson mixing), mixed precision, stop
    at a relative kappa change of 1e-6."""
    import torch
    from paper_2106_02764_gb300.binding import Solver
    s = Solver.from_workload(wl, device=local).set_shard(rank, world)
    buf = torch.empty(s.shard_partials_count(), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    s.shard_begin(precision="mixed", tol=1e-6, max_iter=5000, group_size=8, rows_per_thread=8)
    it = 0
    while True:
        s.shard_sweep(buf)
        if dist:
            dist.all_reduce(buf)
        it += 1
        if s.shard_finalize(buf):
            break
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    k = s.kappa_eff
    return {"ranks": world, "iterations": it, "ms": ms,
            "updates_per_s": wl.n_solid * wl.n_ordinates * it / (ms * 1e-3),
            "kappa_eff": k, "kappa_rel_err": abs(k - kappa_star) / kappa_star if kappa_star else None,
            "exchange": "all-reduce of %d FP64 partials per iteration" % s.shard_partials_count()}


SWEEP_SOURCES = ("sweep2d.cuh", "sweep.cuh", "sweep2d_variants.h", "obte_internal.h")


def sweep_hash():
    """Hash of the sources of the dominant kernel; a stored DRAM-traffic figure
    is used only while it matches."""
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_02764_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(name):
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(name)
    if not e or e.get("sweep_hash") != sweep_hash():
        return None
    return e.get("dram_bytes_per_launch")


def sweep_blocks(st):
    """Thread blocks of one sweep launch: the 2D warp kernel (kernel 2) runs
    one ordinate group per warp, the block kernels one group per block."""
    groups = int(st["n_groups"])
    if st["kernel"] == 2:
        warps = max(1, int(st["threads_per_block"]) // 32)
        return -(-groups // warps)
    return groups


def launches_per_solve(iterations, check_every):
    """Kernels one mixed Anderson solve launches: the first guess (cluster CG)
    and five start-of-solve kernels (state, wall temperatures, records, their
    deviation-form difference fields, Anderson history), then per launched
    iteration the sweep, finalize, the zeroing of the skewed T_L partials,
    the finalisation tail, the three Anderson kernels and the records'
    difference fields.  Iterations go in graph chunks of check_every and a
    solve stops inside a chunk, whose remaining iterations launch and return
    at once."""
    launched = -(-int(iterations) // int(check_every)) * int(check_every)
    return 6 + 8 * launched


def main():
    a = _args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        reference_arm(a, rank, world)
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2106_02764_gb300 import build, inputs as I
    from paper_2106_02764_gb300.binding import Solver
    build.build()
    wl = I.config2()
    n_solid, n_ord = wl.n_solid, wl.n_ordinates
    kstar_file = os.path.join(ROOT, "tests", "golden", "kappa_star_cfg2.json")
    kappa_star, kstar_src = None, None
    if os.path.exists(kstar_file):
        with open(kstar_file) as f:
            kappa_star = json.load(f)["kappa_eff"]
        kstar_src = "oracle mode B (tests/golden/kappa_star_cfg2.json)"

    opts = dict(precision="mixed", tol=1e-6, max_iter=3000, check_every=8, profile=True,
                accel=ACCEL)
    solver = Solver.from_workload(wl, device=local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(a.warmup):
        solver.solve(**opts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, stats = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    for _ in range(a.steps):
        flush.fill_(1.0)                 # L2 flush between timed steps (outside the timing)
        torch.cuda.synchronize()
        ev0.record(stream)
        st = solver.solve(**opts)
        ev1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        stats.append(st)
    clk = clocks.stop()
    total_ms = sum(step_ms)
    updates = sum(n_solid * n_ord * s["iterations"] for s in stats)
    launches = sum(launches_per_solve(s["iterations"], opts["check_every"]) for s in stats)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        u = torch.tensor([float(updates)], device="cuda")
        dist.all_reduce(u)
        updates = float(u.item())
    value = updates / (total_ms * 1e-3)

    # roofline of the sweep kernel, timed per launch inside the steps above
    sweeps = sum(s["n_sweeps"] for s in stats)
    sweep_ms = sum(s["time_sweep_ms"] for s in stats) / max(1, sweeps)
    flops_launch = FLOP_PER_UPDATE_2D * n_solid * n_ord
    achieved = flops_launch / (sweep_ms * 1e-3) / 1e12
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12

    extra = {}
    if not a.no_extra:
        extra["ordinate_sharded_config2"] = sharded_leg(wl, local, rank, world, dist, kappa_star)
    if rank == 0:
        # time to kappa_eff (1e-4 rel): mixed (timed steps) vs plain FP64 sweep
        ref_k = kappa_star
        if ref_k is None:
            extra["kappa_star_source"] = "unavailable (oracle value not stored); final FP64 iterate used"
        else:
            extra["kappa_star_source"] = kstar_src
        fp64 = None
        if not a.no_fp64:
            s64 = Solver.from_workload(wl, device=local)
            fp64 = s64.solve(precision="fp64", tol=1e-6, max_iter=3000, check_every=8, profile=True,
                             accel=ACCEL)
            if ref_k is None:
                ref_k = fp64["kappa_eff"]
        ttk = [time_to_kappa(s, ref_k) for s in stats] if ref_k else []
        ttk_ms = [t for t, _ in ttk if t is not None]
        n_star = ttk[0][1] if ttk else None
        extra["iterations_to_kappa_1e-4"] = n_star
        extra["time_to_kappa_1e-4_ms_derived"] = statistics.median(ttk_ms) if ttk_ms else None
        extra["time_to_kappa_1e-4_ms"] = (measured_time_to_kappa(
            lambda n: solver.solve(**{**opts, "tol": 0.0, "max_iter": n, "profile": False},
                                   allow_not_converged=True), n_star) if n_star else None)
        extra["kappa_eff"] = stats[-1]["kappa_eff"]
        extra["kappa_rel_err"] = abs(stats[-1]["kappa_eff"] - ref_k) / abs(ref_k) if ref_k else None
        extra["iterations_per_step"] = stats[-1]["iterations"]
        extra["fourier_ms"] = stats[-1]["time_fourier_ms"]
        if fp64:
            _t64, n64 = time_to_kappa(fp64, ref_k)
            t64 = measured_time_to_kappa(
                lambda n: s64.solve(precision="fp64", tol=0.0, max_iter=n, check_every=8, accel=ACCEL,
                                    allow_not_converged=True), n64) if n64 else None
            extra["fp64"] = {"time_to_kappa_1e-4_ms": t64, "time_to_kappa_1e-4_ms_derived": _t64,
                             "iterations_to_kappa_1e-4": n64,
                             "updates_per_s": fp64["updates_per_s"],
                             "sweep_ms": fp64["time_sweep_ms"] / max(1, fp64["n_sweeps"]),
                             "kappa_eff": fp64["kappa_eff"], "iterations": fp64["iterations"]}
            if t64 and extra["time_to_kappa_1e-4_ms"]:
                extra["speedup_time_to_kappa_vs_fp64"] = t64 / extra["time_to_kappa_1e-4_ms"]

        # end to end through the C ABI from host buffers
        e2e_ms, h2d, d2h = [], 0, 0
        for i in range(max(2, a.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = Solver.from_workload(wl, device=local)
            st2 = s2.solve(**{**opts, "profile": False})
            TL = s2.T_L()
            k2 = s2.kappa_eff
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            h2d = wl.mask.nbytes + wl.kappa_m.nbytes + wl.lambda_m.nbytes + wl.quad.dirs.nbytes + \
                wl.quad.weights.nbytes
            d2h = TL.nbytes + 8
            s2.close()
        e2e_updates = n_solid * n_ord * st2["iterations"]
        e2e = {"value": e2e_updates / (statistics.median(e2e_ms) * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": statistics.median(e2e_ms)}
        # measured FMA throughput (context for the derived ALU peak)
        from paper_2106_02764_gb300.binding import measure_fma_rate
        fma32 = measure_fma_rate("mixed", local) / 1e12
        fma64 = measure_fma_rate("fp64", local) / 1e12
        if not a.no_extra:
            extra["batched_config4"] = batch_leg(local)
            extra["film_config3"] = film_leg(local)
            extra["small_config1"] = small_leg(local)
            extra["gradient_config5"] = gradient_leg(local)
        cpu = None
        if not a.no_cpu_baseline:
            cpu = cpu_oracle_rate(wl, a.cpu_seconds)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweep / f64 moments",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "mixed", "stop": "rel dkappa < 1e-6",
                       "outer": f"Anderson({ACCEL}) on (T_L, T_w, carried row values)",
                       "l2": "flushed (512 MB write) between timed steps; working set per "
                             "iteration fits L2 and is reused within a step",
                       "group_size": stats[-1]["group_size"], "rows_per_thread": stats[-1]["rows_per_thread"],
                       "threads_per_block": stats[-1]["threads_per_block"],
                       "groups_per_sweep": stats[-1]["n_groups"],
                       "blocks_per_sweep": sweep_blocks(stats[-1]),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic_from_profile("cfg2_mixed"),
                         "kernel": "sweep2d_warp_kernel<float,G,R> (2D warp-per-group sweep)",
                         "flop_per_launch": flops_launch, "avg_launch_ms": sweep_ms,
                         "peak_note": "FP32 FMA pipes: 152 SMs x 128 lanes x 2 flop x 2070 MHz (max clock)",
                         "measured_fma_tflops": {"fp32": fma32, "fp64": fma64},
                         "frac_of_measured_fp32": achieved / fma32 if fma32 > 0 else None},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
