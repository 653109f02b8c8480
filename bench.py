#!/usr/bin/env python3
"""Throughput benchmark of the SPH active-nematic time step on GB300.

Workload: the high-resolution set-up, a 1024 x 1024 jittered lattice (1,048,576 particles) in the
periodic unit box, h = 1.3 dx, zeta = 0.08, K = 0.02, the other parameters of the paper's 2D
set-up, FP32 pair arithmetic with FP64 positions, dt = the stable step (viscous limit).  Inputs are
synthetic (seeded lattice, random director); the working set (~0.5 GB) exceeds the 129 MB L2.

Metric: particle-steps/s (particles x steps / time), with the directed pair interactions per second
reported beside it.  One step = all kernels of the step (predictor, cell sort, passes A-D).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) each rank advances its own ensemble member (seed = rank) with no collective
on the data path: weak scaling; the timing is the max over ranks.  ``--impl reference`` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = 1024
PARAMS = dict(zeta=0.08, K=0.02)
METRIC = "particle-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SRC = os.path.join(ROOT, "paper_2108_08919_gb300", "csrc", "ann_kernels.cu")

# FP32 flops per directed neighbour pair of each pass (FMA = 2), counted from the formulas:
#   pair geometry and kernel value/derivative (d, |d|^2, 1/r, b, quintic pieces)   ~24
#   pass_a (candidate filter): geometry + W + the support test (3)                          = 27
#   pass_a_resort: geometry + W + the cell-stencil candidate tests (5 x ~3.1 per pair)      = 39.5
#   pass B: + alpha (6), velocity-gradient sums (10), Q-Laplacian sums (16), V F d (4)    = 70
#   pass C: + Shepard sum (3), div Q sums (13)                                            = 48
#   pass D: + pressure (7), viscous (12), APD sums (11)                                    = 62
FLOPS_PER_PAIR = {"pass_a": 27.0, "pass_a_resort": 24 + 15.5, "pass_b": 70.0, "pass_c": 48.0,
                  "pass_d": 62.0}
# Compulsory DRAM bytes per particle of each kernel: every array it must read or write, once.
# Candidate lists: 2 B per candidate, ~46 candidates (44 neighbours and the skin), + the count = 96.
#   predict       u, a, r, Q, delta, id, cell key, reference split in (68); u, r, and the
#                 evaluation copy (r, split r, u, Q, delta, id) out (80)                    148
#   cell_order    permutation, state and split position in; the sorted copy out             116
#   pass_a_resort split position in; candidate lists (with their neighbour bits), count,
#                 sum W, V, reference out                                                   140
#   pass_a        split position, candidate lists in; count, sum W, V out (a list word is
#                 rewritten only when a neighbour bit changes: a few per step)              124
#   pass_b        split position, V, u, Q, delta, lists in; Q^{n+1}, (B, k) as one record,
#                 pass C's staged record (V, delta_half, Q^{n+1}) out                      176
#   pass_c        split position, (V, delta_half, Q^{n+1}), sum W, (B, k), u, lists in; p,
#                 (div Q, delta_hat, sum W) and pass D's staged record (V, p/rho^2, u) out 192
#   pass_d        everything the momentum, corrector and APD read (V, p, u as one staged
#                 record; (B, k) and (div Q, delta_hat, sum W) as two); the new state out 216
BYTES_PER_PARTICLE = {"predict": 148, "cell_scan": 0.5, "cell_scatter": 16, "cell_order": 116,
                      "pass_a_resort": 140, "pass_a": 124, "pass_b": 176, "pass_c": 192,
                      "pass_d": 216}
RESORT_BRANCH = ("cell_keys", "cell_scan", "cell_scatter", "cell_order", "pass_a_resort")


def launches_in_steps(steps: int, resorts: int) -> int:
    """Kernels the step graph launches: the commit of the previous step, the predictor, the branch
    condition, then either the five re-sort kernels or the candidate filter, then passes B, C and D."""
    return 7 * steps + 4 * resorts


def _rank_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def ensemble_seed(rank: int) -> int:
    """Each rank advances its own ensemble member: an independent problem of the same size."""
    return rank


def slowest(local_value: float, dist=None, device=None) -> float:
    """The maximum of a per-rank time over all ranks (the job is as slow as its slowest rank)."""
    if dist is None:
        return float(local_value)
    import torch

    t = torch.tensor([float(local_value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size: int, particles: int, steps: int, seconds: float) -> float:
    """Whole-job particle-steps/s: every rank advances `particles` particles `steps` times."""
    return world_size * particles * steps / seconds


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """Nominal FP32 rate: SMs x 128 FP32 lanes x 2 flops (FMA) x clock (context for the measured
    rate of ann_fp32_fma_peak, which is the roofline's denominator)."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def developed_flow_bench(B, stream, steps: int = 6000, u_max: float = 0.1, seed: int = 5):
    """Steps of the headline workload from a moving state, so that the re-sort branch runs as in a
    developed flow: the box-scale cellular flow u = u_max (sin 2 pi y, sin 2 pi x) (V_rms = u_max, the
    level of the developed 256^2 long runs; a box-scale field, since particle-scale velocities decay
    within a few steps at eta = 1), timed over `steps` steps with CUDA events; re-sorts per 1,000
    steps and the step time beside the headline's (which starts from rest and does not re-sort)."""
    import numpy as np
    import torch

    import sph_inputs as si

    ic = si.jittered_lattice(NX, seed=seed)
    ux = u_max * np.sin(2.0 * np.pi * ic["y"])
    uy = u_max * np.sin(2.0 * np.pi * ic["x"])
    p = make_params(B, NX)
    ctx = B.ann_create(p)
    try:
        B.ann_set_stream(ctx, stream)
        B.ann_set_particles(ctx, ic["x"], ic["y"], ux, uy, ic["q11"], ic["q12"], ic["rho"])
        B.ann_step(ctx, 20)
        torch.cuda.synchronize()
        r0 = B.ann_get_diagnostics(ctx)["resorts"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            B.ann_step(ctx, steps)
            e1.record(stream)
        torch.cuda.synchronize()
        d = B.ann_get_diagnostics(ctx)
        ms = e0.elapsed_time(e1)
    finally:
        B.ann_destroy(ctx)
    rs = d["resorts"] - r0
    return {"steps": steps, "ms_per_step": ms / steps, "resorts": rs, "resorts_per_1000_steps": 1000.0 * rs / steps,
            "max_speed": d["max_speed"], "u_max": u_max,
            "particle_steps_per_s": NX * NX * steps / (ms * 1e-3)}


def size_sweep_bench(B, stream, sizes=(256, 512, 1024, 2048, 4096, 8192), work=3e9, warmup=5, peak_tf=None):
    """Throughput of the headline set-up (from rest, h = 1.3 dx, stable dt) against the lattice side:
    each size timed with CUDA events over about `work` particle-steps (20 to 3,000 steps), then the
    per-kernel device times of the profile loop over a tenth of those steps (at least 5), with pass
    D's FP32 rate against `peak_tf`.  Sides above 1024 tile the unit box with copies of a jittered
    1024^2 lattice shrunk to fit, which keeps the particle spacing and neighbour statistics of the
    smaller sizes."""
    import torch

    import sph_inputs as si

    out = []
    for nx in sizes:
        base = min(nx, 1024)
        R = nx // base
        if R * base != nx:
            raise ValueError(f"lattice side {nx} is not a multiple of {base}")
        big, _ = si.periodic_copies(si.jittered_lattice(base, seed=3), R)
        x, y = big["x"], big["y"]
        fields = [big[k] for k in ("ux", "uy", "q11", "q12", "rho")]
        del big
        n = nx * nx
        steps = int(min(3000, max(20, work // n)))
        p = make_params(B, nx)
        try:
            ctx = B.ann_create(p)
        except B.AnnError as e:   # e.g. a box larger than the device memory: recorded, not fatal
            out.append({"nx": nx, "particles": n, "error": str(e)})
            continue
        try:
            B.ann_set_stream(ctx, stream)
            B.ann_set_particles(ctx, x, y, *fields)
            del x, y, fields
            B.ann_step(ctx, warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                B.ann_step(ctx, steps)
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            d = B.ann_get_diagnostics(ctx)
            g = B.ann_grid_info(p)
            psteps = max(5, steps // 10)
            kprof = B.ann_step_profile(ctx, psteps)
        finally:
            B.ann_destroy(ctx)
        kus = {k: 1e3 * v / psteps for k, v in kprof.items() if v > 0}
        row = {"nx": nx, "particles": n, "tiles": g.tiles_per_side ** 2, "steps": steps,
               "ms_per_step": ms / steps, "particle_steps_per_s": n * steps / (ms * 1e-3),
               "device_gb": g.device_bytes / 1e9, "error_bits": d["error_bits"], "kernel_us": kus}
        if peak_tf and kus.get("pass_d"):
            tf = FLOPS_PER_PAIR["pass_d"] * d["nbr_mean"] * n / (kus["pass_d"] * 1e-6) / 1e12
            row["pass_d_tflops"], row["pass_d_frac"] = tf, tf / peak_tf
        out.append(row)
        print(f"size sweep {nx}^2: {row['particle_steps_per_s']:.3e} particle-steps/s, "
              f"{row['ms_per_step']:.4f} ms per step", file=sys.stderr, flush=True)
    return {"sizes": out, "set-up": "from rest, h = 1.3 dx, zeta 0.08, K 0.02, stable dt; sides above 1024 "
                                    "are copies of a 1024^2 jittered lattice", "clock": "CUDA events"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for _, _, hw, hwt, swt, swp in rows:
            for name, v in (("hw_slowdown", hw), ("hw_thermal_slowdown", hwt),
                            ("sw_thermal_slowdown", swt), ("sw_power_cap", swp)):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def make_params(B, nx):
    p = B.ann_default_params(n=nx * nx, h=1.3 / nx, zeta=PARAMS["zeta"], K=PARAMS["K"], dt_mode=1)
    return p


def _traffic_for(kernel: str):
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        with open(KERNEL_SRC, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if t.get("kernel") == kernel and t.get("source_sha256") == sha:
            return t.get("dram_bytes_per_launch"), t
    except (OSError, ValueError):
        pass
    return None, None


def cpu_baseline(nx: int, budget_s: float = 10.0, max_steps: int = 6):
    """The FP64 oracle, as it stands, on the host cores: whole steps of the same workload."""
    import numpy as np  # noqa: F401

    import oracle
    import sph_inputs as si

    ic = si.jittered_lattice(nx, seed=0)
    h = 1.3 / nx
    dt = min(1e-4, 0.125 * h * h / 1.0, 0.125 * h * h / (0.34 * PARAMS["K"]))
    P = oracle.make_params(h=h, dt=dt, zeta=PARAMS["zeta"], K=PARAMS["K"], nbr_mode="cells")
    st = {k: ic[k] for k in ("x", "y", "ux", "uy", "q11", "q12", "rho")}
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        st, _ = oracle.step(P, st, 1)
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    cores = oracle.num_threads()
    # one core: one step of a 256 x 256 box with the same dx, h and parameters (the same work per
    # particle, a bounded sample)
    n1 = 256
    ic1 = si.jittered_lattice(n1, L=n1 / nx, seed=0)
    P1 = oracle.make_params(L=n1 / nx, h=h, dt=dt, zeta=PARAMS["zeta"], K=PARAMS["K"], nbr_mode="cells")
    oracle.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        oracle.step(P1, {k: ic1[k] for k in ("x", "y", "ux", "uy", "q11", "q12", "rho")}, 1)
        el1 = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(cores)
    return {"value": nx * nx * steps / el, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{steps} whole FP64 oracle step(s) of the {nx}x{nx} workload (cell-grid search, "
                      f"OpenMP over particles), {el:.1f} s",
            "single_core_value": n1 * n1 / el1,
            "single_core_sample": f"1 step of a {n1}x{n1} periodic sub-box (same dx, h, parameters) on 1 core, "
                                  f"{el1:.1f} s"}


def run_reference(args):
    """The oracle on the host cores, timed like our arm: each step one oracle step of a periodic
    sub-box of the workload (same dx, h, parameters and density), sized so the run stays short."""
    import oracle
    import sph_inputs as si

    ws, rank, _ = _rank_info()
    if rank != 0:
        return 0
    oracle.build()
    h = 1.3 / NX
    dt = min(1e-4, 0.125 * h * h, 0.125 * h * h / (0.34 * PARAMS["K"]))
    # calibrate the oracle's cost per particle-step on a 64 x 64 sub-box
    def sub(side):
        L = side / NX
        ic = si.jittered_lattice(side, seed=0, L=L)
        P = oracle.make_params(L=L, h=h, dt=dt, zeta=PARAMS["zeta"], K=PARAMS["K"], nbr_mode="cells")
        return P, {k: ic[k] for k in ("x", "y", "ux", "uy", "q11", "q12", "rho")}
    P, st = sub(64)
    t0 = time.perf_counter()
    oracle.step(P, st, 2)
    per = (time.perf_counter() - t0) / (2 * 64 * 64)
    total = args.steps + args.warmup
    side = int(math.sqrt(max(90.0 / (per * max(total, 1)), 32 * 32)))
    side = max(32, min(NX, side))
    P, st = sub(side)
    for _ in range(args.warmup):
        st, _ = oracle.step(P, st, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, _ = oracle.step(P, st, 1)
    el = time.perf_counter() - t0
    value = side * side * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(1),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: one FP64 oracle step of a {side}x{side} periodic sub-box "
                                   f"of the workload (same dx, h, parameters)"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _config(ws):
    return {"workload": f"sph_active_nematic_{NX}x{NX}", "particles": NX * NX, "h_over_dx": 1.3,
            "zeta": PARAMS["zeta"], "K": PARAMS["K"], "dt": "stable (viscous limit)",
            "box": "periodic unit square", "parallelism": f"ensemble x{ws}" if ws > 1 else "single GPU",
            "l2": "working set > L2 (no flush needed)"}


DIAG_M = 1024          # grid nodes per side of the flow diagnostics (one node per particle)
DIAG_TRACERS = 10000   # pathline particles


def diagnostics_times(B, ctx, n, ic, reps=3):
    """Wall time (ms, synchronised C-ABI calls) of the flow diagnostics on the present state:
    gridding + FFT spectrum (first call after a step), then on the cached grid the correlation and
    the defects; mixing on 64 x 64 bins; unwrapped positions of DIAG_TRACERS particles."""
    import numpy as np

    quad = ((ic["x"] >= 0.5).astype(np.uint8) + 2 * (ic["y"] >= 0.5).astype(np.uint8)).astype(np.uint8)
    B.ann_set_colors(ctx, quad)
    ids = np.arange(0, n, max(n // DIAG_TRACERS, 1))[:DIAG_TRACERS]
    t = {"grid_and_spectrum_ms": [], "correlation_ms": [], "defects_ms": [], "mixing_ms": [],
         "pathlines_ms": []}

    def timed(key, fn):
        t0 = time.perf_counter()
        fn()
        t[key].append(1e3 * (time.perf_counter() - t0))

    for r in range(reps + 1):
        B.ann_step(ctx, 1)   # a new state: the next call grids it afresh
        timed("grid_and_spectrum_ms", lambda: B.ann_energy_spectrum(ctx, DIAG_M))
        timed("correlation_ms", lambda: B.ann_vorticity_correlation(ctx, DIAG_M))
        timed("defects_ms", lambda: B.ann_defects(ctx, DIAG_M))
        timed("mixing_ms", lambda: B.ann_mixing_index(ctx, 64))
        timed("pathlines_ms", lambda: B.ann_get_unwrapped(ctx, ids))
    out = {k: min(v[1:]) for k, v in t.items()}   # the first round allocates and builds tables
    out.update({"grid": DIAG_M, "tracers": int(ids.size), "mix_bins": 64,
                "timing": "min of 3 synchronised calls, wall clock"})
    return out


def oracle_grid_ms(nx, M):
    """The oracle's Shepard gridding (cell list, OpenMP) of the same workload's initial state."""
    import oracle
    from oracle import diagnostics as D
    import sph_inputs as si

    ic = si.jittered_lattice(nx, seed=0)
    t0 = time.perf_counter()
    D.grid_shepard(ic["x"], ic["y"], [ic["ux"], ic["uy"], ic["q11"], ic["q12"]], 1.0, 1.3 / nx, M)
    return 1e3 * (time.perf_counter() - t0), oracle.num_threads()


ENSEMBLE_MEMBERS = 64


def ensemble_members(count=ENSEMBLE_MEMBERS, seed=2021):
    """The batched-ensemble workload: side nx uniform in [128, 512] (n = nx^2, uneven), zeta
    log-uniform in [0.01, 0.2], K uniform in [0.01, 0.08]; the other parameters as the 1M set-up."""
    import math as _m

    import sph_inputs as si

    u = si.uniform53(seed, 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        nx = int(round(128 + 384 * u[k, 0]))
        zeta = _m.exp(_m.log(0.01) + u[k, 1] * (_m.log(0.2) - _m.log(0.01)))
        K = 0.01 + 0.07 * u[k, 2]
        out.append((nx, zeta, K))
    return out


def ensemble_bench(B, steps=5000, trial_steps=10, solo_steps=20):
    """Aggregate particle-steps/s of the ensemble over 5,000 steps (one graph launch per step,
    autotuned grouping) against the same members stepped one after another through their own step
    graphs; each member's solo rate shows how far a small member alone leaves the SMs idle (the
    pair passes of a 128^2 member have 64 tiles of 4 x 4 cells, one block each, for 152 SMs)."""
    import numpy as np  # noqa: F401

    import sph_inputs as si

    spec = ensemble_members()
    plist = []
    for nx, zeta, K in spec:
        p = B.ann_default_params(n=nx * nx, h=1.3 / nx, zeta=zeta, K=K, dt_mode=1)
        plist.append(p)
    ens = B.ann_ensemble_create(plist)
    try:
        total = 0
        for k, (nx, _, _) in enumerate(spec):
            ic = si.jittered_lattice(nx, seed=100 + k)
            B.ann_set_particles(B.ann_ensemble_member(ens, k), ic["x"], ic["y"], ic["ux"], ic["uy"],
                                ic["q11"], ic["q12"], ic["rho"])
            total += nx * nx
        groups, _ = B.ann_ensemble_autotune(ens, trial_steps)
        B.ann_ensemble_step(ens, 2)
        t0 = time.perf_counter()
        B.ann_ensemble_step(ens, steps)
        el = time.perf_counter() - t0
        seq = 0.0
        solo = []
        for k in range(len(spec)):
            ctx = B.ann_ensemble_member(ens, k)
            B.ann_step(ctx, 1)
            t1 = time.perf_counter()
            B.ann_step(ctx, solo_steps)
            dt_k = (time.perf_counter() - t1) / solo_steps
            seq += dt_k
            solo.append((spec[k][0] ** 2, spec[k][0] ** 2 / dt_k))
    finally:
        B.ann_ensemble_destroy(ens)
    solo.sort()
    return {"members": len(spec), "particles": total, "groups": groups, "steps": steps,
            "value": total * steps / el, "unit": METRIC, "ms_per_step": 1e3 * el / steps,
            "sequential_value": total / seq, "sequential_ms_per_step": 1e3 * seq,
            "solo_rate_smallest_8": sum(r for _, r in solo[:8]) / 8, "solo_rate_largest_8": sum(r for _, r in solo[-8:]) / 8,
            "solo_sizes": [solo[0][0], solo[-1][0]],
            "speedup_vs_sequential": (total * steps / el) / (total / seq),
            "workload": "64 members, side U[128, 512], zeta log-U[0.01, 0.2], K U[0.01, 0.08], stable dt",
            "timing": "wall clock around synchronised calls"}


def sweep_bench(B, nx=256, zetas=(-0.08, -0.04, 0.04, 0.08, 0.12), Ks=(0.02, 0.04), chunks=3, chunk=1000,
                M=256):
    """The activity and elastic-constant sweep of the results section (contractile zeta < 0 and
    extensile zeta > 0 against K), run as one ensemble of nx^2 members from the same seeded lattice:
    after every `chunk` steps, each member's defect count (grid M) and mean |Q| (the q field)."""
    import sph_inputs as si

    spec = [(z, K) for K in Ks for z in zetas]
    ens = B.ann_ensemble_create([B.ann_default_params(n=nx * nx, h=1.3 / nx, zeta=z, K=K, dt_mode=1) for z, K in spec])
    rows = [{"zeta": z, "K": K, "defects": [], "mean_q": []} for z, K in spec]
    try:
        ic = si.jittered_lattice(nx, seed=77)
        for k in range(len(spec)):
            B.ann_set_particles(B.ann_ensemble_member(ens, k), ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"],
                                ic["q12"], ic["rho"])
        t0 = time.perf_counter()
        for c in range(chunks + 1):
            if c:
                B.ann_ensemble_step(ens, chunk)
            for k in range(len(spec)):
                ctx = B.ann_ensemble_member(ens, k)
                counts, _ = B.ann_defects(ctx, M)
                rows[k]["defects"].append(int(counts[0] + counts[1]))
                rows[k]["mean_q"].append(B.ann_get_diagnostics(ctx)["mean_q"])
        el = time.perf_counter() - t0
    finally:
        B.ann_ensemble_destroy(ens)
    return {"members": rows, "particles_per_member": nx * nx, "steps": chunks * chunk, "every": chunk, "grid": M,
            "seconds": el, "workload": f"{len(spec)} members of {nx}^2, zeta x K grid, one ensemble"}


SG_K = 8                    # steps one surrogate evaluation spans
SG_TEND = ("AX", "AY", "QRATE11", "QRATE12", "LAPQ11", "LAPQ12", "GRADU_XX", "GRADU_XY", "GRADU_YX", "GRADU_YY")
SG_STATE = ("X", "Y", "UX", "UY", "Q11", "Q12", "DRHO")


def _sg_snapshot(B, ctx, n):
    import numpy as np

    f = {k: B.ann_get_field(ctx, k, n).astype(np.float64) for k in SG_STATE + SG_TEND}
    f["tend"] = np.stack([f["AX"], f["AY"], f["QRATE11"], f["QRATE12"], f["LAPQ11"], f["LAPQ12"],
                          f["GRADU_XX"] + f["GRADU_YY"], f["GRADU_YX"] - f["GRADU_XY"]], axis=1)
    return f


def _sg_params(B, nx, zeta, K):
    return B.ann_default_params(n=nx * nx, h=1.3 / nx, zeta=zeta, K=K, dt_mode=1, c0_min=0.5)


def _sg_run(B, ctx, nx, seed, nsnap, spin, u0):
    """Recorded plain-SPH snapshots every SG_K steps (ID order) of a seeded run on context ctx."""
    import sph_inputs as si

    n = nx * nx
    ic = si.jittered_lattice(nx, seed=seed)
    if u0 > 0:
        r = si.uniform53(seed + 900, 2 * n).reshape(2, n) - 0.5
        ic["ux"], ic["uy"] = u0 * r[0], u0 * r[1]
    B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
    B.ann_set_record(ctx, 1)
    B.ann_step(ctx, spin)
    snaps = []
    for _ in range(nsnap + 1):
        snaps.append(_sg_snapshot(B, ctx, n))
        B.ann_step(ctx, SG_K)
    return snaps


def _sg_trajectory(B, nx, zeta, K, seed, nsnap, spin, u0=0.0):
    """Recorded plain-SPH snapshots every SG_K steps (ID order) and the context parameters."""
    p = _sg_params(B, nx, zeta, K)
    ctx = B.ann_create(p)
    try:
        snaps = _sg_run(B, ctx, nx, seed, nsnap, spin, u0)
        dt = B.ann_grid_info(p).dt_effective
    finally:
        B.ann_destroy(ctx)
    return p, dt, snaps


SG_PRE_TRAJ = 200     # seeded 256 x 256 pre-training trajectories
SG_PRE_ZETAS = 8      # activities in [0.02, 0.1], one context each


def _sg_pretrain(B, sg, nx=256, n_traj=SG_PRE_TRAJ, seed0=300, spin=120, nsnap=2, passes=3, lr0=3e-3):
    """Online pre-training on n_traj seeded trajectories at nx^2: trajectory s has activity
    zeta_(s mod 8) and seed seed0 + s, starts from a lattice with random velocities, runs `spin`
    plain steps and gives nsnap pairs of states SG_K steps apart; each pair is used `passes` times
    as it arrives (Adam, the rate dropping to 0.3 lr0 for the last 30 % of the trajectories).  The
    velocity and residual scales come from the first 8 trajectories; a 201st is held out."""
    import numpy as np

    zetas = [0.02 + 0.08 * q / (SG_PRE_ZETAS - 1) for q in range(SG_PRE_ZETAS)]
    ctxs = [B.ann_create(_sg_params(B, nx, z, PARAMS["K"])) for z in zetas]
    n = nx * nx
    try:
        def pairs_of(s):
            return _sg_pairs(_sg_run(B, ctxs[s % SG_PRE_ZETAS], nx, seed0 + s, nsnap, spin, 0.02))

        first = [pairs_of(s) for s in range(8)]
        flat = [pr for prs in first for pr in prs]
        us = float(np.sqrt(np.mean(np.concatenate([np.r_[a["UX"], a["UY"]] for a, _ in flat]) ** 2)))
        B.ann_surrogate_set_scales(sg, us, 1.0, 1.0, SG_K)
        ys = _sg_scales(_sg_residuals(B, sg, ctxs[0], n, flat))
        B.ann_surrogate_set_scales(sg, us, ys[0], ys[2], SG_K)
        losses, iters = [], 0
        for s in range(n_traj):
            prs = first[s] if s < 8 else pairs_of(s)
            ctx = ctxs[s % SG_PRE_ZETAS]
            lr = lr0 if s < 0.7 * n_traj else 0.3 * lr0
            for _ in range(passes):
                for a, b in prs:
                    _sg_load(B, sg, ctx, a)
                    e = B.ann_surrogate_euler(sg, n).astype(np.float64)
                    loss, _ = B.ann_surrogate_gradients(sg, (_sg_truth(a, b) - e) / ys)
                    B.ann_surrogate_adam(sg, lr)
                    losses.append(loss)
                    iters += 1
        held = pairs_of(n_traj)
        e_net, e_eul = _sg_eval(B, sg, ctxs[n_traj % SG_PRE_ZETAS], n, held, ys)
    finally:
        for c in ctxs:
            B.ann_destroy(c)
    return {"resolution": nx, "trajectories": n_traj, "pairs": n_traj * nsnap, "iters": iters,
            "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:])),
            "heldout_err": e_net, "euler_err": e_eul, "us": us, "ys": [float(ys[0]), float(ys[2])]}


def _sg_pairs(snaps):
    return list(zip(snaps[:-1], snaps[1:]))


def _sg_truth(a, b):
    import numpy as np

    return np.stack([b["Q11"] - a["Q11"], b["Q12"] - a["Q12"], b["UX"] - a["UX"], b["UY"] - a["UY"]], axis=1)


def _sg_load(B, sg, ctx, a):
    B.ann_set_particles(ctx, a["X"], a["Y"], a["UX"], a["UY"], a["Q11"], a["Q12"], 1.0 + a["DRHO"])
    B.ann_surrogate_load(sg, ctx, a["tend"])


def _sg_residuals(B, sg, ctx, n, pairs):
    """(true increment, explicit increment of the library) of every pair."""
    out = []
    for a, b in pairs:
        _sg_load(B, sg, ctx, a)
        out.append((_sg_truth(a, b), B.ann_surrogate_euler(sg, n).astype("float64")))
    return out


def _sg_scales(res, floor: float = 0.0):
    """Output scales ys of the network's correction: the spread of the residual (true increment
    minus the explicit one), at least `floor` times the spread of the true increment.  Where the
    explicit increment is already close (the developed 256^2 flow: 0.3 %), the floor keeps the
    features, which are divided by ys, at a trainable size."""
    import numpy as np

    def spread(cs, of_truth):
        return np.std(np.concatenate([(t if of_truth else t - e)[:, cs].ravel() for t, e in res]))

    ysq = max(spread(slice(0, 2), False), floor * spread(slice(0, 2), True))
    ysu = max(spread(slice(2, 4), False), floor * spread(slice(2, 4), True))
    return np.array([ysq, ysq, ysu, ysu])


def _sg_train(B, sg, ctx, n, pairs, res, ys, iters, lr0):
    import numpy as np

    losses = []
    for it in range(iters):
        a, b = pairs[it % len(pairs)]
        truth, euler = res[it % len(pairs)]
        _sg_load(B, sg, ctx, a)
        loss, _ = B.ann_surrogate_gradients(sg, (truth - euler) / ys)
        B.ann_surrogate_adam(sg, lr0 if it < 0.7 * iters else 0.3 * lr0)
        losses.append(loss)
    return float(np.mean(losses[:10])), float(np.mean(losses[-10:]))


def _sg_eval(B, sg, ctx, n, pairs, ys, parts=False):
    """Relative error of the surrogate's k-step increment, and of the explicit one, on held-out pairs;
    with parts, also each for the Q and the u increments alone."""
    import numpy as np

    en, ee, pq, pu = [], [], [], []
    for a, b in pairs:
        truth = _sg_truth(a, b)
        _sg_load(B, sg, ctx, a)
        euler = B.ann_surrogate_euler(sg, n).astype(np.float64)
        pred = euler + B.ann_surrogate_forward(sg, n) * ys
        scale = np.linalg.norm(truth)
        en.append(np.linalg.norm(pred - truth) / scale)
        ee.append(np.linalg.norm(euler - truth) / scale)
        for acc, cs in ((pq, slice(0, 2)), (pu, slice(2, 4))):
            t = np.linalg.norm(truth[:, cs])
            acc.append((np.linalg.norm(pred[:, cs] - truth[:, cs]) / t, np.linalg.norm(euler[:, cs] - truth[:, cs]) / t))
    if not parts:
        return float(np.mean(en)), float(np.mean(ee))
    return (float(np.mean(en)), float(np.mean(ee)), [float(v) for v in np.mean(pq, axis=0)],
            [float(v) for v in np.mean(pu, axis=0)])


NX3 = 96   # the 3D variant's measured size: 96^3 = 884,736 particles


def _params3(B, nx):
    return B.ann3_default_params(n=nx ** 3, h=1.3 / nx, dt=1e-4, eta=0.2, A=0.05, B=0.3, zeta=0.3, c0_min=0.5)


def three_d_bench(B, nx=NX3, warmup=3, steps=20):
    """The 3D variant on an nx^3 jittered cubic lattice with random directors and small random
    velocities: wall time of `steps` steps in one call (one synchronisation), after `warmup`."""
    import numpy as np

    import sph_inputs as si

    n = nx ** 3
    ic = si.jittered_lattice3(nx, seed=5, jitter=0.1, u_scale=0.02)
    ctx = B.ann3_create(_params3(B, nx))
    try:
        B.ann3_set_particles(ctx, ic["x"], ic["y"], ic["z"], ic["u"], ic["q"], ic["rho"])
        B.ann3_step(ctx, warmup)
        t0 = time.perf_counter()
        B.ann3_step(ctx, steps)
        dt = time.perf_counter() - t0
        nn = B.ann3_get_field(ctx, "NNBR", n)
    finally:
        B.ann3_destroy(ctx)
    ms = 1e3 * dt / steps
    return {"workload": f"sph_active_nematic_3d_{nx}cubed", "particles": n, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "value": n / (ms * 1e-3), "unit": "particle-steps/s",
            "pair_interactions_per_s": float(nn.sum()) / (ms * 1e-3), "nbr_mean": float(nn.mean()),
            "clock": "wall around one synchronised call of `steps` steps"}


def oracle3d_baseline(nx=24, steps=1):
    """The FP64 3D oracle, as it stands, on the host cores: `steps` whole steps of a 24^3 lattice (the
    same set-up as three_d_bench, smaller: the per-particle work is the same)."""
    import oracle
    import sph_inputs as si
    from oracle import oracle3d as O3

    ic = si.jittered_lattice3(nx, seed=5, jitter=0.1, u_scale=0.02)
    P = O3.make_params(h=1.3 / nx, dt=1e-4, eta=0.2, A=0.05, B=0.3, zeta=0.3, c0_min=0.5)
    st = {"x": ic["x"], "y": ic["y"], "z": ic["z"], "u": ic["u"], "q": ic["q"], "rho": ic["rho"]}
    t0 = time.perf_counter()
    O3.step(P, st, steps)
    dt = time.perf_counter() - t0
    n = nx ** 3
    return {"value": n * steps / dt, "unit": "particle-steps/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} whole FP64 3D oracle step(s) of a {nx}^3 lattice, {dt:.1f} s"}


def surrogate_cycles(cycles):
    """Cycles of one recorded plain step and one jump on the 1024^2 workload with the library's
    He-initialised weights; prints the mean wall time of a cycle (synchronised calls)."""
    import sph_inputs as si
    from paper_2108_08919_gb300 import binding as B, build

    build.build()
    n = NX * NX
    p = _sg_params(B, NX, PARAMS["zeta"], PARAMS["K"])
    ctx = B.ann_create(p)
    sg = B.ann_surrogate_create(n)
    try:
        ic = si.jittered_lattice(NX, seed=3)
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
        B.ann_set_record(ctx, 1)
        B.ann_surrogate_init(sg, 7)
        B.ann_surrogate_set_scales(sg, 1e-3, 1e-3, 1e-5, SG_K)
        B.ann_step(ctx, 2)
        t0 = time.perf_counter()
        for _ in range(cycles):
            B.ann_step(ctx, 1)
            B.ann_surrogate_jump(sg, ctx, None)
        ms = 1e3 * (time.perf_counter() - t0) / cycles
    finally:
        B.ann_surrogate_destroy(sg)
        B.ann_destroy(ctx)
    print(json.dumps({"surrogate_cycles": cycles, "ms_per_cycle": ms, "particles": n}))
    return 0


def surrogate_bench(B, max_err=0.05):
    """The learned surrogate: pre-trained on 256 x 256 trajectories, fine-tuned and evaluated on the
    1024 x 1024 workload; held-out k-step error, the speed of one recorded plain step plus a jump
    against k + 1 plain steps, and a short rollout's defect density and spectrum slope against plain
    SPH.  The jump is used only when its validation error is below max_err (else plain SPH)."""
    import numpy as np

    t_all = time.perf_counter()
    out = {"k": SG_K, "max_err": max_err}
    # pre-training: 200 seeded 256 x 256 trajectories, zeta in [0.02, 0.1], streamed
    sg = B.ann_surrogate_create(NX * NX)
    try:
        B.ann_surrogate_init(sg, 7)
        t0 = time.perf_counter()
        out["pretrain"] = _sg_pretrain(B, sg)
        out["pretrain"]["seconds"] = time.perf_counter() - t0
    except BaseException:
        B.ann_surrogate_destroy(sg)
        raise
    # fine-tuning and evaluation at 1024 x 1024 (the workload of the headline metric)
    try:
        n = NX * NX
        # fine-tune on a seed-11 trajectory, hold out a trajectory of another seed (12)
        p1, dt1, sn = _sg_trajectory(B, NX, PARAMS["zeta"], PARAMS["K"], 11, 10, 300, u0=0.02)
        _, _, sn_b = _sg_trajectory(B, NX, PARAMS["zeta"], PARAMS["K"], 12, 4, 300, u0=0.02)
        tr1, te1 = _sg_pairs(sn), _sg_pairs(sn_b)
        us1 = float(np.sqrt(np.mean(np.concatenate([np.r_[a["UX"], a["UY"]] for a, _ in tr1]) ** 2)))
        c1 = B.ann_create(p1)
        try:
            B.ann_surrogate_set_scales(sg, us1, 1.0, 1.0, SG_K)
            res1 = _sg_residuals(B, sg, c1, n, tr1)
            ys1 = _sg_scales(res1)
            B.ann_surrogate_set_scales(sg, us1, ys1[0], ys1[2], SG_K)
            t0 = time.perf_counter()
            l0, l1 = _sg_train(B, sg, c1, n, tr1, res1, ys1, 200, 1e-3)
            e_net, e_eul, e_q, e_u = _sg_eval(B, sg, c1, n, te1, ys1, parts=True)
            out["finetune"] = {"resolution": NX, "pairs": len(tr1), "heldout_pairs": len(te1), "train_seed": 11,
                               "heldout_seed": 12, "iters": 200, "loss_first": l0,
                               "loss_last": l1, "seconds": time.perf_counter() - t0, "heldout_err": e_net,
                               "euler_err": e_eul, "heldout_q_err_net_euler": e_q,
                               "heldout_u_err_net_euler": e_u, "velocity_correction": False}
            use = e_net <= max_err
            out["fallback"] = not use
            # timing on the last held-out state: one recorded plain step + a jump vs k + 1 plain steps
            a = te1[-1][0]

            def load():
                B.ann_set_particles(c1, a["X"], a["Y"], a["UX"], a["UY"], a["Q11"], a["Q12"], 1.0 + a["DRHO"])

            load()
            B.ann_set_record(c1, 1)
            B.ann_step(c1, 3)
            reps = 20
            t_plain = []
            for _ in range(reps):
                t1 = time.perf_counter()
                B.ann_step(c1, SG_K + 1)
                t_plain.append(time.perf_counter() - t1)
            t_cycle = []
            for _ in range(reps):
                t1 = time.perf_counter()
                B.ann_step(c1, 1)
                B.ann_surrogate_jump(sg, c1, None)
                t_cycle.append(time.perf_counter() - t1)
            tp, tc = min(t_plain), min(t_cycle)
            out["timing"] = {"plain_ms_per_cycle": 1e3 * tp, "surrogate_ms_per_cycle": 1e3 * tc,
                             "steps_per_cycle": SG_K + 1, "speedup": tp / tc,
                             "speedup_used": tp / tc if use else 1.0,
                             "clock": "wall, synchronised calls, min of 20"}
            # rollout: 25 guarded cycles from the held-out seed's state (the library checks every
            # 5th cycle against plain SPH on a shadow context and falls back past max_err), against
            # plain SPH from the same state
            cyc, every = 25, 5
            load()
            B.ann_step(c1, 1)
            shadow = B.ann_create(p1)
            try:
                B.ann_get_diagnostics(c1)   # synchronises
                t1 = time.perf_counter()
                guard = B.ann_surrogate_advance(sg, c1, shadow, cyc, every, max_err) if use else None
                t_guarded = time.perf_counter() - t1
            except B.AnnError as ex:
                out["rollout"] = {"cycles": cyc, "error": str(ex)[:200]}
                raise _SgRolloutFailed() from ex
            finally:
                B.ann_destroy(shadow)
            vmax = [B.ann_get_diagnostics(c1)["max_speed"]]
            s_counts, _ = B.ann_defects(c1, 256)
            s_E = B.ann_energy_spectrum(c1, 256)
            s_u = {f: B.ann_get_field(c1, f, n).astype(np.float64) for f in ("UX", "UY", "Q11", "Q12")}
            load()
            B.ann_step(c1, 1)
            B.ann_get_diagnostics(c1)
            t1 = time.perf_counter()
            B.ann_step(c1, cyc * (SG_K + 1))
            t_plain_roll = time.perf_counter() - t1
            p_counts, _ = B.ann_defects(c1, 256)
            p_E = B.ann_energy_spectrum(c1, 256)
            p_u = {f: B.ann_get_field(c1, f, n).astype(np.float64) for f in ("UX", "UY", "Q11", "Q12")}
            w = 2 * np.pi * np.arange(s_E.size)
            sl_s = B.ann_spectrum_slope(s_E, 1.0, w[4], w[60])
            sl_p = B.ann_spectrum_slope(p_E, 1.0, w[4], w[60])
            dq = np.concatenate([s_u["Q11"] - p_u["Q11"], s_u["Q12"] - p_u["Q12"]])
            qn = np.concatenate([p_u["Q11"] - a["Q11"], p_u["Q12"] - a["Q12"]])
            du = np.concatenate([s_u["UX"] - p_u["UX"], s_u["UY"] - p_u["UY"]])
            un = np.concatenate([p_u["UX"] - a["UX"], p_u["UY"] - a["UY"]])
            out["rollout"] = {"cycles": cyc, "steps": cyc * (SG_K + 1) + 1, "surrogate_used": use,
                              "guard": guard, "check_every": every,
                              "guarded_ms": 1e3 * t_guarded if use else None, "plain_ms": 1e3 * t_plain_roll,
                              "guarded_speedup": t_plain_roll / t_guarded if use else 1.0,
                              "max_speed": vmax,
                              "defect_density": [float(s_counts[0] + s_counts[1]), float(p_counts[0] + p_counts[1])],
                              "defect_density_rel_err": abs(float(s_counts[0] + s_counts[1] - p_counts[0] - p_counts[1]))
                              / max(float(p_counts[0] + p_counts[1]), 1.0),
                              "spectrum_slope": [sl_s, sl_p], "spectrum_slope_abs_err": abs(sl_s - sl_p),
                              "q_increment_rel_err": float(np.linalg.norm(dq) / np.linalg.norm(qn)),
                              "u_increment_rel_err": float(np.linalg.norm(du) / np.linalg.norm(un)),
                              "grid": 256, "slope_range": "w in [2 pi 4, 2 pi 60]"}
        except _SgRolloutFailed:
            pass
        finally:
            B.ann_destroy(c1)
    finally:
        B.ann_surrogate_destroy(sg)
    out["seconds"] = time.perf_counter() - t_all
    return out


class _SgRolloutFailed(Exception):
    pass


def surrogate_developed_bench(B, nx=256, zeta=0.1, K=0.02, develop=100000, train_seeds=(21, 23, 25, 27, 29, 31),
                              pairs_per_seed=8, heldout_seed=22, heldout_pairs=6, iters=1500, cycles=40, every=5,
                              max_err=0.05, ys_floor=0.05):
    """The surrogate in the developed active flow of the long runs: nx^2, the scaled viscosity
    eta = 0.03 and dt = 1e-4 (paper_2108_08919_gb300.longrun), zeta = 0.1, K = 0.02.  One ensemble
    runs `develop` plain steps from a random director for every training seed and the held-out
    seed (t = 10: the activity-built order and flow of the long-run tables).  The network (output
    layer initialised to zero) is trained on `pairs_per_seed` 8-step pairs of each training seed's
    developed trajectory, its increments are held out on another seed's, and a guarded rollout
    (ann_surrogate_advance, a plain-SPH check every `every` cycles, fallback past max_err) runs
    from the held-out developed state beside plain SPH: spectrum slope, defect density, increments."""
    import numpy as np

    import sph_inputs as si
    from paper_2108_08919_gb300 import longrun

    t_all = time.perf_counter()
    p = longrun.member_params(nx, zeta, K)
    n = nx * nx
    seeds = list(train_seeds) + [heldout_seed]
    out = {"resolution": nx, "zeta": zeta, "K": K, "eta": p.eta, "dt": p.dt, "develop_steps": develop,
           "max_err": max_err}

    def snaps(ctx, count):
        got = []
        for _ in range(count + 1):
            got.append(_sg_snapshot(B, ctx, n))
            B.ann_step(ctx, SG_K)
        return got

    ca, cb, shadow = B.ann_create(p), B.ann_create(p), B.ann_create(p)
    sg = B.ann_surrogate_create(n)
    ens = B.ann_ensemble_create([p] * len(seeds))
    try:
        for k, seed in enumerate(seeds):
            ic = si.jittered_lattice(nx, seed=seed)
            B.ann_set_particles(B.ann_ensemble_member(ens, k), ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"],
                                ic["q12"], ic["rho"])
        t0 = time.perf_counter()
        try:
            B.ann_ensemble_step(ens, develop)
        except B.AnnError as e:   # a failed member keeps its last completed state; the others ran on
            out["develop_error"] = str(e)
        out["develop_seconds"] = time.perf_counter() - t0

        def take(k, ctx):
            # continue member k's developed trajectory on ctx, with the last acceleration, recorded
            st = B.ann_get_state(B.ann_ensemble_member(ens, k), n)
            B.ann_set_state(ctx, st)
            B.ann_update_state(ctx, st)
            B.ann_set_record(ctx, 1)
            B.ann_step(ctx, 1)

        tr = []
        for k in range(len(train_seeds)):
            take(k, ca)
            tr += _sg_pairs(snaps(ca, pairs_per_seed))
        take(len(train_seeds), cb)
        te = _sg_pairs(snaps(cb, heldout_pairs))
        out["vrms_developed"] = float(np.sqrt(2.0 * B.ann_get_diagnostics(cb)["kinetic_energy"]))
        B.ann_surrogate_init(sg, 7)
        us = float(np.sqrt(np.mean(np.concatenate([np.r_[a["UX"], a["UY"]] for a, _ in tr]) ** 2)))
        B.ann_surrogate_set_scales(sg, us, 1.0, 1.0, SG_K)
        res = _sg_residuals(B, sg, ca, n, tr)
        ys = _sg_scales(res, ys_floor)
        B.ann_surrogate_set_scales(sg, us, ys[0], ys[2], SG_K)
        t0 = time.perf_counter()
        l0, l1 = _sg_train(B, sg, ca, n, tr, res, ys, iters, 1e-3)
        e_net, e_eul, e_q, e_u = _sg_eval(B, sg, ca, n, te, ys, parts=True)
        out["train"] = {"pairs": len(tr), "seeds": list(train_seeds), "heldout_pairs": len(te),
                        "heldout_seed": heldout_seed, "iters": iters, "ys_floor": ys_floor,
                        "loss_first": l0, "loss_last": l1, "seconds": time.perf_counter() - t0,
                        "heldout_err": e_net, "euler_err": e_eul, "heldout_q_err_net_euler": e_q,
                        "heldout_u_err_net_euler": e_u}
        a = te[-1][1]

        def load(ctx):
            B.ann_set_particles(ctx, a["X"], a["Y"], a["UX"], a["UY"], a["Q11"], a["Q12"], 1.0 + a["DRHO"])
            B.ann_set_record(ctx, 1)
            B.ann_step(ctx, 1)
            B.ann_get_diagnostics(ctx)

        load(cb)
        t1 = time.perf_counter()
        guard = B.ann_surrogate_advance(sg, cb, shadow, cycles, every, max_err)
        t_g = time.perf_counter() - t1
        s_counts, _ = B.ann_defects(cb, nx)
        s_E = B.ann_energy_spectrum(cb, nx)
        s_f = {f: B.ann_get_field(cb, f, n).astype(np.float64) for f in ("UX", "UY", "Q11", "Q12")}
        load(ca)
        t1 = time.perf_counter()
        B.ann_step(ca, cycles * (SG_K + 1))
        t_p = time.perf_counter() - t1
        p_counts, _ = B.ann_defects(ca, nx)
        p_E = B.ann_energy_spectrum(ca, nx)
        p_f = {f: B.ann_get_field(ca, f, n).astype(np.float64) for f in ("UX", "UY", "Q11", "Q12")}
        # the same cycles without the guard's checks (recorded plain step + jump): what the checks cost
        load(cb)
        t1 = time.perf_counter()
        for _ in range(cycles):
            B.ann_step(cb, 1)
            B.ann_surrogate_jump(sg, cb, None)
        B.ann_get_diagnostics(cb)
        t_u = time.perf_counter() - t1
        w = 2 * np.pi * np.arange(s_E.size)
        sl_s, sl_p = B.ann_spectrum_slope(s_E, 1.0, w[3], w[20]), B.ann_spectrum_slope(p_E, 1.0, w[3], w[20])
        ds, dp = float(s_counts[0] + s_counts[1]), float(p_counts[0] + p_counts[1])

        def rel(fa, fb, ref):
            num = np.linalg.norm(np.concatenate([fa[0] - fb[0], fa[1] - fb[1]]))
            den = np.linalg.norm(np.concatenate([fb[0] - ref[0], fb[1] - ref[1]]))
            return float(num / den) if den > 0 else float("nan")

        out["rollout"] = {"cycles": cycles, "check_every": every, "guard": guard,
                          "guarded_ms": 1e3 * t_g, "plain_ms": 1e3 * t_p, "speedup": t_p / t_g,
                          "unguarded_ms": 1e3 * t_u, "unguarded_speedup": t_p / t_u,
                          "defect_density": [ds, dp], "defect_density_rel_err": abs(ds - dp) / max(dp, 1.0),
                          "spectrum_slope": [sl_s, sl_p], "spectrum_slope_abs_err": abs(sl_s - sl_p),
                          "q_increment_rel_err": rel((s_f["Q11"], s_f["Q12"]), (p_f["Q11"], p_f["Q12"]),
                                                     (a["Q11"], a["Q12"])),
                          "u_increment_rel_err": rel((s_f["UX"], s_f["UY"]), (p_f["UX"], p_f["UY"]), (a["UX"], a["UY"])),
                          "slope_range": "w in [2 pi 3, 2 pi 20]", "grid": nx}
    finally:
        B.ann_surrogate_destroy(sg)
        B.ann_ensemble_destroy(ens)
        for c in (ca, cb, shadow):
            B.ann_destroy(c)
    out["seconds"] = time.perf_counter() - t_all
    return out


def run_ours(args):
    import numpy as np
    import torch

    import sph_inputs as si
    from paper_2108_08919_gb300 import binding as B
    from paper_2108_08919_gb300 import build as cuda_build

    ws, rank, local = _rank_info()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    if dist:
        dist.barrier()
    n = NX * NX
    p = make_params(B, NX)
    grid = B.ann_grid_info(p)
    ic = si.jittered_lattice(NX, seed=ensemble_seed(rank))
    ctx = B.ann_create(p)
    stream = torch.cuda.Stream()
    B.ann_set_stream(ctx, stream)
    B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
    B.ann_step(ctx, max(args.warmup, 3))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    resorts0 = B.ann_get_diagnostics(ctx)["resorts"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            e0.record(stream)
            B.ann_step(ctx, args.steps)
            e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_max = slowest(e0.elapsed_time(e1), dist, "cuda")
    diag = B.ann_get_diagnostics(ctx)
    resorts_timed = diag["resorts"] - resorts0
    pairs_per_step = diag["nbr_mean"] * n
    value = job_throughput(ws, n, args.steps, ms_max * 1e-3)

    # per-kernel device times (CUDA events around each kernel launch, same stream, same state)
    # (the re-sort branch runs in some steps, pass_a in the others: kernel_ms is the per-step
    # average, avg_launch_ms the average over the launches that ran)
    rp0 = B.ann_get_diagnostics(ctx)["resorts"]
    kprof = B.ann_step_profile(ctx, args.profile_steps)
    rp = B.ann_get_diagnostics(ctx)["resorts"] - rp0
    kms = {k: v / args.profile_steps for k, v in kprof.items()}
    klaunch = {k: (rp if k in RESORT_BRANCH else args.profile_steps - rp if k == "pass_a"
                   else args.profile_steps) for k in kprof}
    dom = max(kms, key=kms.get)
    dom_launch_ms = kprof[dom] / max(klaunch[dom], 1)

    # end to end through the C-ABI with host buffers: the host holds the state between steps, in
    # pinned arrays and in the precision the library keeps it (with the last acceleration);
    # every step uploads it (ann_update_state), advances one step and reads it back (ann_get_state)
    src = {"X": ic["x"], "Y": ic["y"], "UX": ic["ux"], "UY": ic["uy"], "Q11": ic["q11"], "Q12": ic["q12"],
           "DRHO": np.asarray(ic["rho"]) / p.rho0 - 1.0, "AX": np.zeros(n), "AY": np.zeros(n)}
    pin = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=B.field_dtype(k))).pin_memory().numpy()
           for k, v in src.items()}
    B.ann_set_state(ctx, pin)
    B.ann_step(ctx, 1)
    B.ann_get_state(ctx, n, out=pin)
    h2d = d2h = sum(a.nbytes for a in pin.values())
    e2e_steps = max(5, min(50, args.steps // 20))

    def e2e_iter():
        B.ann_update_state(ctx, pin)
        B.ann_step(ctx, 1)
        B.ann_get_state(ctx, n, out=pin)

    e2e_iter()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_iter()
    torch.cuda.synchronize()
    e2e_el = time.perf_counter() - t0
    e2e_value = job_throughput(ws, n, e2e_steps, slowest(e2e_el, dist, "cuda"))
    diag_times = diagnostics_times(B, ctx, n, ic) if rank == 0 else None
    B.ann_destroy(ctx)
    fma = B.ann_fp32_fma_peak(stream) if rank == 0 else None
    developed = developed_flow_bench(B, stream) if rank == 0 and not args.no_developed_flow else None

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peaks, src = _peaks()
    clocks = clk.summary()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    flops_launch = FLOPS_PER_PAIR.get(dom, 0.0) * pairs_per_step
    achieved_tf = flops_launch / (dom_launch_ms * 1e-3) / 1e12 if dom_launch_ms > 0 else 0.0
    nominal_tf = fp32_peak_tflops(sm_mhz, fma["sms"])
    peak_tf = max(fma["scalar"], fma["pair"])
    traffic, _ = _traffic_for(dom)
    bytes_launch = BYTES_PER_PARTICLE.get(dom, 0) * n
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 positions and reductions)",
        "data": "synthetic", "config": _config(ws),
        "pair_interactions_per_s": pairs_per_step * ws * args.steps / (ms_max * 1e-3),
        "dt": grid.dt_effective,
        "roofline": {"kernel": dom, "bound": "alu", "achieved": achieved_tf,
                     "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                     "traffic": traffic,
                     "peak_source": f"measured: project FMA microbenchmark ann_fp32_fma_peak, {fma['sms']} SMs, "
                                    f"scalar {fma['scalar']:.1f}, two-lane {fma['pair']:.1f} TFLOP/s (the larger); "
                                    f"nominal {fma['sms']} SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz = {nominal_tf:.1f}",
                     "flops_per_launch": flops_launch, "avg_launch_ms": dom_launch_ms,
                     "hbm_achieved_gbs": bytes_launch / (dom_launch_ms * 1e-3) / 1e9,
                     "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": src,
                     "hbm_frac": bytes_launch / (dom_launch_ms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0)},
        "kernel_ms": kms,
        "kernel_launches": klaunch,
        "kernel_share": {k: v / sum(kms.values()) for k, v in kms.items()},
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": launches_in_steps(args.steps, resorts_timed),
        "resorts": resorts_timed,
        "clocks": clocks,
        "diag": {"nbr_mean": diag["nbr_mean"], "error_bits": diag["error_bits"],
                 "band_checks": diag["band_checks"], "max_speed": diag["max_speed"]},
    }
    if diag_times is not None:
        line["diagnostics"] = diag_times
    line["developed_flow"] = developed
    if ws == 1 and not args.no_ensemble:
        line["ensemble"] = ensemble_bench(B)
    if ws == 1 and not args.no_surrogate:
        line["surrogate"] = surrogate_bench(B)
        line["surrogate_developed"] = surrogate_developed_bench(B)
    if ws == 1 and not args.no_3d:
        line["three_d"] = three_d_bench(B, nx=args.nx3)
    if ws == 1 and not args.no_sweep:
        line["sweep"] = sweep_bench(B)
    if ws == 1 and args.size_sweep:
        line["size_sweep"] = size_sweep_bench(B, stream, tuple(int(v) for v in args.size_sweep.split(",")),
                                              peak_tf=peak_tf)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(NX)
        ms, cores = oracle_grid_ms(NX, DIAG_M)
        line["diagnostics"]["oracle_grid_ms"] = ms
        line["diagnostics"]["oracle_cores"] = cores
        if "three_d" in line:
            line["three_d"]["cpu_baseline"] = oracle3d_baseline()
    print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


LONG_RUN_MEMBERS = ((0.02, 0.04), (0.05, 0.04), (0.1, 0.04), (0.1, 0.02), (0.1, 0.01))


def long_run(steps: int, every: int, nx: int = 256):
    """Long-run statistics of the 256^2 configuration (results section): the activities
    zeta = 0.02, 0.05, 0.1 at K = 0.04 and, at zeta = 0.1, K = 0.02 and 0.01, as one ensemble,
    from the configurations' random director and from the results section's perturbed nematic.
    Prints one JSON line: per initial condition and member, the statistics every `every` steps
    and their means over the last ten snapshots."""
    from paper_2108_08919_gb300 import build as cuda_build
    from paper_2108_08919_gb300 import longrun

    cuda_build.build()
    out = {"metric": "long-run statistics", "workload": f"{nx}^2 members, zeta x K, scaled eta = 0.03, dt = 1e-4",
           "steps": steps, "every": every, "runs": {}}
    for init in ("random_director", "perturbed_nematic"):
        res = longrun.run(LONG_RUN_MEMBERS, nx=nx, steps=steps, every=every, initial=init)
        keep = ("step", "t", "vrms", "mean_q", "defect_density", "corr_zero", "slope", "nbr_max")
        out["runs"][init] = {
            "seconds": res["seconds"], "summary": longrun.summary(res),
            "series": [{"zeta": m["zeta"], "K": m["K"], "failed": m["failed"],
                        "snapshots": [{k: s[k] for k in keep} for s in m["snapshots"]]} for m in res["members"]]}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--profile-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-member ensemble measurement")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate measurement")
    ap.add_argument("--no-3d", action="store_true", help="skip the three-dimensional variant's measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the activity / elastic-constant sweep")
    ap.add_argument("--no-developed-flow", action="store_true", help="skip the moving-state re-sort timing")
    ap.add_argument("--nx3", type=int, default=NX3, help="side of the 3D variant's cubic lattice")
    ap.add_argument("--size-sweep", default="", metavar="SIDES",
                    help="also time the step at these lattice sides (comma-separated, e.g. 256,1024,8192)")
    ap.add_argument("--surrogate-cycles", type=int, default=0,
                    help="only run this many surrogate cycles (recorded step + jump) at the headline size, "
                         "untrained weights, and print their wall time (for launch lists and profiles)")
    ap.add_argument("--long-run", type=int, default=0, metavar="STEPS",
                    help="only run the long-run statistics (this many steps per member) and print them")
    ap.add_argument("--long-run-every", type=int, default=500, help="snapshot interval of --long-run")
    args = ap.parse_args()
    if args.long_run > 0:
        return long_run(args.long_run, args.long_run_every)
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate_cycles > 0:
        return surrogate_cycles(args.surrogate_cycles)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
