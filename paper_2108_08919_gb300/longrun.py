"""Long runs judged by the statistics of the paper's results section (§5).

The results section characterises active turbulence by its statistics rather than by trajectories:
the kinetic-energy spectrum E(w) and its slope at intermediate w (Eq. 31), the vorticity
correlation and its zero-crossing length (Eq. 32), the number of +1/2 and -1/2 defects, the rms
velocity and the nematic order.  `run` advances several (zeta, K) members of one size together
(one ensemble, one CUDA graph per step) and records these statistics every `every` steps, all
computed on the GPU by the library's diagnostics (ann_energy_spectrum, ann_vorticity_correlation,
ann_defects, ann_get_diagnostics) on an M x M grid.

Parameters follow the paper's 2D set-up (Gamma 0.34, lambda 0.7, A 0, C 1, rho0 1) with two readings
needed to reach active times in a finite number of steps:
  * the viscosity is scaled (eta = `eta`, default 0.03) so that the configurations' dt = 1e-4 is
    below the explicit viscous limit 0.125 h^2 / nu at 256^2 (nu <= 0.032); with eta = 1 that limit
    is 3e-6 and the active time eta / zeta = 20 would need ~10^7 steps;
  * the sound speed has the floor c0_min = 10 v_Q with the paper's active velocity
    v_Q = l_Q zeta / Gamma, l_Q = sqrt(K / zeta) (§5), so that the flow stays weakly compressible.
Steps run in ANN_DT_CHECK mode: a member whose step would break a stability limit stops with
CFL_VIOLATION, keeping the state of its last completed step, and is reported as such.
"""
from __future__ import annotations

import math
import time

import numpy as np

import sph_inputs as si

from . import binding as B

DT_CHECK = 2   # ann_params.dt_mode: dt as given, a step beyond a stability limit fails


def active_scales(zeta: float, K: float, Gamma: float = 0.34):
    """(l_Q, v_Q): the active length sqrt(K / |zeta|) and velocity l_Q |zeta| / Gamma of §5."""
    lq = math.sqrt(K / abs(zeta))
    return lq, lq * abs(zeta) / Gamma


def member_params(nx: int, zeta: float, K: float, eta: float = 0.03, dt: float = 1e-4):
    """ann_params of one member on an nx x nx jittered lattice (h = 1.3 dx)."""
    _, vq = active_scales(zeta, K)
    return B.ann_default_params(n=nx * nx, h=1.3 / nx, zeta=zeta, K=K, eta=eta, dt=dt, c0_min=10.0 * vq,
                                dt_mode=DT_CHECK)


def snapshot(ctx, M: int, shells=(3, 20)):
    """Statistics of the present state: t, rms velocity, kinetic energy, mean q, the mean and largest
    neighbour counts (particle disorder: 44 on the initial lattice), defect counts and
    density (per unit area of the unit box), the vorticity correlation's zero-crossing and 0.2-max
    lengths, and the spectrum's slope over the shells n in [shells[0], shells[1]] (w = 2 pi n)."""
    d = B.ann_get_diagnostics(ctx)
    E = B.ann_energy_spectrum(ctx, M)
    w1, w2 = 2.0 * math.pi * shells[0], 2.0 * math.pi * shells[1]
    slope = B.ann_spectrum_slope(E, 1.0, w1, w2) if E[shells[0]:shells[1] + 1].min() > 0.0 else float("nan")
    _, (l0, l02) = B.ann_vorticity_correlation(ctx, M)
    counts, _ = B.ann_defects(ctx, M)
    return {"step": int(d["step"]), "t": d["t"], "vrms": math.sqrt(2.0 * d["kinetic_energy"]),
            "kinetic_energy": d["kinetic_energy"], "max_speed": d["max_speed"], "mean_q": d["mean_q"],
            "nbr_mean": d["nbr_mean"], "nbr_max": int(d["nbr_max"]),
            "defects_plus": int(counts[0]), "defects_minus": int(counts[1]),
            "defect_density": float(counts[0] + counts[1]), "corr_zero": l0, "corr_02": l02, "slope": slope,
            "spectrum": E.tolist()}


INITIAL = {
    # the configurations' initial condition: a random director angle per particle, S = 1
    "random_director": lambda nx, seed: si.jittered_lattice(nx, seed=seed),
    # the results section's: a slightly perturbed ordered nematic (director along x, +-0.05 rad)
    "perturbed_nematic": lambda nx, seed: si.perturbed_nematic(nx, seed=seed, angle=0.0, spread=0.1),
}


def run(members, nx: int = 256, steps: int = 20000, every: int = 500, eta: float = 0.03, dt: float = 1e-4,
        seed: int = 1, M: int = 256, keep_spectra: bool = False, initial: str = "random_director",
        on_snapshot=None):
    """Advance every (zeta, K) member from the same seeded lattice (initial condition `initial`, at
    rest) for `steps` steps, recording `snapshot` every `every` steps (and at step 0).  Returns a
    dict with one series per member, the failure (if any) of each, and the wall time.
    on_snapshot(k, ctx, snap), if given, is called with each member's context right after its
    snapshot (to inspect the state the statistics were taken from)."""
    specs = [member_params(nx, z, K, eta, dt) for z, K in members]
    ens = B.ann_ensemble_create(specs)
    series = [{"zeta": z, "K": K, "eta": eta, "dt": dt, "c0_min": specs[k].c0_min,
               "l_Q": active_scales(z, K)[0], "v_Q": active_scales(z, K)[1], "snapshots": [], "failed": None}
              for k, (z, K) in enumerate(members)]
    try:
        ic = INITIAL[initial](nx, seed)
        for k in range(len(members)):
            B.ann_set_particles(B.ann_ensemble_member(ens, k), ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"],
                                ic["q12"], ic["rho"])
        t0 = time.perf_counter()
        done = 0
        while True:
            for k in range(len(members)):
                if series[k]["failed"] is None:
                    ctx = B.ann_ensemble_member(ens, k)
                    s = snapshot(ctx, M)
                    if on_snapshot is not None:
                        on_snapshot(k, ctx, s)
                    if not keep_spectra:
                        s.pop("spectrum")
                    series[k]["snapshots"].append(s)
            if done >= steps:
                break
            chunk = min(every, steps - done)
            try:
                B.ann_ensemble_step(ens, chunk)
            except B.AnnError as e:
                # a member that failed keeps its last completed state; the others advanced
                for k in range(len(members)):
                    d = B.ann_get_diagnostics(B.ann_ensemble_member(ens, k))
                    if d["error_bits"] and series[k]["failed"] is None:
                        series[k]["failed"] = {"step": int(d["step"]), "error_bits": int(d["error_bits"]),
                                               "message": str(e)}
                if all(s["failed"] is not None for s in series):
                    break
            done += chunk
        seconds = time.perf_counter() - t0
    finally:
        B.ann_ensemble_destroy(ens)
    return {"members": series, "particles_per_member": nx * nx, "steps": steps, "every": every, "grid": M,
            "initial": initial, "slope_shells": [3, 20], "seconds": seconds}


def summary(result, tail: int = 10):
    """Per member: the mean of each statistic over the last `tail` snapshots (the developed state)."""
    out = []
    keys = ("vrms", "mean_q", "defect_density", "corr_zero", "corr_02", "slope", "nbr_mean", "nbr_max")
    for m in result["members"]:
        snaps = [s for s in m["snapshots"] if s["step"] > 0][-tail:]
        row = {"zeta": m["zeta"], "K": m["K"], "l_Q": m["l_Q"], "failed": m["failed"], "snapshots": len(snaps)}
        for k in keys:
            v = np.array([s[k] for s in snaps], dtype=np.float64)
            v = v[np.isfinite(v)]
            row[k] = float(v.mean()) if v.size else float("nan")
        out.append(row)
    return out
