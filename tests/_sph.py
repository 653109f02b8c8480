"""Helpers shared by the GPU parity tests: one parameter vocabulary mapped onto both the oracle and
the C-ABI, runners for each side, and the error measure.

Parity measure: the normwise relative error ||gpu - oracle||_2 / ||oracle||_2 of a whole field over
all particles, the measure the 1e-5 FP32 bound is stated in.  Vector and tensor fields are measured
as such (all their components together): velocity (ux, uy), acceleration, div Q, Q (q11, q12), the
correction tensor B (B11, B12, B12, B22), the velocity gradient (4 components), lap Q.  A lone
off-diagonal component such as B12 is small on a near-isotropic particle set, so its error relative
to itself says nothing about the accuracy of B.

Positions are compared through the displacement from the start (minimum image).  Both sides store
positions in FP64, so a displacement is only resolved to the rounding of the position itself: the
comparison allows one FP64 unit in the last place of L per coordinate on top of the relative bound.
"""
import math

import numpy as np

import sph_inputs as si

# The paper's 2D set-up for the 64 x 64 and 256 x 256 lattices (dx = 1/nx, h = 1.3 dx).
BASE = dict(L=1.0, dt=1e-4, rho0=1.0, eta=1.0, Gamma=0.34, lam=0.7, A=0.0, B=0.0, C=1.0, K=0.04,
            zeta=0.05, gamma_eos=7.0, beta=1.0, c0_min=0.0, c_shift=1.0 / 3.0, apd=1,
            conservative=0, q_new_in_momentum=1, elastic=0)

STATE = ("x", "y", "ux", "uy", "q11", "q12", "drho", "ax", "ay")
GPU_NAME = {"x": "X", "y": "Y", "ux": "UX", "uy": "UY", "q11": "Q11", "q12": "Q12",
            "drho": "DRHO", "ax": "AX", "ay": "AY"}


def params(nx, **kw):
    p = dict(BASE)
    p["h"] = 1.3 / nx * p["L"]
    p.update(kw)
    return p


def stable_dt(p):
    """The smaller of the given dt and the explicit viscous and Q-diffusion limits 0.125 h^2/D."""
    h = p["h"]
    dt = p["dt"]
    nu = p["eta"] / p["rho0"]
    if nu > 0:
        dt = min(dt, 0.125 * h * h / nu)
    if p["Gamma"] * p["K"] > 0:
        dt = min(dt, 0.125 * h * h / (p["Gamma"] * p["K"]))
    return dt


def oracle_params(orc, p, nbr_mode="brute"):
    return orc.make_params(nbr_mode=nbr_mode, **p)


def gpu_params(B, p, n):
    return B.ann_default_params(
        n=n, L=p["L"], h=p["h"], dt=p["dt"], rho0=p["rho0"], eta=p["eta"], Gamma=p["Gamma"],
        lambda_=p["lam"], A=p["A"], B=p["B"], C=p["C"], K=p["K"], zeta=p["zeta"],
        gamma_eos=p["gamma_eos"], beta=p["beta"], c0_min=p["c0_min"], c_shift=p["c_shift"],
        apd=p["apd"], momentum_mode=p["conservative"], q_new_in_momentum=p["q_new_in_momentum"],
        dt_mode=0, elastic_stress=p.get("elastic", 0))


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def min_image(d, L=1.0):
    return (d + 0.5 * L) % L - 0.5 * L


class GpuRun:
    """A context holding one state, advanced through the C-ABI."""

    def __init__(self, B, p, ic):
        self.B = B
        self.n = int(ic["n"]) if "n" in ic else len(ic["x"])
        self.ctx = B.ann_create(gpu_params(B, p, self.n))
        rho = ic.get("rho")
        B.ann_set_particles(self.ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], rho)

    def field(self, name):
        return self.B.ann_get_field(self.ctx, name, self.n).astype(np.float64)

    def state(self):
        return {k: self.field(GPU_NAME[k]) for k in STATE}

    def step(self, k=1):
        self.B.ann_step(self.ctx, k)

    def close(self):
        self.B.ann_destroy(self.ctx)
        self.ctx = None


def oracle_state(ic, rho0=1.0):
    return {"x": ic["x"], "y": ic["y"], "ux": ic["ux"], "uy": ic["uy"], "q11": ic["q11"],
            "q12": ic["q12"], "rho": ic.get("rho", np.full(len(ic["x"]), rho0))}


def relerr_group(gpu_parts, ref_parts):
    return relerr(np.concatenate([np.ravel(a) for a in gpu_parts]),
                  np.concatenate([np.ravel(a) for a in ref_parts]))


def displacement_error(gpu, ref, x0, y0, L=1.0):
    """Relative error of the displacement field, net of the FP64 position rounding."""
    dg = np.concatenate([min_image(gpu["x"] - x0, L), min_image(gpu["y"] - y0, L)])
    do = np.concatenate([min_image(ref["x"] - x0, L), min_image(ref["y"] - y0, L)])
    noise = math.sqrt(dg.size) * np.spacing(L)
    nd = np.linalg.norm(do)
    if nd == 0.0:
        return 0.0 if np.linalg.norm(dg - do) <= noise else float("inf")
    return max(0.0, np.linalg.norm(dg - do) - noise) / nd


def compare_state(gpu, orc_state, x0, y0, rho0=1.0):
    """Normwise relative errors of every state field (positions as displacements)."""
    return {
        "disp": displacement_error(gpu, orc_state, x0, y0),
        "u": relerr_group([gpu["ux"], gpu["uy"]], [orc_state["ux"], orc_state["uy"]]),
        "Q": relerr_group([gpu["q11"], gpu["q12"]], [orc_state["q11"], orc_state["q12"]]),
        "a": relerr_group([gpu["ax"], gpu["ay"]], [orc_state["ax"], orc_state["ay"]]),
        "drho": relerr(gpu["drho"], orc_state["rho"] / rho0 - 1.0),
    }


def random_velocity_ic(nx, seed, u_scale=1e-3, rho_scale=0.0):
    ic = si.jittered_lattice(nx, seed=seed)
    r = si.uniform53(seed + 1000, 3 * ic["n"]).reshape(3, ic["n"]) - 0.5
    ic["ux"] = u_scale * r[0]
    ic["uy"] = u_scale * r[1]
    ic["rho"] = 1.0 + rho_scale * r[2]
    return ic


def smooth_ic(nx, seed, u_amp=1e-2):
    """Smooth periodic velocity (with rotation and divergence), director and density fields: the
    pair sums of smooth fields cancel to leading order, which exercises FP32 accumulation."""
    ic = si.jittered_lattice(nx, seed=seed)
    x, y = ic["x"], ic["y"]
    tp = 2 * math.pi
    ic["ux"] = u_amp * np.sin(tp * x + 0.3) * np.cos(tp * y)
    ic["uy"] = u_amp * (0.5 * np.sin(tp * y) * np.cos(tp * x + 1.0) + 0.4 * np.sin(tp * x))
    th = 0.7 * np.sin(tp * x) + 0.4 * np.cos(2 * tp * y)
    ic["q11"] = 0.8 * np.cos(2 * th)
    ic["q12"] = 0.8 * np.sin(2 * th)
    ic["rho"] = 1.0 + 1e-4 * np.cos(tp * (x + y))
    return ic


def maxerr_group(gpu_parts, ref_parts):
    """Element-wise error of a (vector or tensor) field: max over particles of |g_i - o_i| divided
    by max over particles of |o_i|, the components of a particle taken together.  A few particles
    wrong at 1e-3 pass a normwise bound at 1M particles but not this one."""
    g = np.stack([np.ravel(np.asarray(a, dtype=np.float64)) for a in gpu_parts], axis=1)
    o = np.stack([np.ravel(np.asarray(a, dtype=np.float64)) for a in ref_parts], axis=1)
    scale = np.sqrt((o * o).sum(axis=1)).max()
    diff = np.sqrt(((g - o) ** 2).sum(axis=1)).max()
    if scale == 0.0:
        return float(diff)
    return float(diff / scale)


def compare_state_max(gpu, orc_state, x0, y0, rho0=1.0, L=1.0):
    """Element-wise errors of every state field (maxerr_group); displacements net of one FP64 unit
    of L per coordinate, the resolution of a stored position."""
    dg = np.stack([min_image(gpu["x"] - x0, L), min_image(gpu["y"] - y0, L)], axis=1)
    do = np.stack([min_image(orc_state["x"] - x0, L), min_image(orc_state["y"] - y0, L)], axis=1)
    noise = math.sqrt(2.0) * np.spacing(L)
    scale = np.sqrt((do * do).sum(axis=1)).max()
    diff = max(0.0, np.sqrt(((dg - do) ** 2).sum(axis=1)).max() - noise)
    return {
        "disp": diff / scale if scale > 0 else diff,
        "u": maxerr_group([gpu["ux"], gpu["uy"]], [orc_state["ux"], orc_state["uy"]]),
        "Q": maxerr_group([gpu["q11"], gpu["q12"]], [orc_state["q11"], orc_state["q12"]]),
        "a": maxerr_group([gpu["ax"], gpu["ay"]], [orc_state["ax"], orc_state["ay"]]),
        "drho": maxerr_group([gpu["drho"]], [orc_state["rho"] / rho0 - 1.0]),
    }


def cluster_ic(nx, seed, radius, factor, u_scale=1e-3):
    """A jittered lattice with the particles of the disk |x - (1/2, 1/2)| < radius pulled towards
    its centre by `factor` (density 1/factor^2 there, an empty ring around it): a dense cluster
    whose particles have more neighbours than the lattice's 44."""
    ic = random_velocity_ic(nx, seed, u_scale=u_scale)
    dx, dy = ic["x"] - 0.5, ic["y"] - 0.5
    inside = np.hypot(dx, dy) < radius
    ic["x"] = np.where(inside, 0.5 + factor * dx, ic["x"])
    ic["y"] = np.where(inside, 0.5 + factor * dy, ic["y"])
    return ic


def periodic_copies(ic0, R, L=1.0):
    """R x R shrunk copies of ic0 tiling the box (`sph_inputs.periodic_copies`).  The method is
    local and the box periodic, so with the same h the big box evolves as R x R copies of the
    pattern on its own box of side L / R (c0 takes the largest speed, which the copies share)."""
    return si.periodic_copies(ic0, R, L)
