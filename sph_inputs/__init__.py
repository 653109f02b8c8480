"""Seeded synthetic particle inputs shared by the CUDA path's tests and the oracle's tests.

This module holds no arithmetic of the SPH method: it only draws particle positions and an
initial order-parameter field, and returns plain numpy arrays that either side consumes.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written from its published definition.  SplitMix64 is counter based:
the k-th output (k = 1, 2, ...) is the finaliser applied to ``seed + k * 0x9E3779B97F4A7C15``, so a
whole stream is produced with vectorised numpy integer arithmetic (wrapping modulo 2**64).

Workload recipe (the paper's set-up, §5: a fully periodic unit square, particles on a lattice,
zero initial velocity and a slightly perturbed nematic orientation):

* ``jittered_lattice``: an ``nx x ny`` square lattice in a box of side ``L``; site ``(ix, iy)`` has
  ID ``iy * nx + ix`` and sits at ``((ix + 0.5) dx, (iy + 0.5) dx)``.  Per particle, in ID order, five
  uniforms are drawn: ``jx, jy`` (jitter, uniform in ``[-j, j) * dx``), ``theta`` (director angle,
  uniform in ``[0, pi)``), and two more that Box-Muller turns into normals ``g11, g12`` of standard
  deviation ``sigma``.  The order parameter is ``Q11 = q cos(2 theta) + g11``,
  ``Q12 = q sin(2 theta) + g12`` (2D: Q = 2q(nn - I/2), §2).  Velocity is zero, density is rho0.
* ``uniform_random``: ``n`` positions uniform in the box (irregular cell occupancy, ragged sizes).
* ``hex_lattice``: a triangular lattice patch (used by operator pins that need isotropic moments).
* ``periodic_copies``: R x R copies of a 2D input shrunk to side L / R, tiling the box of side L
  (large boxes with the spacing and neighbourhoods of a small one).
* ``jittered_lattice3``: the 3D variant, an ``nx^3`` cubic lattice (ID ``ix + nx (iy + nx iz)``),
  eight uniforms per particle in ID order: jitter ``jx, jy, jz``, a director uniform on the sphere
  (``cos(polar)``, azimuth) for a uniaxial ``Q = s0 (d d - I/3)``, and optional velocities.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "splitmix64",
    "uniform53",
    "jittered_lattice",
    "jittered_lattice3",
    "uniform_random",
    "hex_lattice",
    "wrap_positions",
    "periodic_copies",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset+1 .. offset+count`` of the SplitMix64 stream started at ``seed`` (uint64)."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform53(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def wrap_positions(p: np.ndarray, L: float) -> np.ndarray:
    """Map coordinates into [0, L) (input generation only)."""
    p = np.where(p < 0.0, p + L, p)
    p = np.where(p >= L, p - L, p)
    return p


def perturbed_nematic(nx: int, *, L: float = 1.0, seed: int = 0, angle: float = 0.0,
                      spread: float = 0.1, q0: float = 1.0) -> dict:
    """The results section's initial condition read literally: an ordered nematic (order q0, one
    director angle ``angle``) slightly perturbed, at rest.  The jittered lattice of
    ``jittered_lattice(nx, seed=seed)`` with each particle's director angle ``angle`` plus a uniform
    perturbation in [-spread/2, spread/2) drawn from the generator stream ``seed + 7919``."""
    ic = jittered_lattice(nx, L=L, seed=seed)
    d = (uniform53(seed + 7919, ic["n"]) - 0.5) * spread
    ic["q11"] = q0 * np.cos(2.0 * (angle + d))
    ic["q12"] = q0 * np.sin(2.0 * (angle + d))
    return ic


def jittered_lattice(nx: int, ny: int | None = None, *, L: float = 1.0, seed: int = 0,
                     jitter: float = 0.05, q0: float = 1.0, sigma: float = 1e-3,
                     rho0: float = 1.0) -> dict:
    """Jittered square lattice with a random director per particle (see module docstring).

    Returns a dict of float64 arrays ``x, y, ux, uy, q11, q12, rho`` and int32 ``id``, plus the
    scalars ``dx`` and ``n``.  The lattice spacing is ``dx = L / nx``; ``ny`` defaults to ``nx``.
    """
    ny = nx if ny is None else ny
    n = nx * ny
    dx = L / nx
    u = uniform53(seed, 5 * n).reshape(n, 5)
    ids = np.arange(n, dtype=np.int64)
    ix = (ids % nx).astype(np.float64)
    iy = (ids // nx).astype(np.float64)
    jx = (u[:, 0] - 0.5) * (2.0 * jitter) * dx
    jy = (u[:, 1] - 0.5) * (2.0 * jitter) * dx
    theta = math.pi * u[:, 2]
    rad = np.sqrt(-2.0 * np.log(1.0 - u[:, 3]))
    g11 = sigma * rad * np.cos(2.0 * math.pi * u[:, 4])
    g12 = sigma * rad * np.sin(2.0 * math.pi * u[:, 4])
    x = wrap_positions((ix + 0.5) * dx + jx, L)
    y = wrap_positions((iy + 0.5) * dx + jy, L)
    return {
        "n": n,
        "dx": dx,
        "x": x,
        "y": y,
        "ux": np.zeros(n),
        "uy": np.zeros(n),
        "q11": q0 * np.cos(2.0 * theta) + g11,
        "q12": q0 * np.sin(2.0 * theta) + g12,
        "rho": np.full(n, rho0),
        "id": ids.astype(np.int32),
    }


def jittered_lattice3(nx: int, *, L: float = 1.0, seed: int = 0, jitter: float = 0.05, s0: float = 0.5,
                      u_scale: float = 0.0, rho0: float = 1.0) -> dict:
    """Jittered cubic lattice of nx^3 particles (spacing dx = L / nx, particle ID = ix + nx (iy + nx iz))
    with a uniaxial Q = s0 (d d - I/3) about a random direction d per particle (uniform on the
    sphere) and, if u_scale > 0, velocities uniform in [-u_scale/2, u_scale/2]^3.

    Returns float64 arrays ``x, y, z, rho`` (n), ``u`` (n, 3), ``q`` (n, 5) = (Q11, Q12, Q13, Q22, Q23),
    and the scalars ``dx`` and ``n``.
    """
    n = nx ** 3
    dx = L / nx
    u = uniform53(seed, 8 * n).reshape(n, 8) if n > 0 else np.zeros((0, 8))
    ids = np.arange(n, dtype=np.int64)
    ix = (ids % nx).astype(np.float64)
    iy = ((ids // nx) % nx).astype(np.float64)
    iz = (ids // (nx * nx)).astype(np.float64)
    pos = [wrap_positions((i + 0.5) * dx + (u[:, c] - 0.5) * (2.0 * jitter) * dx, L)
           for c, i in enumerate((ix, iy, iz))]
    cz = 2.0 * u[:, 3] - 1.0
    ph = 2.0 * math.pi * u[:, 4]
    sz = np.sqrt(np.maximum(1.0 - cz * cz, 0.0))
    d = np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)
    q = s0 * np.stack([d[:, 0] * d[:, 0] - 1.0 / 3.0, d[:, 0] * d[:, 1], d[:, 0] * d[:, 2],
                       d[:, 1] * d[:, 1] - 1.0 / 3.0, d[:, 1] * d[:, 2]], axis=1)
    vel = u_scale * (u[:, 5:8] - 0.5) if u_scale > 0 else np.zeros((n, 3))
    return {"n": n, "dx": dx, "x": pos[0], "y": pos[1], "z": pos[2], "u": vel, "q": q,
            "rho": np.full(n, rho0)}


def uniform_random(n: int, *, L: float = 1.0, seed: int = 0, q_scale: float = 1.0,
                   u_scale: float = 0.0, rho0: float = 1.0, rho_jitter: float = 0.0) -> dict:
    """``n`` particles uniform in the box, with uniform random fields of the given scales."""
    u = uniform53(seed, 7 * n).reshape(n, 7) if n > 0 else np.zeros((0, 7))
    x = wrap_positions(L * u[:, 0], L)
    y = wrap_positions(L * u[:, 1], L)
    return {
        "n": n,
        "x": x,
        "y": y,
        "ux": u_scale * (2.0 * u[:, 2] - 1.0),
        "uy": u_scale * (2.0 * u[:, 3] - 1.0),
        "q11": q_scale * (2.0 * u[:, 4] - 1.0),
        "q12": q_scale * (2.0 * u[:, 5] - 1.0),
        "rho": rho0 * (1.0 + rho_jitter * (2.0 * u[:, 6] - 1.0)),
        "id": np.arange(n, dtype=np.int32),
    }


def hex_lattice(spacing: float, *, L: float = 1.0, origin=(0.0, 0.0)) -> dict:
    """Triangular lattice sites ``origin + i*a1 + j*a2`` that fall inside ``[0, L)^2``.

    ``a1 = (spacing, 0)``, ``a2 = (spacing/2, spacing*sqrt(3)/2)``.  The patch is clipped at the box
    edges, so it is only regular away from them.
    """
    a2y = spacing * math.sqrt(3.0) / 2.0
    rows = int(math.ceil(L / a2y)) + 2
    cols = int(math.ceil(L / spacing)) + 2
    pts = []
    for j in range(-1, rows):
        y = origin[1] + j * a2y
        if y < 0.0 or y >= L:
            continue
        off = (j % 2) * 0.5 * spacing
        for i in range(-1, cols):
            x = origin[0] + off + i * spacing
            if 0.0 <= x < L:
                pts.append((x, y))
    p = np.array(pts, dtype=np.float64)
    n = p.shape[0]
    return {"n": n, "x": p[:, 0].copy(), "y": p[:, 1].copy(), "id": np.arange(n, dtype=np.int32)}


def periodic_copies(ic0: dict, R: int, L: float = 1.0) -> tuple[dict, dict]:
    """R x R copies of the 2D input ``ic0`` (positions in ``[0, L)``) shrunk to a box of side
    ``L / R``, tiling the box of side ``L``: copy ``t = ty R + tx`` holds particle ``t n0 + i`` at the
    shrunk position of particle ``i`` shifted by ``(tx, ty) L / R``; the other per-particle arrays
    (``ux, uy, q11, q12, rho`` where present) are repeated.  Returns ``(big, pattern)``: the big
    box's input and the pattern on its own box of side ``L / R``.  A power-of-two ``R`` keeps the
    shrunk positions exact."""
    n0 = len(ic0["x"])
    L0 = L / R
    x0 = np.asarray(ic0["x"], dtype=np.float64) / R
    y0 = np.asarray(ic0["y"], dtype=np.float64) / R
    t = np.arange(R * R)
    sx = ((t % R) * L0)[:, None]
    sy = ((t // R) * L0)[:, None]
    big = {"n": R * R * n0,
           "x": wrap_positions((x0[None, :] + sx).ravel(), L),
           "y": wrap_positions((y0[None, :] + sy).ravel(), L)}
    pattern = {"n": n0, "x": x0, "y": y0}
    for k in ("ux", "uy", "q11", "q12", "rho"):
        if k in ic0:
            big[k] = np.tile(np.asarray(ic0[k], dtype=np.float64), R * R)
            pattern[k] = np.asarray(ic0[k], dtype=np.float64)
    return big, pattern
