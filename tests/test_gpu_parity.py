"""GPU parity against the FP64 oracle, through the C-ABI.

* Neighbour lists: bit-exact (same sets) on lattices, random sets, ragged tilings, three-cell
  boxes and particles hugging the periodic faces.
* One step's intermediates (V, B, grad u, lap Q, k, rho_half, rho_hat, p, div Q, a, APD).
* State fields per step over 10 steps on the 64 x 64 set-up and on 256 x 256 at three
  activities: normwise relative error <= 1e-5 (FP32 arithmetic against FP64).
* Moving states (random and smooth velocities, c0 > 0, so pressure, viscous and APD terms all act)
  at the full tilings: 10 steps at 256 x 256 and at 1024 x 1024, every state field within
  1e-5 both normwise and element-wise (the largest per-particle error over the field's largest
  per-particle value); the momentum variants (conservative form, elastic stress, Q^n, no APD)
  from a moving state at 256 x 256, five steps.
"""
import numpy as np
import pytest

import sph_inputs as si
from _sph import (GpuRun, cluster_ic, compare_state, compare_state_max, oracle_params, oracle_state, params,
                  random_velocity_ic, relerr, relerr_group, smooth_ic, stable_dt)

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding


def _nbr_case(name):
    if name == "lattice64":
        ic = si.jittered_lattice(64, seed=0)
        return ic, 1.3 / 64
    if name == "ragged45":         # 11 cells across: the last tile column / row is partial
        ic = si.jittered_lattice(45, seed=2, jitter=0.3)
        return ic, 1.3 / 45
    if name == "random3000":       # Poisson counts: mean pi 3.3^2 = 34 neighbours, far below 64
        ic = si.uniform_random(3000, seed=4)
        return ic, 1.1 / np.sqrt(3000)
    if name == "three_cells":
        ic = si.uniform_random(160, seed=6)
        return ic, 1.0 / 9.5 * 0.999
    if name == "faces":
        # 100 particles in each 2e-3 strip along the four faces, 600 uniform
        u = si.uniform53(11, 2000).reshape(1000, 2)
        e = 2e-3 * u[:, 0]
        x = np.concatenate([e[:100], 1.0 - e[100:200], u[200:, 0]])
        y = np.concatenate([u[:200, 1], e[200:300], 1.0 - e[300:400], u[400:, 1]])
        ic = {"x": si.wrap_positions(x, 1.0), "y": si.wrap_positions(y, 1.0)}
        ic.update({k: np.zeros(1000) for k in ("ux", "uy", "q11", "q12")})
        return ic, 0.018
    if name == "lattice256":
        ic = si.jittered_lattice(256, seed=1)
        return ic, 1.3 / 256
    if name == "cluster":          # a dense disk: up to 112 candidates, 82 particles above 64
        return cluster_ic(64, 3, 0.1, 0.65), 1.3 / 64
    raise KeyError(name)


@pytest.mark.parametrize("case", ["lattice64", "ragged45", "random3000", "three_cells", "faces",
                                  "lattice256", "cluster"])
def test_neighbor_lists_bit_exact(B, orc, case):
    ic, h = _nbr_case(case)
    n = len(ic["x"])
    p = params(64, h=h)
    run = GpuRun(B, p, ic)
    try:
        rp_g, cols_g = B.ann_get_neighbors(run.ctx, n)
    finally:
        run.close()
    mode = "cells" if n > 20000 else "brute"
    rp_o, cols_o = orc.neighbors(ic["x"], ic["y"], 1.0, h, mode)
    assert np.array_equal(rp_g, rp_o)
    assert np.array_equal(cols_g, cols_o)


def _oracle_one_step(orc, p, ic, nbr_mode="brute"):
    st, rec = orc.step(oracle_params(orc, p, nbr_mode), oracle_state(ic), 1, record=True)
    return st, rec


@pytest.mark.parametrize("kind", ["random_u", "smooth"])
def test_one_step_intermediates(B, orc, kind):
    nx = 64
    ic = random_velocity_ic(nx, 3, rho_scale=2e-4) if kind == "random_u" else smooth_ic(nx, 5)
    p = params(nx, c0_min=0.05)
    run = GpuRun(B, p, ic)
    try:
        B.ann_set_record(run.ctx, True)
        run.step(1)
        g = {k: run.field(k) for k in ("SUMW", "V", "B11", "B12", "B22", "K", "DRHO_HALF",
                                       "DRHO_HAT", "P", "DIVQX", "DIVQY", "AX", "AY", "LAPQ11",
                                       "LAPQ12", "GRADU_XX", "GRADU_XY", "GRADU_YX", "GRADU_YY",
                                       "APDX", "APDY", "QRATE11", "QRATE12", "NNBR")}
    finally:
        run.close()
    _, r = _oracle_one_step(orc, p, ic)
    assert np.array_equal(g["NNBR"], r["nnbr"])
    r11, r12, r22 = r["B11"], r["B12"], r["B22"]
    errs = {
        "SUMW": relerr(g["SUMW"], r["sumW"]), "V": relerr(g["V"], r["V"]),
        "B": relerr_group([g["B11"], g["B12"], g["B12"], g["B22"]], [r11, r12, r12, r22]),
        "K": relerr(g["K"], r["k"]),
        "DRHO_HALF": relerr(g["DRHO_HALF"], r["rho_half"] - 1.0),
        "DRHO_HAT": relerr(g["DRHO_HAT"], r["rho_hat"] - 1.0),
        "P": relerr(g["P"], r["p"]),
        "divQ": relerr_group([g["DIVQX"], g["DIVQY"]], [r["divQx"], r["divQy"]]),
        "a": relerr_group([g["AX"], g["AY"]], [r["ax"], r["ay"]]),
        "lapQ": relerr_group([g["LAPQ11"], g["LAPQ12"]], [r["lapQ11"], r["lapQ12"]]),
        "gradu": relerr_group([g["GRADU_XX"], g["GRADU_XY"], g["GRADU_YX"], g["GRADU_YY"]],
                              [r["gradu"][:, 0], r["gradu"][:, 1], r["gradu"][:, 2], r["gradu"][:, 3]]),
        "apd": relerr_group([g["APDX"], g["APDY"]], [r["apdx"], r["apdy"]]),
        "qrate": relerr_group([g["QRATE11"], g["QRATE12"]], [r["qrate11"], r["qrate12"]]),
    }
    bad = {k: e for k, e in errs.items() if not e <= TOL}
    assert not bad, errs


def _ten_steps(B, orc, nx, p, ic, nbr_mode, nsteps=10):
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, nbr_mode)
    worst = {}
    try:
        for s in range(nsteps):
            run.step(1)
            st, _ = orc.step(P, st, 1)
            errs = compare_state(run.state(), st, ic["x"], ic["y"])
            for k, e in errs.items():
                worst[k] = max(worst.get(k, 0.0), e)
    finally:
        run.close()
    return worst


def test_ten_steps_64(B, orc):
    """The 64 x 64 set-up: random director, S = 1, 1e-3 noise, u = 0, dt = 1e-4, zeta = 0.05."""
    ic = si.jittered_lattice(64, seed=0)
    worst = _ten_steps(B, orc, 64, params(64), ic, "brute")
    print("64 ten steps", {k: f"{v:.2e}" for k, v in worst.items()})
    bad = {k: e for k, e in worst.items() if not e <= TOL}
    assert not bad, worst


@pytest.mark.parametrize("zeta", [0.02, 0.05, 0.1])
def test_ten_steps_256(B, orc, zeta):
    """256 x 256 at three activities.  dt = 1e-4 is 30x beyond the explicit viscous limit
    0.125 h^2/nu at this resolution (the run diverges within a few steps on both sides), so the
    stable dt is used."""
    ic = si.jittered_lattice(256, seed=1)
    p = params(256, zeta=zeta)
    p["dt"] = stable_dt(p)
    worst = _ten_steps(B, orc, 256, p, ic, "cells")
    print(f"256 zeta {zeta} ten steps", {k: f"{v:.2e}" for k, v in worst.items()})
    bad = {k: e for k, e in worst.items() if not e <= TOL}
    assert not bad, worst


@pytest.mark.parametrize("variant", ["conservative", "q_old", "c_half", "no_apd", "beta_half",
                                     "landau_A", "elastic", "elastic_conservative", "contractile"])
def test_variants_five_steps(B, orc, variant):
    kw = {"conservative": dict(conservative=1, c0_min=0.05), "q_old": dict(q_new_in_momentum=0),
          "c_half": dict(c_shift=0.5), "no_apd": dict(apd=0), "beta_half": dict(beta=0.5),
          "landau_A": dict(A=0.3, C=0.5),
          # Eq. (12) elastic stress, with a B term so that its isotropic part of H enters too
          "elastic": dict(elastic=1, A=0.3, B=0.2, C=0.5),
          "elastic_conservative": dict(elastic=1, conservative=1, c0_min=0.05, A=0.3, B=0.2, C=0.5),
          # contractile activity (zeta < 0) with a larger elastic constant: the sweeps' other half
          "contractile": dict(zeta=-0.1, K=0.08)}[variant]
    ic = random_velocity_ic(48, 9, rho_scale=1e-4)
    worst = _ten_steps(B, orc, 48, params(48, **kw), ic, "brute", nsteps=5)
    bad = {k: e for k, e in worst.items() if not e <= TOL}
    assert not bad, worst


def _moving_ic(kind, nx):
    if kind == "random_u":
        return random_velocity_ic(nx, 13, u_scale=2e-2, rho_scale=2e-4)
    return smooth_ic(nx, 17, u_amp=2e-2)


def _round32(st):
    """The oracle's state with every field the library keeps in FP32 rounded to FP32 (positions stay
    FP64, as on the GPU)."""
    return {k: (v if k in ("x", "y") else np.asarray(v, np.float32).astype(np.float64)) for k, v in st.items()}


def _parity_steps(B, orc, p, ic, nsteps, nbr_mode="cells"):
    """Worst normwise and element-wise errors of every state field over nsteps single steps, and,
    for the acceleration, the worst ratio of the GPU's error to the floor that the FP32 storage of
    the state sets: the change of the oracle's own FP64 step when its input state is rounded to
    FP32 (exact arithmetic on FP32 inputs)."""
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, nbr_mode)
    norm, elem, floor = {}, {}, {"a": 0.0, "a_ratio": 0.0}
    try:
        for _ in range(nsteps):
            run.step(1)
            st32, _ = orc.step(P, _round32(st), 1)
            st, _ = orc.step(P, st, 1)
            g = run.state()
            for k, e in compare_state(g, st, ic["x"], ic["y"]).items():
                norm[k] = max(norm.get(k, 0.0), e)
            for k, e in compare_state_max(g, st, ic["x"], ic["y"]).items():
                elem[k] = max(elem.get(k, 0.0), e)
            fa = relerr_group([st32["ax"], st32["ay"]], [st["ax"], st["ay"]])
            ea = relerr_group([g["ax"], g["ay"]], [st["ax"], st["ay"]])
            floor["a"] = max(floor["a"], fa)
            floor["a_ratio"] = max(floor["a_ratio"], ea / max(fa, 1e-300))
    finally:
        run.close()
    return norm, elem, floor


# The acceleration is the one field built from pair terms much larger than itself: on smooth flows
# the viscous second difference of u sums terms ~1/(k h) times its value, and the FP32 rounding of
# the stored velocity (2^-24 |u|) already moves it by the `floor` above (~4e-5 at 256^2, ~4e-4 at
# 1024^2 for the smooth field).  A pair term has about four independent FP32 roundings of that
# size (the two stored velocities, the pair vector, the product u_ij . d), so to first order the
# FP32 path's error is about sqrt(4) = 2 times the storage floor; the bound is 1e-5 or, where the
# floor exceeds it, 3 times the floor (room for the spread of the worst step).  Every state field
# (positions, u, Q, rho) is held to 1e-5 normwise and element-wise.
FLOOR_FACTOR = 3.0


def _check_moving(norm, elem, floor):
    bad = {}
    for k, e in list(norm.items()) + [("max_" + k, v) for k, v in elem.items()]:
        if k in ("a", "max_a"):
            continue
        if not e <= TOL:
            bad[k] = e
    lim_a = max(TOL, FLOOR_FACTOR * floor["a"])
    if not norm["a"] <= lim_a:
        bad["a"] = (norm["a"], lim_a)
    return bad


@pytest.mark.parametrize("kind", ["random_u", "smooth"])
def test_ten_steps_256_moving(B, orc, kind):
    """256 x 256 from moving states with c0 = max(10 max|u|, 0.2): the pressure, viscous and APD
    paths act from the first step, over the full tiling (65 x 65 tiles of 4 x 4 cells)."""
    ic = _moving_ic(kind, 256)
    p = params(256, c0_min=0.2)
    p["dt"] = stable_dt(p)
    norm, elem, floor = _parity_steps(B, orc, p, ic, 10)
    print(f"256 {kind} normwise", {k: f"{v:.2e}" for k, v in norm.items()},
          "element-wise", {k: f"{v:.2e}" for k, v in elem.items()}, "a floor", floor)
    bad = _check_moving(norm, elem, floor)
    assert not bad, (bad, norm, elem, floor)


@pytest.mark.parametrize("kind", ["random_u", "smooth"])
def test_ten_steps_1024_moving(B, orc, kind):
    """The benchmark's size, 1024 x 1024 (1,048,576 particles, 4225 tiles), from moving states:
    ten steps, every particle compared at every step (the oracle's cell search, OpenMP)."""
    ic = _moving_ic(kind, 1024)
    p = params(1024, zeta=0.08, K=0.02, c0_min=0.2)
    p["dt"] = stable_dt(p)
    norm, elem, floor = _parity_steps(B, orc, p, ic, 10)
    print(f"1024 {kind} normwise", {k: f"{v:.2e}" for k, v in norm.items()},
          "element-wise", {k: f"{v:.2e}" for k, v in elem.items()}, "a floor", floor)
    bad = _check_moving(norm, elem, floor)
    assert not bad, (bad, norm, elem, floor)


@pytest.mark.parametrize("variant", ["conservative", "q_old", "elastic", "elastic_conservative", "no_apd"])
def test_variants_256_moving(B, orc, variant):
    """The momentum variants over the full 256 x 256 tiling from a moving state (random velocities
    2e-2, density noise, c0 >= 0.2): five steps, every particle, with the bounds of the moving-state
    cases (state fields 1e-5 normwise and element-wise, the acceleration 1e-5 or 3 x its FP32
    storage floor)."""
    kw = {"conservative": dict(conservative=1), "q_old": dict(q_new_in_momentum=0), "no_apd": dict(apd=0),
          "elastic": dict(elastic=1, A=0.3, B=0.2, C=0.5),
          "elastic_conservative": dict(elastic=1, conservative=1, A=0.3, B=0.2, C=0.5)}[variant]
    ic = _moving_ic("random_u", 256)
    p = params(256, c0_min=0.2, **kw)
    p["dt"] = stable_dt(p)
    norm, elem, floor = _parity_steps(B, orc, p, ic, 5)
    print(f"256 {variant} normwise", {k: f"{v:.2e}" for k, v in norm.items()},
          "element-wise", {k: f"{v:.2e}" for k, v in elem.items()}, "a floor", floor)
    bad = _check_moving(norm, elem, floor)
    assert not bad, (bad, norm, elem, floor)
