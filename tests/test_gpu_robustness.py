"""GPU behaviour at full size and at the edges, through the C-ABI.

* The 1024 x 1024 (~1.05 M particle) high-resolution set-up, in the launch configuration the
  benchmark times: two steps against the oracle on every particle (the oracle's cell-grid search,
  itself pinned bit-exact to brute force).
* Error statuses raised on the host or by the kernels' own bounds checks: wrong n, NaN input,
  an overfull cell, stepping before loading; none of them faults the device.
* Checkpoint and resume continue bit-identically; two contexts on the same input agree bitwise.
* Conservative momentum mode keeps total momentum to FP32 round-off on the GPU.
"""
import os

import numpy as np
import pytest

import sph_inputs as si
from _sph import (GpuRun, cluster_ic, compare_state, gpu_params, oracle_params, oracle_state, params,
                  random_velocity_ic, stable_dt)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding


def test_full_size_two_steps(B, orc):
    p = params(1024, zeta=0.08, K=0.02)
    gp = gpu_params(B, p, 1024 * 1024)
    gp.dt_mode = 1
    p["dt"] = B.ann_grid_info(gp).dt_effective
    ic = si.jittered_lattice(1024, seed=0)
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, "cells")
    try:
        for _ in range(2):
            run.step(1)
            st, rec = orc.step(P, st, 1, record=True)
            errs = compare_state(run.state(), st, ic["x"], ic["y"])
            bad = {k: e for k, e in errs.items() if not e <= 1e-5}
            assert not bad, errs
        assert np.array_equal(run.field("NNBR"), rec["nnbr"])
        d = B.ann_get_diagnostics(run.ctx)
        assert d["error_bits"] == 0 and d["nbr_min"] == 44 and d["nbr_max"] == 44
    finally:
        run.close()


def test_wrong_n_and_null_inputs(B):
    ic = si.jittered_lattice(32, seed=0)
    ctx = B.ann_create(gpu_params(B, params(32), 32 * 32))
    try:
        with pytest.raises(B.AnnError) as e:
            B.ann_set_particles(ctx, ic["x"][:-1], ic["y"][:-1], ic["ux"][:-1], ic["uy"][:-1],
                                ic["q11"][:-1], ic["q12"][:-1])
        assert e.value.status == -1
        with pytest.raises(B.AnnError) as e:
            B.ann_step(ctx, 1)
        assert e.value.status == -9            # no particles yet
        with pytest.raises(B.AnnError) as e:
            B.ann_get_field(ctx, "UX", 1024)
        assert e.value.status == -9
    finally:
        B.ann_destroy(ctx)


def test_nonfinite_input_is_rejected(B):
    ic = si.jittered_lattice(32, seed=0)
    ctx = B.ann_create(gpu_params(B, params(32), 32 * 32))
    try:
        q = ic["q11"].copy()
        q[100] = np.nan
        with pytest.raises(B.AnnError) as e:
            B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], q, ic["q12"])
        assert e.value.status == -6
        # a clean load afterwards works and steps
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        B.ann_step(ctx, 2)
    finally:
        B.ann_destroy(ctx)


def test_overfull_cell_is_reported_not_faulted(B):
    # 100 extra particles piled into one cell: the cell-capacity check raises CELL_OVERFLOW
    ic = si.jittered_lattice(32, seed=0)
    x, y = ic["x"].copy(), ic["y"].copy()
    x[:100] = 0.5 + 1e-4 * np.arange(100) / 100
    y[:100] = 0.5
    ctx = B.ann_create(gpu_params(B, params(32), 32 * 32))
    try:
        B.ann_set_particles(ctx, x, y, ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        with pytest.raises(B.AnnError) as e:
            B.ann_step(ctx, 1)
        assert e.value.status == -4
        assert B.ann_get_diagnostics(ctx)["error_bits"] & 1
        # the context stays usable: a fresh load clears the sticky bits
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        B.ann_step(ctx, 1)
    finally:
        B.ann_destroy(ctx)


def test_neighbour_bits_follow_pairs_crossing_the_cutoff(B, orc):
    """Between re-sorts pass A rewrites each list entry's neighbour bit in place.  Uniform random
    positions in a shear flow u = (2 sin 2 pi y, 0) (no displacement term, so nothing else moves the
    particles): pairs cross 3h every step while no particle leaves half the skin, so the
    neighbour counts change from step to step on the lists of the first step.  At every step they
    equal the oracle's (FP64 definition, brute force) for one step from the same state."""
    import math

    nx = 64
    p = params(nx, c0_min=0.05, apd=0)
    p["dt"] = stable_dt(p)
    ic = si.uniform_random(nx * nx, seed=29)
    ic["ux"] = 2.0 * np.sin(2.0 * math.pi * ic["y"])
    ic["uy"] = np.zeros(ic["n"])
    run = GpuRun(B, p, ic)
    P = oracle_params(orc, p, "brute")
    prev, changed = None, 0
    try:
        run.step(1)
        for _ in range(4):
            g = run.state()
            st = {"x": g["x"], "y": g["y"], "ux": g["ux"], "uy": g["uy"], "q11": g["q11"], "q12": g["q12"],
                  "rho": 1.0 + g["drho"], "ax": g["ax"], "ay": g["ay"]}
            _, rec = orc.step(P, st, 1, record=True)
            run.step(1)
            nn = run.field("NNBR")
            assert np.array_equal(nn, rec["nnbr"])
            if prev is not None:
                changed += int((nn != prev).sum())
            prev = nn
        d = B.ann_get_diagnostics(run.ctx)
    finally:
        run.close()
    assert d["resorts"] == 1, d   # steps 2 to 5 filtered the lists of the first
    assert changed > 50, changed


def test_dense_cluster_beyond_64_candidates_matches_the_oracle(B, orc):
    """A dense cluster (particles with up to 112 candidates, 82 of them above 64): the lists, masks
    and sums reach past the first 64 candidates in every pass -- the re-sort step and two steps
    that filter the same lists -- and the state stays within the parity bound of the oracle."""
    ic = cluster_ic(64, 3, 0.1, 0.65, u_scale=1e-3)
    p = params(64, c0_min=0.05)
    p["dt"] = stable_dt(p)
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, "brute")
    try:
        for _ in range(3):
            run.step(1)
            st, _ = orc.step(P, st, 1)
            errs = compare_state(run.state(), st, ic["x"], ic["y"])
            assert all(e <= 1e-5 for e in errs.values()), errs
        d = B.ann_get_diagnostics(run.ctx)
        assert d["nbr_max"] > 64 and d["resorts"] == 1 and d["error_bits"] == 0, d
    finally:
        run.close()


def test_cluster_beyond_the_list_capacity_is_reported(B):
    """A cluster whose particles have up to ~165 candidates, beyond the 128 a list holds: the step
    reports NBR_OVERFLOW (no fault, no silent truncation) and the context stays usable."""
    ic = cluster_ic(64, 3, 0.12, 0.55)
    ctx = B.ann_create(gpu_params(B, params(64), 64 * 64))
    try:
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        with pytest.raises(B.AnnError) as e:
            B.ann_step(ctx, 1)
        assert e.value.status == -5
        assert B.ann_get_diagnostics(ctx)["error_bits"] & 4
        lat = si.jittered_lattice(64, seed=3)
        B.ann_set_particles(ctx, lat["x"], lat["y"], lat["ux"], lat["uy"], lat["q11"], lat["q12"])
        B.ann_step(ctx, 1)
    finally:
        B.ann_destroy(ctx)


def test_checkpoint_resume_is_bit_identical(B, tmp_path):
    ic = random_velocity_ic(64, 4)
    p = params(64, c0_min=0.05)
    a = GpuRun(B, p, ic)
    b = GpuRun(B, p, ic)
    try:
        a.step(20)
        b.step(10)
        path = str(tmp_path / "state.bin")
        B.ann_save_state(b.ctx, path)
        b.close()
        c = GpuRun(B, p, si.jittered_lattice(64, seed=99))
        B.ann_load_state(c.ctx, path)
        assert B.ann_get_diagnostics(c.ctx)["step"] == 10
        c.step(10)
        sa, sc = a.state(), c.state()
        for k in sa:
            assert np.array_equal(sa[k], sc[k]), k
        c.close()
    finally:
        a.close()


def test_two_contexts_agree_bitwise(B):
    ic = random_velocity_ic(96, 5)
    p = params(96, c0_min=0.05)
    p["dt"] = stable_dt(p)
    runs = [GpuRun(B, p, ic) for _ in range(2)]
    try:
        for r in runs:
            r.step(15)
        s0, s1 = runs[0].state(), runs[1].state()
        for k in s0:
            assert np.array_equal(s0[k], s1[k]), k
    finally:
        for r in runs:
            r.close()


def test_conservative_momentum_on_gpu(B):
    ic = random_velocity_ic(64, 8)
    p = params(64, conservative=1, c0_min=0.5, eta=0.05, dt=5e-5)
    run = GpuRun(B, p, ic)
    try:
        m = 1.0 / run.n
        p0 = m * np.array([ic["ux"].sum(), ic["uy"].sum()])
        run.step(100)
        s = run.state()
        p1 = m * np.array([s["ux"].sum(), s["uy"].sum()])
        scale = m * (np.abs(s["ux"]).sum() + np.abs(s["uy"]).sum())
        assert np.abs(s["ux"] - ic["ux"]).max() > 1e-6
        assert np.abs(p1 - p0).max() <= 1e-5 * scale
    finally:
        run.close()


def test_device_inputs_and_outputs(B):
    import torch

    ic = si.jittered_lattice(48, seed=3)
    n = ic["n"]
    p = params(48)
    dev = {k: torch.tensor(ic[k], dtype=torch.float64, device="cuda") for k in
           ("x", "y", "ux", "uy", "q11", "q12", "rho")}
    ctx = B.ann_create(gpu_params(B, p, n))
    try:
        B.ann_set_stream(ctx, torch.cuda.current_stream())
        B.ann_set_particles(ctx, dev["x"], dev["y"], dev["ux"], dev["uy"], dev["q11"], dev["q12"],
                            dev["rho"])
        B.ann_step(ctx, 3)
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        B.ann_get_field(ctx, "Q11", n, out=out)
        host = B.ann_get_field(ctx, "Q11", n)
        assert np.array_equal(out.cpu().numpy(), host)
    finally:
        B.ann_destroy(ctx)


def _moving_case(nx=64):
    """Velocities of order 1: particles move ~1e-4 per step, so the candidate lists are rebuilt
    (particles re-sorted) every few steps.  eta = 0.1 keeps dt = 1e-4 inside the viscous limit."""
    ic = random_velocity_ic(nx, 12, u_scale=2.0, rho_scale=1e-4)
    return ic, params(nx, eta=0.1, c0_min=0.5)


def test_parity_across_resorts(B, orc):
    ic, p = _moving_case()
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, "brute")
    worst = {}
    try:
        for _ in range(30):
            run.step(1)
            st, _ = orc.step(P, st, 1)
            for k, e in compare_state(run.state(), st, ic["x"], ic["y"]).items():
                worst[k] = max(worst.get(k, 0.0), e)
        d = B.ann_get_diagnostics(run.ctx)
        rp, cols = B.ann_get_neighbors(run.ctx, run.n)
    finally:
        run.close()
    assert d["resorts"] >= 4, d
    bad = {k: e for k, e in worst.items() if not e <= 1e-5}
    assert not bad, worst
    rp_o, cols_o = orc.neighbors(st["x"], st["y"], 1.0, p["h"], "brute")
    # positions differ at the 1e-12 level between the two sides: compare lists away from ties
    assert abs(int(rp[-1]) - int(rp_o[-1])) <= 2


def test_profiled_steps_match_graph_steps(B):
    """ann_step_profile launches the same kernels one by one: same state bit for bit, and each
    kernel is billed only in the steps where its branch ran."""
    ic, p = _moving_case()
    a = GpuRun(B, p, ic)
    b = GpuRun(B, p, ic)
    try:
        a.step(30)
        prof = B.ann_step_profile(b.ctx, 30)
        ra = B.ann_get_diagnostics(a.ctx)["resorts"]
        rb = B.ann_get_diagnostics(b.ctx)["resorts"]
        sa, sb = a.state(), b.state()
    finally:
        a.close()
        b.close()
    assert ra == rb and 4 <= ra < 30, (ra, rb)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    names = [B.ann_kernel_name(k) for k in range(B.ann_kernel_count())]
    assert set(prof) == set(names)
    assert all(v > 0.0 for v in prof.values()), prof
    # one step of re-sort: the resort branch's kernels must not be billed for the other steps
    c = GpuRun(B, p, ic)
    try:
        prof1 = B.ann_step_profile(c.ctx, 1)   # the first step after ann_set_particles re-sorts
        assert B.ann_get_diagnostics(c.ctx)["resorts"] == 1
    finally:
        c.close()
    assert prof1["pass_a"] == 0.0 and prof1["pass_a_resort"] > 0.0, prof1


def test_checkpoint_across_resorts(B, tmp_path):
    ic, p = _moving_case()
    a = GpuRun(B, p, ic)
    b = GpuRun(B, p, ic)
    try:
        a.step(30)
        b.step(13)
        path = str(tmp_path / "state.bin")
        B.ann_save_state(b.ctx, path)
        b.close()
        c = GpuRun(B, p, si.jittered_lattice(64, seed=5))
        B.ann_load_state(c.ctx, path)
        c.step(17)
        assert B.ann_get_diagnostics(a.ctx)["resorts"] >= 4
        sa, sc = a.state(), c.state()
        for k in sa:
            assert np.array_equal(sa[k], sc[k]), k
        c.close()
    finally:
        a.close()


def test_late_resort_within_the_step(B, orc):
    """A uniform translation fast enough that particles cross half the candidate skin within one
    half step: the step notices it at the evaluation point and re-sorts before the pair passes,
    so results still match the oracle (which searches from scratch every step)."""
    nx = 32
    ic = si.jittered_lattice(nx, seed=0)
    n = ic["n"]
    ic["q11"] = np.full(n, 0.6)
    ic["q12"] = np.full(n, 0.2)
    ic["ux"] = np.full(n, 15.0)
    ic["uy"] = np.full(n, -4.0)
    p = params(nx, eta=0.01, zeta=0.0, K=0.0)
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, "brute")
    try:
        for _ in range(4):
            run.step(1)
            st, _ = orc.step(P, st, 1)
            errs = compare_state(run.state(), st, ic["x"], ic["y"])
            assert errs["disp"] <= 1e-5 and errs["u"] <= 1e-5, errs
        d = B.ann_get_diagnostics(run.ctx)
    finally:
        run.close()
    # a full step moves dt |u| = 1.55e-3, more than half the skin 0.5 * 0.02 * 3h = 1.2e-3, so
    # every step finds the lists of the previous one stale and re-sorts
    assert d["resorts"] >= 2, d


def test_pairs_at_the_cutoff_take_the_fp64_band_test(B, orc):
    """h = 4/3 dx on an unjittered lattice puts every particle's four lattice neighbours at
    distance 4 dx = 3h exactly: each pair falls in the FP32 rounding band and is decided by the
    FP64 definition, first in the re-sort pass, then (nothing moves) in the candidate filter of
    the following steps.  Neighbour counts equal the oracle's bit for bit."""
    nx = 64
    ic = si.jittered_lattice(nx, seed=0, jitter=0.0)
    p = params(nx, h=4.0 / (3.0 * nx), zeta=0.0)
    run = GpuRun(B, p, ic)
    st = oracle_state(ic)
    P = oracle_params(orc, p, "brute")
    try:
        for _ in range(3):
            run.step(1)
            st, rec = orc.step(P, st, 1, record=True)
            assert np.array_equal(run.field("NNBR"), rec["nnbr"])
        d = B.ann_get_diagnostics(run.ctx)
    finally:
        run.close()
    assert d["band_checks"] >= 3 * 4 * nx * nx, d
    assert d["resorts"] == 1, d   # steps 2 and 3 ran the candidate filter


def test_dt_check_mode_reports_cfl_violations(B):
    """dt_mode ANN_DT_CHECK: a step whose dt exceeds the viscous limit 0.125 h^2 / nu, or
    0.25 h / (c0 + max|u|) with c0 = 10 max|u| of its midpoint, fails with CFL_VIOLATION (the bit
    stays set); below both limits it runs."""
    nx = 64
    ic = random_velocity_ic(nx, 21, u_scale=1.0)
    h = 1.3 / nx

    def run(**kw):
        gp = gpu_params(B, params(nx, **kw), ic["n"])
        gp.dt_mode = 2
        ctx = B.ann_create(gp)
        try:
            B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
            try:
                B.ann_step(ctx, 3)
                status = 0
            except B.AnnError as e:
                status = e.status
            return status, B.ann_get_diagnostics(ctx)["error_bits"]
        finally:
            B.ann_destroy(ctx)

    assert 0.125 * h * h < 1e-4          # eta = 1: the viscous limit is below dt = 1e-4
    assert run(dt=1e-4) == (-13, 32)
    umax = float(np.hypot(ic["ux"], ic["uy"]).max())
    lim = 0.25 * h / (11.0 * umax)      # the first midpoint velocity is u itself (a^0 = 0)
    assert lim < 0.125 * h * h / (0.34 * 0.04) and lim < 0.125 * h * h / 1e-3
    assert run(dt=2.0 * lim, eta=1e-3) == (-13, 32)
    assert run(dt=0.4 * lim, eta=1e-3) == (0, 0)


def test_context_on_the_torch_caching_allocator(B):
    """Every device buffer of a context made by ann_create_with_allocator comes from the given
    allocator (here PyTorch's caching allocator) and goes back to it on destroy (the neighbour
    export's transient buffer at the end of its call); the steps and the flow diagnostics are
    bit-identical to a context on cudaMalloc."""
    import torch

    ic = random_velocity_ic(96, 5)
    p = params(96, c0_min=0.05)
    p["dt"] = stable_dt(p)
    gp = gpu_params(B, p, ic["n"])
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    ctx = B.ann_create_with_allocator(gp, B.torch_allocator())
    ref = GpuRun(B, p, ic)
    try:
        held = torch.cuda.memory_allocated() - base
        assert held >= 0.8 * B.ann_grid_info(gp).device_bytes
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
        B.ann_step(ctx, 15)
        ref.step(15)
        for f in ("X", "Y", "UX", "UY", "Q11", "Q12", "DRHO"):
            assert np.array_equal(B.ann_get_field(ctx, f, ref.n), B.ann_get_field(ref.ctx, f, ref.n)), f
        assert np.array_equal(B.ann_energy_spectrum(ctx, 64), B.ann_energy_spectrum(ref.ctx, 64))
        assert torch.cuda.memory_allocated() - base > held   # the spectrum's scratch
        # the neighbour export's buffer (4 ANN_MAX_NEIGHBORS bytes per particle) comes from the
        # allocator for the call only
        before = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        rp, cols = B.ann_get_neighbors(ctx, ref.n)
        assert torch.cuda.max_memory_allocated() - before >= 4 * 128 * ref.n
        assert torch.cuda.memory_allocated() == before
        assert rp[-1] == cols.size and np.all(np.diff(rp) >= 0)
    finally:
        B.ann_destroy(ctx)
        ref.close()
    assert torch.cuda.memory_allocated() == base


def test_get_state_equals_the_field_reads(B):
    """ann_get_state returns, in one call, exactly what ann_get_field returns field by field, to
    host arrays and to device tensors, and skips the fields it is not given."""
    import torch

    ic = random_velocity_ic(64, 9)
    p = params(64, c0_min=0.05)
    p["dt"] = stable_dt(p)
    run = GpuRun(B, p, ic)
    try:
        run.step(7)
        ref = {f: B.ann_get_field(run.ctx, f, run.n) for f in B.FULL_STATE}
        host = B.ann_get_state(run.ctx, run.n)
        dev = {f: torch.zeros(run.n, dtype=torch.float64 if f in ("X", "Y") else torch.float32, device="cuda")
               for f in B.FULL_STATE if f not in ("UY", "Q12")}
        B.ann_get_state(run.ctx, run.n, out=dev)
        for f in B.FULL_STATE:
            assert np.array_equal(host[f], ref[f]), f
            if f in dev:
                assert np.array_equal(dev[f].cpu().numpy(), ref[f]), f
    finally:
        run.close()


def test_set_state_is_set_particles_in_native_precision(B):
    """ann_set_state of a state read with ann_get_state loads the same state as ann_set_particles of
    the same values in FP64: the steps after it are bit-identical (host arrays and device tensors);
    a density deviation <= -1 is rejected."""
    import torch

    ic = random_velocity_ic(64, 13, rho_scale=1e-3)
    p = params(64, c0_min=0.05)
    p["dt"] = stable_dt(p)
    src = GpuRun(B, p, ic)
    a, b = GpuRun(B, p, ic), GpuRun(B, p, ic)
    try:
        src.step(4)
        st = B.ann_get_state(src.ctx, src.n)
        B.ann_set_particles(a.ctx, st["X"], st["Y"], st["UX"].astype(np.float64), st["UY"].astype(np.float64),
                            st["Q11"].astype(np.float64), st["Q12"].astype(np.float64),
                            1.0 + st["DRHO"].astype(np.float64))
        B.ann_set_state(b.ctx, {k: torch.from_numpy(v).cuda() for k, v in st.items()})
        assert np.array_equal(B.ann_get_state(b.ctx, b.n)["DRHO"], st["DRHO"])
        a.step(6)
        b.step(6)
        sa, sb = B.ann_get_state(a.ctx, a.n), B.ann_get_state(b.ctx, b.n)
        for f in B.STATE_FIELDS:
            assert np.array_equal(sa[f], sb[f]), f
        B.ann_set_state(b.ctx, st)   # host arrays
        b.step(6)
        sh = B.ann_get_state(b.ctx, b.n)
        for f in B.STATE_FIELDS:
            assert np.array_equal(sa[f], sh[f]), f
        bad = dict(st)
        bad["DRHO"] = st["DRHO"].copy()
        bad["DRHO"][7] = -1.0
        with pytest.raises(B.AnnError) as e:
            B.ann_set_state(b.ctx, bad)
        assert e.value.status == -6
    finally:
        for r in (src, a, b):
            r.close()


def test_update_state_round_trip_and_moved_particles(B, orc):
    """ann_get_state -> ann_update_state of the same values between steps (pageable host arrays,
    device tensors, and page-locked host arrays, which the kernels read and write over the host
    link) leaves the trajectory bit-identical to plain steps, with no extra re-sort.  A state
    moved far from where the last re-sort put the particles makes the next step re-sort, and that
    step matches the oracle started from the moved state."""
    import torch

    ic = random_velocity_ic(64, 17)
    p = params(64, c0_min=0.05)
    p["dt"] = stable_dt(p)
    a, b = GpuRun(B, p, ic), GpuRun(B, p, ic)
    pinned = {f: torch.empty(b.n, dtype=torch.float64 if f in ("X", "Y") else torch.float32).pin_memory().numpy()
              for f in B.FULL_STATE}
    try:
        a.step(12)
        b.step(3)
        for k in range(9):
            if k % 3 == 2:
                st = B.ann_get_state(b.ctx, b.n, out=pinned)
            else:
                st = B.ann_get_state(b.ctx, b.n)
                if k % 3 == 1:
                    st = {f: torch.from_numpy(v).cuda() for f, v in st.items()}
            B.ann_update_state(b.ctx, st)
            b.step(1)
        sa, sb = B.ann_get_state(a.ctx, a.n), B.ann_get_state(b.ctx, b.n)
        for f in B.FULL_STATE:
            assert np.array_equal(sa[f], sb[f]), f
        da, db = B.ann_get_diagnostics(a.ctx), B.ann_get_diagnostics(b.ctx)
        assert da["resorts"] == db["resorts"] and da["step"] == db["step"] == 12
        # move every particle by (0.37, 0.81) mod 1 and restart the accelerations
        moved = {f: sb[f] for f in ("UX", "UY", "Q11", "Q12", "DRHO")}
        moved["X"] = np.mod(sb["X"] + 0.37, 1.0)
        moved["Y"] = np.mod(sb["Y"] + 0.81, 1.0)
        B.ann_update_state(b.ctx, moved)
        b.step(1)
        assert B.ann_get_diagnostics(b.ctx)["resorts"] == db["resorts"] + 1
        st = {"x": moved["X"], "y": moved["Y"], "ux": moved["UX"].astype(np.float64),
              "uy": moved["UY"].astype(np.float64), "q11": moved["Q11"].astype(np.float64),
              "q12": moved["Q12"].astype(np.float64), "rho": 1.0 + moved["DRHO"].astype(np.float64)}
        want, _ = orc.step(oracle_params(orc, p, "cells"), st, 1, record=True)
        errs = compare_state(b.state(), want, moved["X"], moved["Y"])
        assert all(e <= 1e-5 for e in errs.values()), errs
    finally:
        a.close()
        b.close()


def test_state_transfer_through_page_locked_host_memory(B):
    """ann_get_state into page-locked host arrays (one kernel writes them over the host link) gives
    the bytes of the staged copy, with some destinations NULL and with a mix of page-locked and
    pageable arrays (which takes the staged path); ann_update_state from page-locked arrays, with
    DRHO, AX and AY left out, gives the state that the same pageable arrays give."""
    import torch

    def pin(v):
        return torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()

    ic = random_velocity_ic(48, 23)
    p = params(48, c0_min=0.05)
    p["dt"] = stable_dt(p)
    a, b = GpuRun(B, p, ic), GpuRun(B, p, ic)
    try:
        a.step(5)
        b.step(5)
        ref = B.ann_get_state(a.ctx, a.n)
        full = B.ann_get_state(a.ctx, a.n, out={f: pin(np.zeros_like(v)) for f, v in ref.items()})
        part = B.ann_get_state(a.ctx, a.n, out={f: pin(np.zeros_like(ref[f])) for f in ("Y", "UX", "Q12", "AY")})
        mixed = {f: (pin(np.zeros_like(v)) if i % 2 else np.zeros_like(v)) for i, (f, v) in enumerate(ref.items())}
        mixed = B.ann_get_state(a.ctx, a.n, out=mixed)
        for f in B.FULL_STATE:
            assert np.array_equal(full[f], ref[f]), f
            assert np.array_equal(mixed[f], ref[f]), f
        for f, v in part.items():
            assert np.array_equal(v, ref[f]), f
        # a new state (velocities halved, positions shifted by a tenth of a cell), DRHO/AX/AY absent
        new = {"X": np.mod(ref["X"] + 0.002, 1.0), "Y": ref["Y"], "UX": 0.5 * ref["UX"], "UY": 0.5 * ref["UY"],
               "Q11": ref["Q11"], "Q12": ref["Q12"]}
        B.ann_update_state(a.ctx, {f: pin(v) for f, v in new.items()})
        B.ann_update_state(b.ctx, new)
        sa, sb = B.ann_get_state(a.ctx, a.n), B.ann_get_state(b.ctx, b.n)
        for f in B.FULL_STATE:
            assert np.array_equal(sa[f], sb[f]), f
        assert np.all(sa["DRHO"] == 0.0) and np.all(sa["AX"] == 0.0)
        a.step(3)
        b.step(3)
        sa, sb = B.ann_get_state(a.ctx, a.n), B.ann_get_state(b.ctx, b.n)
        for f in B.FULL_STATE:
            assert np.array_equal(sa[f], sb[f]), f
        bad = {f: pin(v) for f, v in new.items()}
        bad["UY"][3] = np.nan
        with pytest.raises(B.AnnError) as e:
            B.ann_update_state(a.ctx, bad)
        assert e.value.status == -6
    finally:
        a.close()
        b.close()


def test_isolated_particle_is_a_singular_correction_tensor(B, orc):
    """The method's degenerate case: a particle with no neighbour within 3h has alpha = 0 (Eq. 22
    cannot be inverted).  The step reports SINGULAR_ALPHA instead of producing infinities, and the
    context stays usable.  The ring of particles pushed out to make the gap keeps full supports."""
    nx = 64
    ic = si.jittered_lattice(nx, seed=6)
    h = 1.3 / nx
    x, y = ic["x"].copy(), ic["y"].copy()
    cx = cy = 0.5
    dx, dy = x - cx, y - cy
    r = np.hypot(dx, dy)
    inside = r < 4.0 * h
    k0 = int(np.argmin(r))
    scale = np.where(inside, 4.0 * h / np.maximum(r, 1e-12), 1.0)
    x, y = cx + dx * scale, cy + dy * scale
    x[k0], y[k0] = cx, cy                       # the isolated particle
    rp, cols = orc.neighbors(x, y, 1.0, h)
    assert rp[k0 + 1] == rp[k0]                 # no neighbour within 3h
    ctx = B.ann_create(gpu_params(B, params(nx), nx * nx))
    try:
        B.ann_set_particles(ctx, x, y, ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        with pytest.raises(B.AnnError) as e:
            B.ann_step(ctx, 1)
        assert e.value.status == -7
        assert B.ann_get_diagnostics(ctx)["error_bits"] & 16
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        B.ann_step(ctx, 1)
    finally:
        B.ann_destroy(ctx)


def _bits(state):
    """The state's arrays as raw bytes, so that NaN compares equal to itself bit for bit."""
    return {f: np.ascontiguousarray(v).view(np.uint8) for f, v in state.items()}


def test_failed_step_leaves_the_last_completed_state(B):
    """Section 3.1's boundary contract: a step that fails leaves the state of the last completed
    step.  A strongly active flow (zeta = 50, eta = 0.01) in ANN_DT_CHECK mode accelerates until its
    midpoint velocity breaks 0.25 h / (c0 + max|u|) in pass C of some step k, after pass B has
    written Q^{n+1} and (for a re-sorting step) the cell structure has moved.  A reference context
    steps one call at a time to find k; a second context runs all the steps in one call.  The
    second one reports CFL_VIOLATION, and its state, step count, time and pathline image counts
    equal the reference's after step k - 1 bit for bit.  Reloading a checkpoint then continues
    both bit-identically."""
    import os
    import tempfile

    nx = 64
    ic = random_velocity_ic(nx, 31, u_scale=1e-3)
    p = params(nx, zeta=50.0, eta=0.01, dt=1e-4)
    gp = gpu_params(B, p, ic["n"])
    gp.dt_mode = 2
    ids = np.arange(0, ic["n"], 7, dtype=np.int64)
    ref, run = B.ann_create(gp), B.ann_create(gp)
    tmp = tempfile.mkdtemp()
    try:
        for c in (ref, run):
            B.ann_set_particles(c, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
        good, k = None, None
        for step in range(1, 81):
            try:
                B.ann_step(ref, 1)
            except B.AnnError as e:
                assert e.status == -13, e
                k = step
                break
            good = (B.ann_get_state(ref, ic["n"]), B.ann_get_unwrapped(ref, ids))
            if step == 1:
                B.ann_save_state(ref, os.path.join(tmp, "s1.bin"))
        assert k is not None and k >= 3, "the flow should break the CFL bound after a few steps"
        with pytest.raises(B.AnnError) as e:
            B.ann_step(run, k + 5)
        assert e.value.status == -13
        d = B.ann_get_diagnostics(run)
        assert d["step"] == k - 1 and d["error_bits"] & 32
        assert d["t"] == pytest.approx((k - 1) * p["dt"], rel=1e-12)
        got = B.ann_get_state(run, ic["n"])
        want = _bits(good[0])
        for f, v in _bits(got).items():
            assert np.array_equal(v, want[f]), f
        assert np.array_equal(B.ann_get_unwrapped(run, ids), good[1])
        # the reference, also rolled back, holds the same state
        for f, v in _bits(B.ann_get_state(ref, ic["n"])).items():
            assert np.array_equal(v, want[f]), f
        # a checkpoint load clears the error; both contexts continue identically
        for c in (ref, run):
            B.ann_load_state(c, os.path.join(tmp, "s1.bin"))
            B.ann_step(c, 1)
        a, b = _bits(B.ann_get_state(ref, ic["n"])), _bits(B.ann_get_state(run, ic["n"]))
        for f in a:
            assert np.array_equal(a[f], b[f]), f
    finally:
        B.ann_destroy(ref)
        B.ann_destroy(run)


def test_singular_step_fails_without_a_trace(B, orc):
    """The degenerate case of Eq. 22 (a particle with no neighbour, alpha = 0) fails the step in
    pass B with SINGULAR_ALPHA after pass B has written Q^{n+1} into the step's output set; the
    state read back afterwards is the loaded one, bit for bit, at step 0."""
    nx = 64
    ic = si.jittered_lattice(nx, seed=6)
    h = 1.3 / nx
    x, y = ic["x"].copy(), ic["y"].copy()
    dx, dy = x - 0.5, y - 0.5
    r = np.hypot(dx, dy)
    k0 = int(np.argmin(r))
    scale = np.where(r < 4.0 * h, 4.0 * h / np.maximum(r, 1e-12), 1.0)
    x, y = 0.5 + dx * scale, 0.5 + dy * scale
    x[k0], y[k0] = 0.5, 0.5                      # the isolated particle
    rp, _ = orc.neighbors(x, y, 1.0, h)
    assert rp[k0 + 1] == rp[k0]
    ctx = B.ann_create(gpu_params(B, params(nx), nx * nx))
    try:
        B.ann_set_particles(ctx, x, y, ic["ux"], ic["uy"], ic["q11"], ic["q12"])
        put = _bits(B.ann_get_state(ctx, nx * nx))
        with pytest.raises(B.AnnError) as e:
            B.ann_step(ctx, 3)
        assert e.value.status == -7
        d = B.ann_get_diagnostics(ctx)
        assert d["step"] == 0 and d["t"] == 0.0 and d["error_bits"] & 16
        for f, v in _bits(B.ann_get_state(ctx, nx * nx)).items():
            assert np.array_equal(v, put[f]), f
    finally:
        B.ann_destroy(ctx)
