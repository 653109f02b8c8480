"""GPU flow diagnostics (results section) against the oracle, through the C-ABI.

* Shepard gridding of the present state matches the FP64 oracle on the same particle state
  (downloaded from the GPU) to FP32 round-off, whichever arrays hold the state: after
  ann_set_particles (the call runs the search itself), after steps, after a neighbour export.
* Spectrum, correlation, defects and mixing match the oracle's definitions applied to the GPU's
  own grid / positions: FFT and sums to 1e-12, defect maps and bin counts exactly.
* Pathlines: the image counts follow particles across the periodic faces.
* Calling the diagnostics leaves the trajectory bit-identical; checkpoints keep image counts and
  colours.
* Full size: 1024 x 1024 particles on a 1024 x 1024 grid, sampled nodes against the oracle.
"""
import numpy as np
import pytest

import sph_inputs as si
from _sph import GpuRun, oracle_params, oracle_state, params, random_velocity_ic, relerr, stable_dt

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-5   # FP32 Shepard sums against FP64


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding


@pytest.fixture(scope="module")
def D():
    from oracle import diagnostics

    return diagnostics


def _state(run):
    return {k: run.field(f) for k, f in (("x", "X"), ("y", "Y"), ("ux", "UX"), ("uy", "UY"),
                                          ("q11", "Q11"), ("q12", "Q12"))}


def _check_grid(B, D, run, p, M):
    g = B.ann_grid_fields(run.ctx, M)
    s = _state(run)
    want, ws = D.grid_shepard(s["x"], s["y"], [s["ux"], s["uy"], s["q11"], s["q12"]], p["L"], p["h"], M)
    errs = [relerr(g[q], want[q]) for q in range(4)] + [relerr(g[4], ws)]
    assert max(errs) <= GRID_TOL, errs
    return g


def _case(nx=64, seed=4):
    ic = random_velocity_ic(nx, seed, u_scale=1e-2, rho_scale=1e-4)
    p = params(nx, c0_min=0.05)
    p["dt"] = stable_dt(p)
    return ic, p


def test_grid_matches_oracle_from_every_state_source(B, D):
    ic, p = _case()
    run = GpuRun(B, p, ic)
    try:
        _check_grid(B, D, run, p, 64)        # after ann_set_particles: the call searches first
        run.step(3)
        _check_grid(B, D, run, p, 64)        # after steps: the state arrays, cell order of the step
        _check_grid(B, D, run, p, 128)       # finer than the particle spacing
        _check_grid(B, D, run, p, 32)
        B.ann_get_neighbors(run.ctx, run.n)  # the evaluation copy re-sorted at the present state
        _check_grid(B, D, run, p, 64)
    finally:
        run.close()


def test_spectrum_correlation_defects_on_the_gpu_grid(B, D):
    ic, p = _case(seed=6)
    run = GpuRun(B, p, ic)
    try:
        run.step(5)
        M = 64
        g = B.ann_grid_fields(run.ctx, M)
        E = B.ann_energy_spectrum(run.ctx, M)
        C1, l1 = B.ann_vorticity_correlation(run.ctx, M, all_origins=True)
        C0, _ = B.ann_vorticity_correlation(run.ctx, M, all_origins=False)
        counts, m = B.ann_defects(run.ctx, M, with_map=True)
    finally:
        run.close()
    w, Ew = D.energy_spectrum(g[0], g[1], p["L"])
    assert E.size == Ew.size == B.ann_spectrum_shells(M)
    assert np.abs(E - Ew).max() <= 1e-12 * Ew.sum()
    assert E.sum() == pytest.approx(0.5 * np.mean(g[0] ** 2 + g[1] ** 2), rel=1e-12)
    om = D.vorticity(g[0], g[1], p["L"])
    assert np.abs(C1 - D.correlation(om, True)).max() < 1e-12
    assert np.abs(C0 - D.correlation(om, False)).max() < 1e-9 * np.abs(C0).max()
    want_l = D.length_scales(D.correlation(om, True), p["L"])
    for a, b in zip(l1, want_l):
        assert (np.isnan(a) and np.isnan(b)) or a == pytest.approx(b, rel=1e-10)
    mo, co = D.defects(g[2], g[3])
    assert np.array_equal(m, mo) and list(counts) == list(co)
    assert int(m.astype(np.int64).sum()) == 0   # total charge on the torus
    slope = B.ann_spectrum_slope(E, p["L"], w[2], w[20])
    assert slope == pytest.approx(D.spectrum_slope(w, E, w[2], w[20]), rel=1e-10, abs=1e-12)


def test_known_defects_from_particles(B, D):
    """Particles carrying (Q11, Q12) = (sin 2 pi (x - x0), sin 2 pi (y - y0)): two +1/2 and two
    -1/2 defects, placed inside plaquettes of the grid."""
    nx, M = 64, 64
    ic = si.jittered_lattice(nx, seed=2)
    x0 = y0 = 0.37 / M
    ic["q11"] = np.sin(2 * np.pi * (ic["x"] - x0))
    ic["q12"] = np.sin(2 * np.pi * (ic["y"] - y0))
    run = GpuRun(B, params(nx), ic)
    try:
        counts, m = B.ann_defects(run.ctx, M, with_map=True)
    finally:
        run.close()
    assert list(counts) == [2, 2, 0]
    assert m[0, 0] == 1 and m[M // 2, M // 2] == 1 and m[0, M // 2] == -1 and m[M // 2, 0] == -1


def test_mixing_index(B, D):
    ic, p = _case(seed=8)
    x, y = ic["x"], ic["y"]
    quad = ((x >= 0.5).astype(np.uint8) + 2 * (y >= 0.5).astype(np.uint8)).astype(np.uint8)
    run = GpuRun(B, p, ic)
    try:
        I0, per0 = B.ann_mixing_index(run.ctx, 2)
        assert I0 == 0.0 and np.all(np.isnan(per0))   # one colour: nothing to mix
        B.ann_set_colors(run.ctx, quad)
        I, per = B.ann_mixing_index(run.ctx, 2)
        assert I == pytest.approx(1.0, abs=1e-15) and np.allclose(per[:4], 1.0, atol=1e-15)
        assert np.all(np.isnan(per[4:]))
        run.step(10)
        s = _state(run)
        for G in (2, 8, 13):
            got, per = B.ann_mixing_index(run.ctx, G)
            want, pw = D.mixing_index(s["x"], s["y"], quad, p["L"], G)
            assert got == pytest.approx(want, rel=1e-13, abs=1e-15)
            assert np.allclose(per[:4], pw, rtol=1e-13, atol=1e-15)
        with pytest.raises(B.AnnError):
            B.ann_set_colors(run.ctx, np.full(run.n, 16, dtype=np.uint8))
        with pytest.raises(B.AnnError):
            B.ann_mixing_index(run.ctx, 0)
    finally:
        run.close()


def test_pathlines_across_periodic_faces(B, D, orc):
    """A uniform translation (exact: no pressure, viscous, active or APD force acts) carries every
    particle across the x faces and many across the y faces; unwrapped positions follow the
    straight lines, agree with unwrapping the GPU's own wrapped positions step by step, and with
    the oracle's trajectory."""
    nx = 32
    ic = si.jittered_lattice(nx, seed=0)
    n = ic["n"]
    ic["q11"] = np.full(n, 0.6)
    ic["q12"] = np.full(n, 0.2)
    ic["ux"] = np.full(n, 15.0)
    ic["uy"] = np.full(n, -4.0)
    p = params(nx, eta=0.01, zeta=0.0, K=0.0)
    run = GpuRun(B, p, ic)
    ids = np.arange(n)
    host = D.Unwrapper(ic["x"], ic["y"], 1.0)
    st = oracle_state(ic)
    P = oracle_params(orc, p, "cells")
    orc_u = D.Unwrapper(ic["x"], ic["y"], 1.0)
    try:
        for _ in range(40):
            run.step(20)
            host.update(run.field("X"), run.field("Y"))
            st, _ = orc.step(P, st, 20)
            orc_u.update(st["x"], st["y"])
        xy = B.ann_get_unwrapped(run.ctx, ids)
    finally:
        run.close()
    t = 800 * p["dt"]
    assert np.abs(xy[:, 0] - host.ux).max() < 1e-12 and np.abs(xy[:, 1] - host.uy).max() < 1e-12
    assert np.abs(xy[:, 0] - (ic["x"] + 15.0 * t)).max() < 1e-6
    assert np.abs(xy[:, 1] - (ic["y"] - 4.0 * t)).max() < 1e-6
    # the GPU adds FP32 increments dt/2 u to FP64 positions (relative rounding 3e-8 per increment)
    assert np.abs(xy[:, 0] - orc_u.ux).max() < 1e-6 and np.abs(xy[:, 1] - orc_u.uy).max() < 1e-6
    assert (xy[:, 0] >= 1.0).all() and (xy[:, 1] < 0.0).any()


def test_diagnostics_leave_the_trajectory_unchanged(B):
    ic, p = _case(seed=10)
    a = GpuRun(B, p, ic)
    b = GpuRun(B, p, ic)
    try:
        for run in (a,):
            B.ann_grid_fields(run.ctx, 64)          # before any step: runs the search
            B.ann_defects(run.ctx, 32)
        a.step(7)
        b.step(7)
        B.ann_energy_spectrum(a.ctx, 64)
        B.ann_vorticity_correlation(a.ctx, 128)
        B.ann_mixing_index(a.ctx, 4)
        B.ann_get_unwrapped(a.ctx, np.arange(10))
        a.step(9)
        b.step(9)
        sa, sb = a.state(), b.state()
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
    finally:
        a.close()
        b.close()


def test_checkpoint_keeps_images_and_colours(B, tmp_path):
    nx = 32
    ic = si.jittered_lattice(nx, seed=1)
    n = ic["n"]
    ic["ux"] = np.full(n, 9.0)
    ic["uy"] = np.full(n, 5.0)
    p = params(nx, eta=0.01, zeta=0.0, K=0.0)
    col = (np.arange(n) % 3).astype(np.uint8)
    a = GpuRun(B, p, ic)
    try:
        B.ann_set_colors(a.ctx, col)
        a.step(300)
        path = str(tmp_path / "s.bin")
        B.ann_save_state(a.ctx, path)
        b = GpuRun(B, p, si.jittered_lattice(nx, seed=9))
        try:
            B.ann_load_state(b.ctx, path)
            ua, ub = B.ann_get_unwrapped(a.ctx, np.arange(n)), B.ann_get_unwrapped(b.ctx, np.arange(n))
            assert np.array_equal(ua, ub) and (ua[:, 0] > 1.0).any() and (ua[:, 1] > 1.0).any()
            (Ia, pa), (Ib, pb) = B.ann_mixing_index(a.ctx, 4), B.ann_mixing_index(b.ctx, 4)
            assert Ia == Ib and Ia > 0.0 and np.array_equal(pa, pb, equal_nan=True)
            a.step(5)
            b.step(5)
            assert np.array_equal(B.ann_get_unwrapped(a.ctx, np.arange(n)), B.ann_get_unwrapped(b.ctx, np.arange(n)))
        finally:
            b.close()
    finally:
        a.close()


def test_bad_arguments(B):
    ic, p = _case(nx=32)
    run = GpuRun(B, p, ic)
    try:
        for M in (7, 12, 4096, 0):
            with pytest.raises(B.AnnError):
                B.ann_grid_fields(run.ctx, M)
        with pytest.raises(B.AnnError):
            B.ann_get_unwrapped(run.ctx, np.array([run.n]))
        with pytest.raises(B.AnnError):
            B.ann_get_unwrapped(run.ctx, np.array([-1]))
        assert B.ann_spectrum_shells(64) == 46
    finally:
        run.close()


def test_full_size_grid_sampled_nodes(B, D):
    """1024 x 1024 particles after two steps of the benchmark set-up, gridded at M = 1024: sampled
    nodes against the oracle's per-node sums over all particles; spectrum sums (Parseval), defect
    counts and mixing against the oracle's definitions on the GPU grid and positions."""
    nx, M = 1024, 1024
    p = params(nx, zeta=0.08, K=0.02)
    from _sph import gpu_params

    gp = gpu_params(B, p, nx * nx)
    gp.dt_mode = 1
    p["dt"] = B.ann_grid_info(gp).dt_effective
    ic = si.jittered_lattice(nx, seed=0)
    run = GpuRun(B, p, ic)
    try:
        quad = ((ic["x"] >= 0.5).astype(np.uint8) + 2 * (ic["y"] >= 0.5).astype(np.uint8)).astype(np.uint8)
        B.ann_set_colors(run.ctx, quad)
        run.step(2)
        g = B.ann_grid_fields(run.ctx, M)
        E = B.ann_energy_spectrum(run.ctx, M)
        counts, m = B.ann_defects(run.ctx, M, with_map=True)
        I, _ = B.ann_mixing_index(run.ctx, 16)
        s = _state(run)
    finally:
        run.close()
    rng = si.uniform53(77, 200)
    nodes = np.unique((rng * M * M).astype(np.int64))[:100]
    want, ws = D.grid_nodes(s["x"], s["y"], [s["ux"], s["uy"], s["q11"], s["q12"]], 1.0, p["h"], M, nodes)
    got = np.stack([g[q].ravel()[nodes] for q in range(4)], axis=1)
    assert relerr(got[:, 2:], want[:, 2:]) <= GRID_TOL
    assert relerr(g[4].ravel()[nodes], ws) <= GRID_TOL
    assert E.sum() == pytest.approx(0.5 * np.mean(g[0] ** 2 + g[1] ** 2), rel=1e-10)
    mo, co = D.defects(g[2], g[3])
    assert np.array_equal(m, mo) and list(counts) == list(co) and counts[0] > 0
    assert I == pytest.approx(D.mixing_index(s["x"], s["y"], quad, 1.0, 16)[0], rel=1e-12)
