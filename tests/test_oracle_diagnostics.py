"""Pins of the diagnostics oracle (results section: energy spectrum, vorticity correlation,
defects, mixing, pathlines) against closed forms, exact counts and invariants."""
import math

import numpy as np
import pytest

import sph_inputs as si


@pytest.fixture(scope="module")
def D():
    from oracle import diagnostics

    return diagnostics


def _lattice(nx, jitter=0.0, seed=0):
    ic = si.jittered_lattice(nx, seed=seed, jitter=jitter)
    return ic, 1.3 * ic["dx"]


# ---------------------------------------------------------------- Shepard gridding


def test_single_particle_weight_is_the_kernel(D):
    """One particle on a node: the weight is W(0) = 66 a_d with a_d = 7 / (478 pi h^2) (Eq. 18),
    and the value is the particle's own; nodes beyond 3h get weight 0 and value 0."""
    L, h, M = 1.0, 0.05, 16
    x, y = np.array([4 / 16]), np.array([8 / 16])
    g, ws = D.grid_shepard(x, y, [np.array([2.5])], L, h, M, mode="brute")
    w0 = 66.0 * 7.0 / (478.0 * math.pi * h * h)
    assert ws[8, 4] == pytest.approx(w0, rel=1e-14)
    assert g[0, 8, 4] == pytest.approx(2.5, rel=1e-15)
    # one node over: r = 1/16 = 1.25 h, W = a_d ((3 - b)^5 - 6 (2 - b)^5)
    b = (1 / 16) / h
    assert ws[8, 5] == pytest.approx(7.0 / (478.0 * math.pi * h * h) * ((3 - b) ** 5 - 6 * (2 - b) ** 5),
                                     rel=1e-13)
    far = (np.arange(M)[None, :] - 4) ** 2 + (np.arange(M)[:, None] - 8) ** 2 >= (3 * h * M) ** 2
    assert np.all(ws[far] == 0.0) and np.all(g[0][far] == 0.0)


def test_constants_exact_and_brute_equals_cells(D):
    ic, h = _lattice(32, jitter=0.2, seed=3)
    r = si.uniform53(5, ic["n"]) - 0.5
    g1, w1 = D.grid_shepard(ic["x"], ic["y"], [np.full(ic["n"], 0.7), r], 1.0, h, 32, mode="brute")
    g2, w2 = D.grid_shepard(ic["x"], ic["y"], [np.full(ic["n"], 0.7), r], 1.0, h, 32, mode="cells")
    assert np.all(w1 > 0)
    assert np.abs(g1[0] - 0.7).max() < 1e-15
    assert np.abs(g1 - g2).max() < 1e-14 and np.abs(w1 - w2).max() < 1e-10 * w1.max()


def test_linear_field_exact_at_symmetric_nodes(D):
    """Unjittered lattice, nodes at the centres of lattice squares: every node's neighbourhood is
    point-symmetric, so the weighted centroid is the node and linear fields come out exactly."""
    ic, h = _lattice(32)
    x, y = ic["x"], ic["y"]
    g, _ = D.grid_shepard(x, y, [0.3 + 2.0 * x - 1.5 * y], 1.0, h, 32, mode="cells")
    gx = np.arange(32)[None, :] / 32
    gy = np.arange(32)[:, None] / 32
    inner = (np.abs(gx - 0.5) < 0.5 - 4 * h) & (np.abs(gy - 0.5) < 0.5 - 4 * h)
    want = 0.3 + 2.0 * gx - 1.5 * gy
    assert np.abs((g[0] - want)[inner]).max() < 1e-13


def test_sampled_nodes_equal_grid(D):
    ic, h = _lattice(24, jitter=0.1, seed=1)
    f = [ic["q11"], ic["q12"]]
    g, ws = D.grid_shepard(ic["x"], ic["y"], f, 1.0, h, 24, mode="brute")
    nodes = np.array([0, 5, 24 * 7 + 3, 24 * 24 - 1])
    v, w = D.grid_nodes(ic["x"], ic["y"], f, 1.0, h, 24, nodes)
    assert np.array_equal(v[:, 0], g[0].ravel()[nodes]) and np.array_equal(w, ws.ravel()[nodes])


# ---------------------------------------------------------------- spectrum


def test_parseval_and_single_modes(D):
    M, L = 32, 1.0
    rng = si.uniform53(9, 2 * M * M).reshape(2, M, M) - 0.5
    w, E = D.energy_spectrum(rng[0], rng[1], L)
    assert E.sum() == pytest.approx(0.5 * np.mean(rng[0] ** 2 + rng[1] ** 2), rel=1e-12)
    assert w[3] == pytest.approx(2 * math.pi * 3)
    X, Y = np.meshgrid(np.arange(M) / M, np.arange(M) / M)
    for kx, ky, n in ((4, 0, 4), (3, 4, 5), (0, 7, 7)):
        w, E = D.energy_spectrum(np.cos(2 * math.pi * (kx * X + ky * Y)), np.zeros((M, M)), L)
        assert E[n] == pytest.approx(0.25, rel=1e-12)
        assert np.abs(np.delete(E, n)).max() < 1e-25


def test_shell_membership_counts(D):
    """Modes per shell equal a direct count of integer wavevectors with n - 1/2 <= |k| < n + 1/2
    (4 |k|^2 compared with (2n -+ 1)^2 in integers)."""
    M = 16
    s = D.shell_index(M)
    ks = np.fft.fftfreq(M, d=1.0 / M).round().astype(int)
    for n in range(D.n_shells(M)):
        lo = (2 * n - 1) ** 2 if n > 0 else 0
        cnt = sum(1 for a in ks for b in ks if lo <= 4 * (a * a + b * b) < (2 * n + 1) ** 2)
        assert int((s == n).sum()) == cnt, n
    assert s.max() == D.n_shells(M) - 1


def test_slope_of_a_power_law(D):
    w = 2 * np.pi * np.arange(40)
    E = np.zeros(40)
    E[1:] = 3.0 * w[1:] ** -4.0
    assert D.spectrum_slope(w, E, w[2], w[30]) == pytest.approx(-4.0, abs=1e-12)


# ---------------------------------------------------------------- vorticity and correlation


def test_vorticity_central_difference_closed_form(D):
    M, L = 64, 1.0
    X, Y = np.meshgrid(np.arange(M) / M, np.arange(M) / M)
    ux, uy = -np.sin(2 * np.pi * Y), np.sin(2 * np.pi * X)
    om = D.vorticity(ux, uy, L)
    Dx = L / M
    fac = math.sin(2 * math.pi * Dx) / Dx   # central difference of sin(2 pi x)
    assert np.abs(om - fac * (np.cos(2 * np.pi * X) + np.cos(2 * np.pi * Y))).max() < 1e-11
    assert np.abs(D.vorticity(np.full((M, M), 0.3), np.full((M, M), -1.0), L)).max() == 0.0


def test_correlation_of_a_cosine(D):
    M, m = 64, 2
    X = np.arange(M) / M
    f = np.tile(np.cos(2 * np.pi * m * X + 0.3), (M, 1))
    C = D.correlation(f, all_origins=True)
    k = np.arange(M // 2 + 1)
    assert np.abs(C - np.cos(2 * np.pi * m * k / M)).max() < 1e-13
    C1 = D.correlation(f, all_origins=False)
    i0 = M // 2
    want = np.cos(2 * np.pi * m * (i0 + k) / M + 0.3) / np.cos(2 * np.pi * m * i0 / M + 0.3)
    assert np.abs(C1 - want).max() < 1e-12
    l0, l2 = D.length_scales(C, 1.0)
    assert l0 == pytest.approx(1.0 / (4 * m), abs=1e-12)
    # 0.2 max: between the grid points around acos(0.2) / (2 pi m), linear interpolation
    r02 = math.acos(0.2) / (2 * math.pi * m)
    assert abs(l2 - r02) < (1.0 / M) ** 2 * (2 * math.pi * m) ** 2


# ---------------------------------------------------------------- defects


def _offset_grid(M):
    g = (np.arange(M) + 0.25) / M
    return np.meshgrid(g, g)


def test_four_known_defects(D):
    """(Q11, Q12) = (sin 2 pi x, sin 2 pi y) vanishes at (0,0) and (1/2,1/2) with winding +1 and at
    (1/2,0), (0,1/2) with winding -1: two +1/2 and two -1/2 director defects."""
    M = 32
    X, Y = _offset_grid(M)
    m, counts = D.defects(np.sin(2 * np.pi * X), np.sin(2 * np.pi * Y))
    assert list(counts) == [2, 2, 0]
    a, b = M - 1, M // 2 - 1   # plaquettes containing coordinate 0 and 1/2
    assert m[a, a] == 1 and m[b, b] == 1 and m[a, b] == -1 and m[b, a] == -1
    # nematic symmetry: Q -> -Q (director turned by pi/2) keeps the charges
    m2, c2 = D.defects(-np.sin(2 * np.pi * X), -np.sin(2 * np.pi * Y))
    assert np.array_equal(m, m2)
    # a uniform director has none
    _, c0 = D.defects(np.full((M, M), 0.4), np.full((M, M), -0.9))
    assert list(c0) == [0, 0, 0]


def test_total_charge_vanishes_on_the_torus(D):
    for seed in range(4):
        r = si.uniform53(100 + seed, 2 * 24 * 24).reshape(2, 24, 24) - 0.5
        m, counts = D.defects(r[0], r[1])
        assert int(m.astype(np.int64).sum()) == 0
        assert counts[0] + counts[1] > 0


# ---------------------------------------------------------------- mixing


def test_mixing_index_limits(D):
    ic, _ = _lattice(32)
    x, y = ic["x"], ic["y"]
    seg = (x >= 0.5).astype(int)
    assert D.mixing_index(x, y, seg, 1.0, 2)[0] == pytest.approx(1.0, abs=1e-15)
    assert D.mixing_index(x, y, seg, 1.0, 4)[0] == pytest.approx(1.0, abs=1e-15)
    ix = np.floor(x * 32).astype(int)
    iy = np.floor(y * 32).astype(int)
    checker = (ix + iy) % 2
    assert D.mixing_index(x, y, checker, 1.0, 8)[0] == pytest.approx(0.0, abs=1e-15)
    assert D.mixing_index(x, y, np.zeros(x.size, dtype=int), 1.0, 4)[0] == 0.0
    quad = (x >= 0.5).astype(int) + 2 * (y >= 0.5).astype(int)
    I, Is = D.mixing_index(x, y, quad, 1.0, 2)
    assert I == pytest.approx(1.0, abs=1e-15) and np.all(np.abs(Is - 1.0) < 1e-15)


def test_mixing_index_hand_example(D):
    """Two bins: left holds colours (0, 0, 1), right (1, 1, 1, 0).  a_1 = 4/7; f = 1/3, 3/4;
    I_1 = ((1/3 - 4/7)^2 + (3/4 - 4/7)^2) / 2 / (4/7 * 3/7); I_0 = I_1 (two species)."""
    x = np.array([0.1, 0.2, 0.3, 0.6, 0.7, 0.8, 0.9])
    y = np.full(7, 0.5)
    c = np.array([0, 0, 1, 1, 1, 1, 0])
    I, Is = D.mixing_index(x, y, c, 1.0, 2)
    a = 4 / 7
    # bins 2 x 2: the particles sit in the top row (y = 0.5 -> row 1), bins (0, 1) and (1, 1)
    want = ((1 / 3 - a) ** 2 + (3 / 4 - a) ** 2) / 2 / (a * (1 - a))
    assert I == pytest.approx(want, rel=1e-14) and Is[0] == pytest.approx(want, rel=1e-14)


def test_unwrapper_follows_a_translation(D):
    ic, _ = _lattice(8)
    u = D.Unwrapper(ic["x"], ic["y"], 1.0)
    x, y = ic["x"].copy(), ic["y"].copy()
    for _ in range(30):
        x = (x + 0.07) % 1.0
        y = (y - 0.11) % 1.0
        u.update(x, y)
    assert np.abs(u.ux - (ic["x"] + 30 * 0.07)).max() < 1e-13
    assert np.abs(u.uy - (ic["y"] - 30 * 0.11)).max() < 1e-13
