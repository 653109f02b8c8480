"""Pins of the surrogate oracle: the hand-derived backward pass against central finite
differences of the FP64 forward pass, the aggregation and its adjoint, and invariants."""
import numpy as np
import pytest

import sph_inputs as si


@pytest.fixture(scope="module")
def S():
    from oracle import surrogate

    return surrogate


def _graph(S, orc, nx=10, seed=3, radius=3.0):
    ic = si.jittered_lattice(nx, seed=seed, jitter=0.2)
    h = 1.3 * ic["dx"]
    rp, cols = orc.neighbors(ic["x"], ic["y"], 1.0, h)
    return ic, S.Graph(ic["x"], ic["y"], 1.0, h, rp, cols, radius=radius)


def test_network_graph_is_the_2h_part_of_the_support(S, orc):
    """The 2h graph keeps exactly the support pairs closer than 2h (brute force over all pairs),
    is symmetric, and is still an SPH mean."""
    ic, G2 = _graph(S, orc, radius=2.0)
    _, G3 = _graph(S, orc)
    h, n = 1.3 * ic["dx"], G2.n
    dx = ic["x"][:, None] - ic["x"][None, :]
    dy = ic["y"][:, None] - ic["y"][None, :]
    dx -= np.round(dx)
    dy -= np.round(dy)
    r = np.sqrt(dx * dx + dy * dy)
    want = {(i, j) for i, j in zip(*np.nonzero((r < 2 * h) & ~np.eye(n, dtype=bool)))}
    got = set(zip(G2.rows.tolist(), G2.cols.tolist()))
    assert got == want and {(j, i) for i, j in got} == got
    assert len(G3.rows) > 2 * len(G2.rows)
    assert np.abs(G2.agg(np.full((n, 2), -1.5)) + 1.5).max() < 1e-14


def test_aggregation_mean_and_adjoint(S, orc):
    ic, G = _graph(S, orc)
    n = G.n
    assert np.abs(G.agg(np.full((n, 3), 2.5)) - 2.5).max() < 1e-14   # an SPH mean
    rng = si.uniform53(5, 2 * 3 * n).reshape(2, n, 3) - 0.5
    lhs = np.sum(G.agg(rng[0]) * rng[1])
    rhs = np.sum(rng[0] * G.agg_T(rng[1]))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # each row's weights: W(r)/S with S = W(0) + sum W (Eq. 19's sum), positive, summing to 1
    assert np.all(G.w > 0) and np.all(G.w_self > 0)
    assert np.abs(G.w_self + np.bincount(G.rows, weights=G.w, minlength=n) - 1.0).max() < 1e-14


def _random_problem(S, orc, seed=0):
    ic, G = _graph(S, orc, radius=2.0)
    p = S.init_params(seed)
    for k, b in (("b1", 0), ("b2", 1), ("b3", 2), ("bo", 3)):
        p[k] = 0.2 * (si.uniform53(seed + 60 + b, p[k].size) - 0.5)
    ux = 0.3 * (si.uniform53(seed + 50, G.n) - 0.5)
    uy = 0.3 * (si.uniform53(seed + 70, G.n) - 0.5)
    tend = si.uniform53(seed + 90, 8 * G.n).reshape(G.n, 8) - 0.5
    x = S.features(G, ic["q11"], ic["q12"], ux, uy, tend, 0.1, 8e-4, 0.02, 0.01, 0.005)
    t = si.uniform53(seed + 80, 4 * G.n).reshape(G.n, 4) - 0.5
    return G, p, x, t


def test_backward_matches_finite_differences(S, orc):
    G, p, x, t = _random_problem(S, orc)
    y, c = S.forward(p, G, x)
    g = S.backward(p, G, c, y, t)
    eps = 1e-6
    for ki, k in enumerate(S.ORDER):
        flat = p[k].reshape(-1)
        idx = np.unique((si.uniform53(300 + ki, 6) * flat.size).astype(int))
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp = S.loss(S.forward(p, G, x)[0], t)
            flat[i] = old - eps
            lm = S.loss(S.forward(p, G, x)[0], t)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-4), (k, i, fd, an)


def test_zero_weights_give_the_bias_and_permutation_equivariance(S, orc):
    G, p, x, t = _random_problem(S, orc, seed=1)
    z = {k: np.zeros_like(v) for k, v in p.items()}
    z["bo"] = np.array([0.1, -0.2, 0.3, 0.0])
    y, _ = S.forward(z, G, x)
    assert np.array_equal(y, np.tile(z["bo"], (G.n, 1)))
    # relabel the particles: outputs follow the relabelling
    ic, _ = _graph(S, orc)
    perm = np.argsort(si.uniform53(9, G.n))
    x2, y2 = ic["x"][perm], ic["y"][perm]
    rp, cols = orc.neighbors(x2, y2, 1.0, 1.3 * ic["dx"])
    G2 = S.Graph(x2, y2, 1.0, 1.3 * ic["dx"], rp, cols, radius=2.0)
    ya, _ = S.forward(p, G, x)
    yb, _ = S.forward(p, G2, x[perm])
    assert np.abs(yb - ya[perm]).max() < 1e-12


def test_features_of_a_uniform_state(S, orc):
    ic, G = _graph(S, orc)
    n = G.n
    tend = np.tile([2.0, -1.0, 3.0, 4.0, 0.5, 0.25, -0.5, 1.0], (n, 1))
    x = S.features(G, np.full(n, 0.4), np.full(n, -0.1), np.full(n, 0.02), np.full(n, 0.01), tend,
                   0.1, 8e-4, 0.02, 0.01, 0.005)
    assert np.abs(x[:, 4:8]).max() < 1e-15
    assert np.allclose(x[:, :4], [0.4, -0.1, 0.2, 0.1], atol=1e-15)
    # tendencies scaled to increments over k dt: a k dt / ys_u, m k dt / ys_q,
    # lap Q Gamma K k dt / ys_q, (div u, vort u) k dt
    want = [2 * 8e-4 / 0.005, -8e-4 / 0.005, 3 * 8e-4 / 0.01, 4 * 8e-4 / 0.01,
            0.5 * 0.02 * 8e-4 / 0.01, 0.25 * 0.02 * 8e-4 / 0.01, -0.5 * 8e-4, 8e-4]
    assert np.allclose(x[:, 8:], want, rtol=1e-14, atol=0)
    e = S.euler_increment(G, tend, 8e-4)   # uniform rates: the SPH mean leaves them unchanged
    assert np.allclose(e, [3 * 8e-4, 4 * 8e-4, 2 * 8e-4, -8e-4], rtol=1e-14, atol=0)


def test_smoothed_increment_damps_the_grid_scale(S, orc):
    """A checkerboard acceleration (the highest lattice wavenumber) is nearly removed by the SPH
    mean, while a long wave passes almost unchanged: the explicit velocity increment cannot amplify
    grid-scale modes.  The Q rate is taken as it is, particle by particle."""
    ic = si.jittered_lattice(24, seed=0, jitter=0.0)
    h = 1.3 * ic["dx"]
    rp, cols = orc.neighbors(ic["x"], ic["y"], 1.0, h)
    G = S.Graph(ic["x"], ic["y"], 1.0, h, rp, cols)
    ix = np.floor(ic["x"] * 24).astype(int)
    iy = np.floor(ic["y"] * 24).astype(int)
    checker = np.where((ix + iy) % 2 == 0, 1.0, -1.0)
    wave = np.cos(2 * np.pi * ic["x"])
    z = np.zeros(G.n)
    for f, lo, hi in ((checker, 0.0, 0.01), (wave, 0.8, 1.0)):
        tend = np.stack([z, f, z, z, z, z, z, z], axis=1)
        inc = S.euler_increment(G, tend, 1.0)
        ratio = np.linalg.norm(inc[:, 3]) / np.linalg.norm(f)
        assert lo <= ratio <= hi, ratio
        assert not inc[:, 2].any()
        tend = np.stack([z, z, z, f, z, z, z, z], axis=1)
        inc = S.euler_increment(G, tend, 0.5)
        assert np.array_equal(inc[:, 1], 0.5 * f) and not inc[:, [0, 2, 3]].any()


def test_jump_and_a_plain_step_damp_every_lattice_velocity_mode(S, orc):
    """Stability of a surrogate cycle with an untrained network: for shear and compressive plane
    waves of every lattice wavenumber along x and the diagonal, the acceleration of the method's
    momentum equation (Eq. 23, zeta = 0, uniform density) gives the jump's velocity factor
    1 + <du, u> / <u, u>; times the modified-Euler factor 1 - z + z^2 / 2 of the plain step that
    follows (z = dt lambda), it stays inside the unit circle at dt = 0.125 h^2 / nu and k = 8."""
    nx, k = 24, 8
    dx = 1.0 / nx
    h = 1.3 * dx
    g = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel(), Y.ravel()
    n = x.size
    dt = 0.125 * h * h
    P = orc.make_params(h=h, dt=dt, eta=1.0, zeta=0.0, c0_min=0.5)
    nb = orc.Nbrs(x, y, 1.0, h, "cells")
    _, V = orc.volumes(nb)
    Bc = orc.correction(nb, V)[:3]
    G = S.Graph(x, y, 1.0, h, nb.rowptr, nb.cols[:nb.rowptr[-1]])
    one, z0 = np.ones(n), np.zeros(n)
    worst = 0.0
    for diag in (False, True):
        for m in range(1, nx // 2 + 1):
            f = np.cos(2 * np.pi * m * (x + y if diag else x))
            for ux, uy in ((f, f) if diag else (f, z0), (f, -f) if diag else (z0, f)):
                ax, ay, _, _ = orc.momentum_paper(P, nb, V, Bc, one, z0, ux, uy, z0, z0)
                uu = np.dot(ux, ux) + np.dot(uy, uy)
                zr = -dt * (np.dot(ax, ux) + np.dot(ay, uy)) / uu
                tend = np.stack([ax, ay, z0, z0, z0, z0, z0, z0], axis=1)
                inc = S.euler_increment(G, tend, k * dt)
                jump = 1.0 + (np.dot(inc[:, 2], ux) + np.dot(inc[:, 3], uy)) / uu
                worst = max(worst, abs(jump * (1.0 - zr + 0.5 * zr * zr)))
    assert worst < 0.97, worst


def test_recorded_q_rate_is_the_step_increment_over_dt(orc, S):
    """The oracle's recorded Q rate (Eq. 24's m) equals (Q^{n+1} - Q^n) / dt of the step, and the
    tendencies assembled from a record follow the velocity-gradient convention D_ab = du_a/dx_b."""
    ic = si.jittered_lattice(16, seed=1)
    P = orc.make_params(h=1.3 / 16)
    st = {k: ic[k] for k in ("x", "y", "ux", "uy", "q11", "q12", "rho")}
    out, rec = orc.step(P, st, 1, record=True)
    for c in ("11", "12"):
        m = (out["q" + c] - ic["q" + c]) / P.dt
        assert np.abs(rec["qrate" + c] - m).max() <= 1e-11 * np.abs(m).max()
    tnd = S.tendencies_from_record(rec)
    gu = rec["gradu"].reshape(-1, 4)
    assert np.array_equal(tnd[:, 6], gu[:, 0] + gu[:, 3]) and np.array_equal(tnd[:, 7], gu[:, 2] - gu[:, 1])


def test_first_adam_step_moves_by_the_learning_rate(S):
    """Step 1: m = (1 - b1) g, v = (1 - b2) g^2, bias correction gives mh = g, vh = g^2, so every
    parameter moves by lr g / (|g| + eps) = lr sign(g) (up to eps)."""
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -1e-3, 4.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    S.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p["a"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=0, atol=1e-7)
