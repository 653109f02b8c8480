"""Pins of the three-dimensional FP64 oracle against closed forms, exact reproduction properties of
the corrected SPH operators, symmetry and the viscous decay rate of plane waves (the 2(d + 2) = 10
factor of the 3D viscous term)."""
import numpy as np
import pytest

import sph_inputs as si


@pytest.fixture(scope="module")
def O():
    from oracle import oracle3d

    return oracle3d


def test_kernel_normalisation_in_3d(O):
    """Eq. (18)'s 3D constant a_d = 3 / (359 pi h^3) as printed: since int_0^3 w(b) b^2 db = 30
    exactly (the polynomial's moment), 4 pi int W r^2 dr = 360/359, not 1 -- the exact constant is
    1 / (120 pi h^3).  The step does not depend on it: V = 1 / sum W scales as 1 / a_d and every
    sum weighs V_j W_ij or V_j grad W_ij.  W' is the derivative of W."""
    h = 0.37
    r = np.linspace(0.0, 3.0 * h, 200001)
    w = O.W(r / h, h)
    assert O.kernel_ad(h) == pytest.approx(3.0 / (359.0 * np.pi * h ** 3), rel=1e-15)
    assert 4.0 * np.pi * np.trapezoid(w * r * r, r) == pytest.approx(360.0 / 359.0, rel=1e-8)
    b = np.array([0.3, 1.4, 2.6])
    fd = (O.W(b + 1e-6, h) - O.W(b - 1e-6, h)) / 2e-6
    assert np.allclose(O.dWdb(b, h), fd, rtol=1e-7)


def test_neighbours_match_brute_force(O):
    ic = si.jittered_lattice3(7, seed=2, jitter=0.3)
    h = 1.3 / 7 * 0.8   # cells of side >= 3h: the grid path (7 // 2.4 = 2 < 3 -> brute); use a larger box
    nb = O.Nbrs3(ic["x"], ic["y"], ic["z"], 1.0, h)
    d = [ic[c][:, None] - ic[c][None, :] for c in ("x", "y", "z")]
    r2 = sum((v - np.round(v)) ** 2 for v in d)
    want = (r2 < 9 * h * h) & ~np.eye(ic["n"], dtype=bool)
    got = np.zeros_like(want)
    for i in range(ic["n"]):
        got[i, nb.cols[nb.rowptr[i]:nb.rowptr[i + 1]]] = True
    assert np.array_equal(got, want)
    ic = si.jittered_lattice3(12, seed=3, jitter=0.3)   # 12 / (3 * 1.3) -> 3 cells: the grid path
    h = 1.3 / 12
    nb = O.Nbrs3(ic["x"], ic["y"], ic["z"], 1.0, h)
    d = [ic[c][:, None] - ic[c][None, :] for c in ("x", "y", "z")]
    r2 = sum((v - np.round(v)) ** 2 for v in d)
    want = (r2 < 9 * h * h) & ~np.eye(ic["n"], dtype=bool)
    assert nb.rowptr[-1] == want.sum()
    for i in range(0, ic["n"], 97):
        assert np.array_equal(np.sort(nb.cols[nb.rowptr[i]:nb.rowptr[i + 1]]), np.nonzero(want[i])[0])


def _interior(ic, margin):
    return np.all([(ic[c] > margin) & (ic[c] < 1.0 - margin) for c in ("x", "y", "z")], axis=0)


def test_corrected_gradient_is_exact_for_linear_fields(O):
    """Eq. (20) with B = alpha^-1 (Eq. 22) reproduces a linear field's gradient on any particle set
    (away from the periodic seam, where a linear field is not periodic)."""
    ic = si.jittered_lattice3(12, seed=4, jitter=0.25)
    h = 1.3 / 12
    nb = O.Nbrs3(ic["x"], ic["y"], ic["z"], 1.0, h)
    _, V = O.volumes(nb)
    Bm, bad = O.correction(nb, V)
    assert bad == 0
    f = 2.0 * ic["x"] - 1.0 * ic["y"] + 3.0 * ic["z"]
    g = O.gradient(nb, V, Bm, f)
    m = _interior(ic, 3.2 * h)
    assert m.sum() > 50
    assert np.abs(g[m] - [2.0, -1.0, 3.0]).max() < 1e-11


def test_corrected_laplacian_is_exact_for_quadratics_on_a_lattice(O):
    """On a perfect cubic lattice (2nd-rank moments isotropic, odd moments zero) the scalar corrected
    Laplacian 2 sum V (f_i - f_j) (d . B grad W) / r^2 returns lap f of a quadratic exactly; the
    factor 2 is the one that does (a factor 8/5 would give 0.8 lap f)."""
    ic = si.jittered_lattice3(12, seed=5, jitter=0.0)
    h = 1.3 / 12
    nb = O.Nbrs3(ic["x"], ic["y"], ic["z"], 1.0, h)
    _, V = O.volumes(nb)
    Bm, _ = O.correction(nb, V)
    x, y, z = ic["x"], ic["y"], ic["z"]
    f = x * x + 2.0 * y * y + 3.0 * z * z + x * y - 2.0 * y * z + 0.5 * x
    lap = O.laplacian(nb, V, Bm, f)
    m = _interior(ic, 3.2 * h)
    assert np.abs(lap[m] - 12.0).max() < 1e-8


def test_q_rate_closed_forms(O):
    """Bulk molecular field of a uniaxial Q = s (nn - I/3): H = (-A + B s/3 - 2 C s^2 / 3) Q (Eq. 7 in
    3D), so m = Gamma H; a pure rotation D = Omega gives S = Omega Q - Q Omega (Eq. 2)."""
    P = O.make_params(A=0.3, B=0.7, C=1.1, K=0.0, Gamma=0.25, lam=0.6)
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    s = 0.6
    Q = s * (np.outer(n, n) - np.eye(3) / 3)
    q5 = np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]])
    m, tr = O.q_rate(P, q5, np.zeros((3, 3)), np.zeros(5))
    want = 0.25 * (-0.3 + 0.7 * s / 3 - 2 * 1.1 * s * s / 3) * q5
    assert np.allclose(m, want, rtol=1e-13, atol=1e-15) and abs(tr) < 1e-14
    P = O.make_params(A=0.0, B=0.0, C=0.0, K=0.0, Gamma=0.25, lam=0.6)
    w = np.array([0.2, -0.7, 0.4])
    Om = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    m, _ = O.q_rate(P, q5, Om, np.zeros(5))
    S = Om @ Q - Q @ Om
    assert np.allclose(m, [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2]], rtol=1e-12, atol=1e-15)
    # a general gradient: the rate is symmetric and traceless by construction, and the K term adds
    # Gamma K lap Q
    D = np.array([[0.1, 0.4, -0.2], [0.3, -0.3, 0.5], [-0.6, 0.2, 0.2]])
    P1 = O.make_params(A=0.3, B=0.7, C=1.1, K=0.0, Gamma=0.25, lam=0.6)
    P2 = O.make_params(A=0.3, B=0.7, C=1.1, K=0.05, Gamma=0.25, lam=0.6)
    lq = np.array([1.0, -2.0, 0.5, 0.3, 0.7])
    m1, _ = O.q_rate(P1, q5, D, lq)
    m2, _ = O.q_rate(P2, q5, D, lq)
    assert np.allclose(m2 - m1, 0.25 * 0.05 * lq, rtol=1e-12, atol=1e-15)




@pytest.mark.parametrize("kind, rate", [("shear", 1.0), ("compressive", 3.0)])
def test_viscous_term_decays_plane_waves_at_nu_k2(O, kind, rate):
    """On a cubic lattice, the viscous term of Eq. (23) with 2 (d + 2) nu = 10 nu gives a shear wave
    u_x = e sin(k z) the rate -nu k^2 and a compressive wave u_x = e sin(k x) the rate -3 nu k^2
    (lap u + 2 grad div u), to the discretisation error of the wave (k h = 0.34 here: about 4 %)."""
    nx = 24
    ic = si.jittered_lattice3(nx, seed=0, jitter=0.0)
    h = 1.3 / nx
    nb = O.Nbrs3(ic["x"], ic["y"], ic["z"], 1.0, h)
    _, V = O.volumes(nb)
    Bm, _ = O.correction(nb, V)
    n = ic["n"]
    k = 2 * np.pi
    u = np.zeros((n, 3))
    u[:, 0] = 1e-3 * np.sin(k * (ic["z"] if kind == "shear" else ic["x"]))
    P = O.make_params(eta=0.7, zeta=0.0, rho0=1.0)
    a, _ = O.momentum(P, nb, V, Bm, np.ones(n), np.zeros(n), u, np.zeros((n, 5)))
    got = -np.dot(a[:, 0], u[:, 0]) / np.dot(u[:, 0], u[:, 0])
    assert got == pytest.approx(rate * 0.7 * k * k, rel=0.06)   # 8 nu instead of 10 nu: -20 %
    assert np.abs(a[:, 1:]).max() < 1e-9 * np.abs(a[:, 0]).max()


def test_uniform_state_relaxes_only_by_the_bulk_term(O):
    """Uniform Q, rest and uniform density: every pair difference vanishes, so one step moves Q by
    dt Gamma H_bulk(Q) and nothing else moves."""
    ic = si.jittered_lattice3(10, seed=6, jitter=0.2)
    n = ic["n"]
    q5 = np.array([0.2, -0.1, 0.05, -0.15, 0.08])
    P = O.make_params(h=1.3 / 10, dt=1e-4, A=0.1, B=0.3, C=1.0)
    st = {"x": ic["x"], "y": ic["y"], "z": ic["z"], "u": np.zeros((n, 3)), "q": np.tile(q5, (n, 1)),
          "rho": np.ones(n)}
    out, rec = O.step(P, st, 1, record=True)
    m, _ = O.q_rate(P, q5, np.zeros((3, 3)), np.zeros(5))
    assert np.abs(out["q"] - (q5 + 1e-4 * m)).max() < 1e-12
    assert np.abs(out["u"]).max() < 1e-12 and np.abs(out["rho"] - 1).max() < 1e-12
    assert np.abs(out["x"] - ic["x"]).max() < 1e-15
    assert rec["status"] == 0 and rec["nnbr"].min() > 200


def test_step_is_equivariant_under_a_cyclic_axis_permutation(O):
    """Relabelling the axes x -> y -> z -> x (a proper rotation that maps the periodic box to itself)
    commutes with a whole step: positions, u and a rotate as vectors and Q as a tensor."""
    ic = si.jittered_lattice3(8, seed=7, jitter=0.3, u_scale=0.2)
    n = ic["n"]
    P = O.make_params(h=1.3 / 8, dt=2e-4, A=0.1, B=0.2, C=1.0, zeta=0.3, c0_min=0.5)
    st = {"x": ic["x"], "y": ic["y"], "z": ic["z"], "u": ic["u"], "q": ic["q"], "rho": np.ones(n)}
    R = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], dtype=float)   # (x, y, z) -> (z, x, y)

    def rot(s):
        r = np.stack([s["x"], s["y"], s["z"]], axis=1) @ R.T
        q = s["q"]
        Q = np.zeros((n, 3, 3))
        Q[:, 0, 0], Q[:, 0, 1], Q[:, 0, 2], Q[:, 1, 1], Q[:, 1, 2] = q.T
        Q[:, 1, 0], Q[:, 2, 0], Q[:, 2, 1] = Q[:, 0, 1], Q[:, 0, 2], Q[:, 1, 2]
        Q[:, 2, 2] = -Q[:, 0, 0] - Q[:, 1, 1]
        Qr = R @ Q @ R.T
        out = {"x": r[:, 0], "y": r[:, 1], "z": r[:, 2], "u": s["u"] @ R.T, "rho": s["rho"],
               "q": np.stack([Qr[:, 0, 0], Qr[:, 0, 1], Qr[:, 0, 2], Qr[:, 1, 1], Qr[:, 1, 2]], axis=1)}
        if "a" in s:
            out["a"] = s["a"] @ R.T
        return out

    a1, _ = O.step(P, rot(st), 2)
    a2 = rot(O.step(P, st, 2)[0])
    for k in ("x", "y", "z", "u", "q", "rho", "a"):
        assert np.abs(np.asarray(a1[k]) - np.asarray(a2[k])).max() < 1e-11, k
