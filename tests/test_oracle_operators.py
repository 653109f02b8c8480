"""Pins of the oracle's SPH operators (§3) against exact results of the mathematics.

Each pin is chosen so that a plausible slip in the oracle fails it:
* corrected gradient (Eq. 20 with Eq. 22): exact for every linear field on any particle set
  (a transposed B, a wrong sign of r_ji or a dropped V_j breaks it);
* corrected Laplacian (Eq. 21, scalar reading): exact for quadratics on a point-symmetric
  neighbourhood with isotropic alpha, i.e. on square and triangular lattices (a factor other than
  2, or the sign of (f_i - f_j), breaks it);
* momentum (Eq. 23): the symmetric pressure form gives -grad p / rho for a linear pressure on a
  lattice; the "8 nu" viscous form gives nu (lap u + 2 grad div u) for quadratic u where the
  4th moments are isotropic (triangular lattice); the active term is -zeta div Q / rho exactly for
  linear Q on any particle set;
* continuity (Eq. 25): k = -rho div u exactly for a linear velocity field;
* density filter (Eq. 28): constants and, on a lattice, linear fields are unchanged;
* APD (Eq. 29): zero on a perfect lattice; pushes a displaced particle away from its crowded side;
* EoS (Eq. 26): p(rho0) = 0, dp/drho = c0^2 at rho0, the closed form for gamma = 1.
Fields that are polynomials of position are not periodic, so these checks use particles further
than the support (or twice the support where neighbour volumes matter) from the box faces.
"""
import math

import numpy as np
import pytest

import sph_inputs as si


def _setup(orc, ic, h, mode="brute"):
    nb = orc.Nbrs(ic["x"], ic["y"], 1.0, h, mode)
    sumW, V = orc.volumes(nb)
    b11, b12, b22, bad = orc.correction(nb, V)
    assert bad == 0
    return nb, V, (b11, b12, b22)


def _interior(ic, margin):
    x, y = ic["x"], ic["y"]
    return (x > margin) & (x < 1 - margin) & (y > margin) & (y < 1 - margin)


@pytest.fixture(scope="module")
def jittered(orc):
    ic = si.jittered_lattice(48, seed=4, jitter=0.2)
    h = 1.3 * ic["dx"]
    return ic, h, _setup(orc, ic, h)


@pytest.fixture(scope="module")
def square(orc):
    ic = si.jittered_lattice(48, seed=0, jitter=0.0)
    h = 1.3 * ic["dx"]
    return ic, h, _setup(orc, ic, h)


@pytest.fixture(scope="module")
def hexa(orc):
    ic = si.hex_lattice(1.0 / 40.0, origin=(0.013, 0.007))
    h = 1.3 / 40.0
    return ic, h, _setup(orc, ic, h)


def test_gradient_of_linear_field_is_exact(orc, jittered):
    ic, h, (nb, V, B) = jittered
    m = _interior(ic, 3 * h + 1e-3)
    for gx, gy in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.9)):
        f = 3.0 + gx * ic["x"] + gy * ic["y"]
        g = orc.gradient(nb, V, B, f)
        assert np.abs(g[m, 0] - gx).max() < 1e-12
        assert np.abs(g[m, 1] - gy).max() < 1e-12


def test_gradient_and_laplacian_of_constant_vanish(orc, jittered):
    ic, h, (nb, V, B) = jittered
    f = np.full(nb.n, 2.5)
    assert np.abs(orc.gradient(nb, V, B, f)).max() == 0.0
    assert np.abs(orc.laplacian(nb, V, B, f)).max() == 0.0


@pytest.mark.parametrize("lattice", ["square", "hexa"])
def test_laplacian_of_quadratics_is_exact(orc, lattice, square, hexa):
    ic, h, (nb, V, B) = square if lattice == "square" else hexa
    m = _interior(ic, 6 * h + 1e-3)
    assert m.sum() > 100
    x, y = ic["x"], ic["y"]
    for f, lap in ((x * x, 2.0), (y * y, 2.0), (x * y, 0.0), (x * x + y * y, 4.0),
                   (3 * x * x - 2 * x * y + 0.5 * y * y + x, 7.0)):
        out = orc.laplacian(nb, V, B, f)
        assert np.abs(out[m] - lap).max() < 1e-9


def test_laplacian_converges_on_jittered_lattice(orc):
    # no exactness on an irregular set, but the error of lap(x^2 + y^2) shrinks as the jitter does
    errs = []
    for j in (0.2, 0.1, 0.05):
        ic = si.jittered_lattice(48, seed=4, jitter=j)
        h = 1.3 * ic["dx"]
        nb, V, B = _setup(orc, ic, h)
        m = _interior(ic, 3 * h + 1e-3)
        out = orc.laplacian(nb, V, B, ic["x"] ** 2 + ic["y"] ** 2)
        errs.append(np.abs(out[m] - 4.0).max())
    assert errs[0] > errs[1] > errs[2]


def test_continuity_linear_velocity(orc, jittered):
    ic, h, (nb, V, B) = jittered
    m = _interior(ic, 3 * h + 1e-3)
    eps, shear = 0.3, 0.8
    ux = eps * ic["x"] + shear * ic["y"]
    uy = eps * ic["y"] - 0.1 * ic["x"]
    rho = 1.0 + 0.01 * ic["x"]
    k = orc.continuity(nb, V, B, ux, uy, rho)
    assert np.abs(k[m] - (-rho[m] * 2 * eps)).max() < 1e-12


def test_density_filter_constant_and_linear(orc, square):
    ic, h, (nb, V, B) = square
    rho = np.full(nb.n, 1.003)
    assert np.abs(orc.density_filter(nb, rho) - 1.003).max() < 1e-15
    m = _interior(ic, 3 * h + 1e-3)
    rho = 1.0 + 0.01 * ic["x"] - 0.02 * ic["y"]
    out = orc.density_filter(nb, rho)
    assert np.abs(out[m] - rho[m]).max() < 1e-14
    # beta = 0 switches the filter off; beta = 1 is Shepard's interpolation
    rnd = 1.0 + 1e-3 * si.uniform53(3, nb.n)
    assert np.array_equal(orc.density_filter(nb, rnd, beta=0.0), rnd)
    sh = orc.density_filter(nb, rnd, beta=1.0)
    assert np.abs(sh).min() > 0.999 and np.std(sh) < np.std(rnd)


def _params(orc, **kw):
    base = dict(zeta=0.0, eta=0.0, Gamma=0.0, K=0.0, A=0.0, C=0.0)
    base.update(kw)
    return orc.make_params(**base)


def test_pressure_term_gives_minus_grad_p_over_rho(orc, square):
    ic, h, (nb, V, B) = square
    m = _interior(ic, 3 * h + 1e-3)
    rho = np.full(nb.n, 1.2)
    gx, gy = 0.4, -1.3
    p = 2.0 + gx * ic["x"] + gy * ic["y"]
    z = np.zeros(nb.n)
    ax, ay, _, _ = orc.momentum_paper(_params(orc, h=h), nb, V, B, rho, p, z, z, z, z)
    assert np.abs(ax[m] + gx / 1.2).max() < 1e-11
    assert np.abs(ay[m] + gy / 1.2).max() < 1e-11


def test_viscous_term_on_triangular_lattice(orc, hexa):
    ic, h, (nb, V, B) = hexa
    m = _interior(ic, 6 * h + 1e-3)
    x, y = ic["x"], ic["y"]
    nu, rho0, rho = 0.6, 1.0, 1.0
    z = np.zeros(nb.n)
    P = _params(orc, h=h, eta=nu * rho0, rho0=rho0)
    # 8 nu sum V_j (u_ij . d)/r^2 B grad W  ->  nu (lap u + 2 grad div u) for quadratic u
    cases = [((y * y, z), (2.0, 0.0)),        # lap u = (2,0), div u = 0
             ((x * x, z), (6.0, 0.0)),        # lap u = (2,0), grad div u = (2,0)
             ((x * y, z), (0.0, 2.0)),        # lap u = 0, grad div u = (0,1)
             ((z, x * y), (2.0, 0.0))]        # lap u = 0, grad div u = (1,0)
    for (ux, uy), (ex, ey) in cases:
        ax, ay, _, _ = orc.momentum_paper(P, nb, V, B, np.full(nb.n, rho), z, ux, uy, z, z)
        assert np.abs(ax[m] - nu * ex).max() < 1e-8
        assert np.abs(ay[m] - nu * ey).max() < 1e-8


def test_active_term_is_minus_zeta_div_q(orc, jittered):
    ic, h, (nb, V, B) = jittered
    m = _interior(ic, 3 * h + 1e-3)
    zeta, rho = 0.07, 1.1
    a, b, c, d = 0.3, -0.8, 1.7, 0.25
    q11 = a * ic["x"] + b * ic["y"]
    q12 = c * ic["x"] + d * ic["y"]
    z = np.zeros(nb.n)
    ax, ay, dqx, dqy = orc.momentum_paper(_params(orc, h=h, zeta=zeta), nb, V, B,
                                          np.full(nb.n, rho), z, z, z, q11, q12)
    # div Q = (dQ11/dx + dQ12/dy, dQ21/dx + dQ22/dy) with Q21 = Q12, Q22 = -Q11
    assert np.abs(dqx[m] - (a + d)).max() < 1e-11
    assert np.abs(dqy[m] - (c - b)).max() < 1e-11
    assert np.abs(ax[m] + zeta / rho * (a + d)).max() < 1e-11
    assert np.abs(ay[m] + zeta / rho * (c - b)).max() < 1e-11


def test_apd_vanishes_on_perfect_lattice(orc, square):
    ic, h, (nb, V, B) = square
    rnd = si.uniform53(8, 2 * nb.n).reshape(2, nb.n) - 0.5
    dx, dy = orc.apd(nb, rnd[0], rnd[1], 1e-4)
    scale = 1e-4 * np.abs(rnd).max()
    assert np.abs(dx).max() < 1e-12 * scale and np.abs(dy).max() < 1e-12 * scale
    # uniform velocity: u_v = 0 everywhere, on any particle set
    ic2 = si.jittered_lattice(32, seed=2, jitter=0.3)
    nb2 = orc.Nbrs(ic2["x"], ic2["y"], 1.0, 1.3 * ic2["dx"])
    dx, dy = orc.apd(nb2, np.full(nb2.n, 0.3), np.full(nb2.n, -0.2), 1e-3)
    assert np.abs(dx).max() == 0.0 and np.abs(dy).max() == 0.0


def test_apd_pushes_away_from_crowded_side(orc):
    ic = si.jittered_lattice(32, seed=0, jitter=0.0)
    x, y = ic["x"].copy(), ic["y"].copy()
    i = 16 * 32 + 16
    x[i] += 0.3 * ic["dx"]            # towards its right-hand neighbour
    h = 1.3 * ic["dx"]
    nb = orc.Nbrs(x, y, 1.0, h)
    ux = np.zeros(nb.n)
    ux[i] = 1.0                       # a velocity variance so u_v > 0
    dx, dy = orc.apd(nb, ux, np.zeros(nb.n), 1e-3)
    assert dx[i] < 0.0 and abs(dy[i]) < 1e-12 * abs(dx[i])


def test_equation_of_state(orc):
    rho0, c0 = 1.0, 0.3
    assert orc.eos([rho0], rho0, c0)[0] == 0.0
    d = 1e-7
    slope = (orc.eos([rho0 + d], rho0, c0)[0] - orc.eos([rho0 - d], rho0, c0)[0]) / (2 * d)
    assert slope == pytest.approx(c0 * c0, rel=1e-8)
    rho = np.array([0.9, 1.0, 1.1])
    assert np.allclose(orc.eos(rho, rho0, c0, 1.0), c0 * c0 * (rho - rho0), rtol=0, atol=1e-16)
    assert np.all(np.diff(orc.eos(np.linspace(0.95, 1.05, 11), rho0, c0)) > 0)


def test_correction_tensor_isotropic_on_lattices(orc, square, hexa):
    for ic, h, (nb, V, B) in (square, hexa):
        m = _interior(ic, 6 * h + 1e-3)
        b11, b12, b22 = B
        assert np.abs(b11[m] - b22[m]).max() < 1e-12 * np.abs(b11[m]).max()
        assert np.abs(b12[m]).max() < 1e-12 * np.abs(b11[m]).max()


# ---------------------------------------------------------------------------------------------
# APD magnitude (Eq. 29): delta r_i = dt u_v r0^2 sum_j d_ij / |d_ij|^3 with
# u_v = |sum_j (u_i - u_j) W_ij| / sum_j W_ij (self term in the denominator) and r0 the mean
# neighbour distance.  Pinned by closed forms of two- and three-particle configurations and by the
# scaling laws the formula fixes.
# ---------------------------------------------------------------------------------------------

def _apd_of(orc, pts, u, h, dt, L=1.0):
    pts = np.asarray(pts, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    nb = orc.Nbrs(pts[:, 0], pts[:, 1], L, h)
    return np.stack(orc.apd(nb, u[:, 0], u[:, 1], dt), axis=1)


@pytest.mark.parametrize("b", [0.3, 1.2, 2.1, 2.9])
def test_apd_two_particles_closed_form(orc, b):
    # particle 1 at distance r = b h from particle 0, along a direction e; only particle 1 moves.
    # For particle 0: u_v = |u_1| W / (W(0) + W), r0 = r, sum d/r^3 = -e / r^2, so
    # delta r_0 = -dt |u_1| W / (W(0) + W) e; particle 1 gets the opposite displacement.
    h, dt = 0.04, 3e-3
    W0, Wr = orc.W([0.0, b], h)
    for e in ((1.0, 0.0), (0.6, -0.8)):
        e = np.array(e)
        p0 = np.array([0.31, 0.57])
        pts = [p0, p0 + b * h * e]
        u = [[0.0, 0.0], [0.7, -2.4]]          # |u_1| = 2.5
        got = _apd_of(orc, pts, u, h, dt)
        mag = dt * 2.5 * Wr / (W0 + Wr)
        assert np.abs(got[0] + mag * e).max() <= 1e-14 * mag
        assert np.abs(got[1] - mag * e).max() <= 1e-14 * mag


def test_apd_two_particles_across_the_periodic_face(orc):
    # the pair vector is the minimum image: particle 1 sits just across x = 0 from particle 0
    h, dt, b = 0.04, 3e-3, 1.7
    W0, Wr = orc.W([0.0, b], h)
    pts = [[0.01, 0.5], [1.0 + 0.01 - b * h, 0.5]]    # x_0 - x_1 = +b h by minimum image
    got = _apd_of(orc, pts, [[0.0, 0.0], [0.0, 1.5]], h, dt)
    mag = dt * 1.5 * Wr / (W0 + Wr)
    assert got[0, 0] == pytest.approx(mag, rel=1e-12) and abs(got[0, 1]) <= 1e-14 * mag
    assert got[1, 0] == pytest.approx(-mag, rel=1e-12)


def test_apd_three_particles_closed_form(orc):
    # particle 0 with neighbours 1 (at +r1 along x) and 2 (at +r2 along y), r1^2 + r2^2 > (3h)^2 so
    # 1 and 2 do not see each other; only particle 1 moves, with speed U along x.
    #   particle 0: u_v = U W(r1) / (W(0) + W(r1) + W(r2)), r0 = (r1 + r2)/2,
    #               delta r_0 = dt u_v r0^2 (-1/r1^2, -1/r2^2)
    #   particle 1: delta r_1 = dt U W(r1) / (W(0) + W(r1)) (1, 0);  particle 2: 0
    h, dt, U = 0.05, 2e-3, 0.9
    b1, b2 = 2.5, 2.0
    r1, r2 = b1 * h, b2 * h
    W0, W1, W2 = orc.W([0.0, b1, b2], h)
    pts = [[0.5, 0.5], [0.5 + r1, 0.5], [0.5, 0.5 + r2]]
    got = _apd_of(orc, pts, [[0.0, 0.0], [U, 0.0], [0.0, 0.0]], h, dt)
    uv = U * W1 / (W0 + W1 + W2)
    r0 = 0.5 * (r1 + r2)
    want0 = dt * uv * r0 * r0 * np.array([-1.0 / r1**2, -1.0 / r2**2])
    want1 = dt * U * W1 / (W0 + W1) * np.array([1.0, 0.0])
    assert np.abs(got[0] - want0).max() <= 1e-14 * np.abs(want0).max()
    assert np.abs(got[1] - want1).max() <= 1e-14 * np.abs(want1).max()
    assert np.abs(got[2]).max() == 0.0


def test_apd_scaling_laws(orc):
    # delta r is linear in dt and in the amplitude of the velocity differences (even in its sign),
    # and unchanged when positions, h and L scale by s with u fixed (r0^2 ~ s^2, sum d/r^3 ~ s^-2,
    # u_v ~ s^0 since W scales out of the ratio).  A dropped square on r0, a d/r^2 for d/r^3, a u_v
    # without its division by sum W, or a missing dt breaks one of these.
    ic = si.jittered_lattice(24, seed=9, jitter=0.3)
    h = 1.3 * ic["dx"]
    r = si.uniform53(31, 2 * ic["n"]).reshape(2, ic["n"]) - 0.5
    nb = orc.Nbrs(ic["x"], ic["y"], 1.0, h)
    base = np.stack(orc.apd(nb, r[0], r[1], 1e-3), axis=1)
    scale = np.abs(base).max()
    assert scale > 0.0
    twice_dt = np.stack(orc.apd(nb, r[0], r[1], 2e-3), axis=1)
    assert np.abs(twice_dt - 2.0 * base).max() <= 1e-13 * scale
    for a in (3.0, -2.0):
        amp = np.stack(orc.apd(nb, a * r[0] + 0.4, a * r[1] - 0.1, 1e-3), axis=1)   # offsets cancel
        assert np.abs(amp - abs(a) * base).max() <= 1e-12 * abs(a) * scale
    s = 2.5
    nbs = orc.Nbrs(s * ic["x"], s * ic["y"], s, s * h)
    assert np.array_equal(nbs.rowptr, nb.rowptr) and np.array_equal(nbs.cols, nb.cols)
    scaled = np.stack(orc.apd(nbs, r[0], r[1], 1e-3), axis=1)
    assert np.abs(scaled - base).max() <= 1e-12 * scale
