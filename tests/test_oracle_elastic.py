"""Pins of the oracle's elastic stress (Eq. 12 without -p I; off by default, as the paper drops it).

Pi_el = 2 lambda M (Q:H) - lambda (H M + M H) with M = Q + c I.  In 2D, with Q = [[a, b], [b, -a]],
q^2 = a^2 + b^2 and Q^2 = q^2 I, the tensor algebra gives by hand:
  * H = h Q:      Pi = lambda h [(4 q^2 - 2c) Q + (4 c q^2 - 2 q^2) I]
  * H = h0 I:     Pi = -2 lambda h0 (Q + c I)            (Q:I = 0)
The force is (1/rho) div Pi through the corrected divergence (paper mode) or the pair-antisymmetric
form (conservative mode).
"""
import math

import numpy as np
import pytest

import sph_inputs as si


@pytest.mark.parametrize("c_shift", [1.0 / 3.0, 0.5])
def test_closed_forms(orc, c_shift):
    lam = 0.7
    P = orc.make_params(lam=lam, c_shift=c_shift)
    rng = si.uniform53(31, 24).reshape(8, 3) - 0.5
    I = np.eye(2)
    for a, b, h in rng:
        Q = np.array([[a, b], [b, -a]])
        q2 = a * a + b * b
        got = orc.elastic_stress(P, a, b, h * Q)
        want = lam * h * ((4 * q2 - 2 * c_shift) * Q + (4 * c_shift * q2 - 2 * q2) * I)
        assert np.abs(got - want).max() < 1e-15
        got = orc.elastic_stress(P, a, b, h * I)
        want = -2 * lam * h * (Q + c_shift * I)
        assert np.abs(got - want).max() < 1e-15
        # general symmetric H: Pi is symmetric
        Hs = np.array([[h, 0.3], [0.3, -0.2]])
        got = orc.elastic_stress(P, a, b, Hs)
        assert abs(got[0, 1] - got[1, 0]) < 1e-15


def test_force_is_divergence_of_linear_stress(orc):
    ic = si.jittered_lattice(40, seed=2, jitter=0.2)
    h = 1.3 * ic["dx"]
    nb = orc.Nbrs(ic["x"], ic["y"], 1.0, h)
    _, V = orc.volumes(nb)
    B = orc.correction(nb, V)[:3]
    x, y = ic["x"], ic["y"]
    m = (np.abs(x - 0.5) < 0.5 - 3 * h - 1e-3) & (np.abs(y - 0.5) < 0.5 - 3 * h - 1e-3)
    # Pi = [[p11, p12], [p12, p22]] linear in position
    p11 = 0.2 + 0.5 * x - 0.3 * y
    p12 = -0.1 + 0.7 * x + 0.4 * y
    p22 = 0.05 - 0.6 * x + 0.9 * y
    pel = np.stack([p11, p12, p22], axis=1)
    z = np.zeros(nb.n)
    rho = 1.25
    P = orc.make_params(h=h, zeta=0.0, eta=0.0, elastic=1)
    ax, ay, _, _ = orc.momentum_paper(P, nb, V, B, np.full(nb.n, rho), z, z, z, z, z, pel=pel)
    # div Pi = (d_x p11 + d_y p12, d_x p12 + d_y p22) = (0.5 + 0.4, 0.7 + 0.9)
    assert np.abs(ax[m] - 0.9 / rho).max() < 1e-11
    assert np.abs(ay[m] - 1.6 / rho).max() < 1e-11
    P0 = orc.make_params(h=h, zeta=0.0, eta=0.0, elastic=0)
    ax0, _, _, _ = orc.momentum_paper(P0, nb, V, B, np.full(nb.n, rho), z, z, z, z, z, pel=pel)
    assert np.abs(ax0).max() == 0.0


def test_uniform_q_unaffected(orc):
    ic = si.jittered_lattice(24, seed=0, jitter=0.0)
    n = ic["n"]
    st = {k: ic[k] for k in ("x", "y", "ux", "uy", "rho")}
    st["q11"] = np.full(n, 0.5)
    st["q12"] = np.full(n, 0.3)
    h = 1.3 * ic["dx"]
    outs = [orc.step(orc.make_params(h=h, A=0.2, C=1.0, zeta=0.0, elastic=e), st, 5)[0] for e in (0, 1)]
    for k in ("q11", "q12", "ux", "uy"):
        assert np.abs(outs[0][k] - outs[1][k]).max() < 1e-15


def test_conservative_momentum_with_elastic_stress(orc):
    ic = si.jittered_lattice(24, seed=7)
    st = {k: ic[k] for k in ("x", "y", "q11", "q12", "rho")}
    r = si.uniform53(77, 2 * ic["n"]).reshape(2, ic["n"]) - 0.5
    st["ux"], st["uy"] = 1e-3 * r[0], 1e-3 * r[1]
    h = 1.3 * ic["dx"]
    P = orc.make_params(h=h, dt=5e-5, conservative=1, c0_min=0.5, zeta=0.05, eta=0.05, elastic=1,
                        K=0.04, A=0.1)
    out, _ = orc.step(P, st, 50)
    mass = 1.0 / ic["n"]
    p0 = mass * np.array([st["ux"].sum(), st["uy"].sum()])
    p1 = mass * np.array([out["ux"].sum(), out["uy"].sum()])
    scale = mass * (np.abs(out["ux"]).sum() + np.abs(out["uy"]).sum())
    assert np.abs(p1 - p0).max() <= 1e-12 * scale
    # and the elastic stress did act
    out0, _ = orc.step(orc.make_params(h=h, dt=5e-5, conservative=1, c0_min=0.5, zeta=0.05, eta=0.05,
                                       elastic=0, K=0.04, A=0.1), st, 50)
    assert np.abs(out["ux"] - out0["ux"]).max() > 1e-9
