"""Pins of the oracle's neighbour search.

* The definition (all j != i with |d_ij|^2 < (3h)^2, minimum image) against a literal transcription
  of the paper's periodic ghost layer (§3.1, Eq. 30) and against the paper's cell grid (§4).
* Counts on lattices against integer-lattice enumeration, and the paper's "about 45 neighbours"
  for h = 4/3 dx (§3, text under Eq. 18).
* Tiny hand-built cases across the periodic faces.
"""
import json
import math
import os

import numpy as np
import pytest

import sph_inputs as si

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kernel_constants.json")))


def _lattice_count(R_over_dx):
    """Integer lattice points (a, b) != 0 with a^2 + b^2 < R^2: exact neighbour count on a lattice."""
    m = int(math.ceil(R_over_dx)) + 1
    return sum(1 for a in range(-m, m + 1) for b in range(-m, m + 1)
               if (a, b) != (0, 0) and a * a + b * b < R_over_dx ** 2)


def _sets(rowptr, cols):
    return [tuple(cols[rowptr[i]:rowptr[i + 1]]) for i in range(len(rowptr) - 1)]


def test_jittered_lattice_count_is_44(orc):
    ic = si.jittered_lattice(64, seed=0)
    h = 1.3 * ic["dx"]
    rp, cols = orc.neighbors(ic["x"], ic["y"], 1.0, h, "brute")
    # R = 3.9 dx: the lattice shells up to 13 dx^2 are inside, the next (16 dx^2) lies 0.1 dx
    # outside, which the +-0.05 dx jitter of both particles cannot bridge.
    assert _lattice_count(3.9) == 44
    assert np.all(np.diff(rp) == 44)


def test_paper_smoothing_length_gives_about_45(orc):
    # h = 4/3 dx puts the support radius exactly on the 4 dx lattice shell.  Just inside it the
    # lattice count plus the particle itself is the paper's "about 45"; with jitter the 4 dx shell
    # is half in, half out.
    assert _lattice_count(4.0) + 1 == GOLD["neighbours_approx_paper"]
    ic = si.jittered_lattice(64, seed=3, jitter=0.0)
    h = GOLD["h_over_dx_paper"] * ic["dx"] * (1.0 - 1e-9)
    rp, _ = orc.neighbors(ic["x"], ic["y"], 1.0, h, "brute")
    assert np.all(np.diff(rp) + 1 == GOLD["neighbours_approx_paper"])
    ic = si.jittered_lattice(64, seed=3)
    rp, _ = orc.neighbors(ic["x"], ic["y"], 1.0, GOLD["h_over_dx_paper"] * ic["dx"], "brute")
    assert 45.0 <= np.diff(rp).mean() + 1 <= 47.0


@pytest.mark.parametrize("case", ["lattice", "random", "small_box", "three_cells", "edges"])
def test_brute_ghost_cells_agree(orc, case):
    if case == "lattice":
        ic = si.jittered_lattice(48, seed=1)
        h = 1.3 * ic["dx"]
    elif case == "random":
        ic = si.uniform_random(3001, seed=2)
        h = 1.3 / math.sqrt(3001)
    elif case == "small_box":
        ic = si.uniform_random(200, seed=5)
        h = 1.0 / 12.5  # 3h = 0.24: four cells across
    elif case == "three_cells":
        ic = si.uniform_random(150, seed=6)
        h = 1.0 / 9.5   # exactly three cells across
    else:
        # particles hugging every face and corner
        rng = si.uniform53(11, 800).reshape(400, 2)
        eps = 1e-3 * rng
        x = np.concatenate([eps[:100, 0], 1.0 - eps[100:200, 0], rng[200:, 0]])
        y = np.concatenate([rng[:200, 1], eps[200:300, 1], 1.0 - eps[300:, 1]])
        ic = {"x": si.wrap_positions(x, 1.0), "y": si.wrap_positions(y, 1.0)}
        h = 0.02
    b = orc.neighbors(ic["x"], ic["y"], 1.0, h, "brute")
    g = orc.neighbors(ic["x"], ic["y"], 1.0, h, "ghost")
    c = orc.neighbors(ic["x"], ic["y"], 1.0, h, "cells")
    assert np.array_equal(b[0], g[0]) and np.array_equal(b[1], g[1])
    assert np.array_equal(b[0], c[0]) and np.array_equal(b[1], c[1])


def test_lists_are_symmetric(orc):
    ic = si.uniform_random(2000, seed=9)
    rp, cols = orc.neighbors(ic["x"], ic["y"], 1.0, 0.012, "brute")
    pairs = {(i, int(j)) for i in range(2000) for j in cols[rp[i]:rp[i + 1]]}
    assert all((j, i) in pairs for (i, j) in pairs)
    assert all(i != j for (i, j) in pairs)


def test_tiny_periodic_cases(orc):
    h = 0.01  # support radius R = 0.03
    pts = [
        (0.005, 0.005),    # 0
        (0.985, 0.005),    # 1: 0.02 from 0 across the x face
        (0.995, 0.995),    # 2: sqrt(2)*0.01 from 0 across the corner, from 1 across the y face
        (0.0351, 0.005),   # 3: 0.0301 from 0 (outside)
        (0.005, 0.0349),   # 4: 0.0299 from 0 (inside); 0.036 from 1 (outside)
    ]
    x = np.array([p[0] for p in pts])
    y = np.array([p[1] for p in pts])
    rp, cols = orc.neighbors(x, y, 1.0, h, "brute")
    s = _sets(rp, cols)
    assert s[0] == (1, 2, 4)
    assert s[1] == (0, 2)
    assert s[2] == (0, 1)
    assert s[3] == ()
    assert s[4] == (0,)


def test_strict_cutoff(orc):
    # a pair whose FP64 |d|^2 equals (3h)^2 exactly is excluded (the test is strict)
    h = 0.125                     # 3h = 0.375, exactly representable
    x = np.array([0.125, 0.5])    # d = -0.375 exactly
    y = np.array([0.5, 0.5])
    rp, _ = orc.neighbors(x, y, 1.0, h, "brute")
    assert rp[1] - rp[0] == 0
    x[1] = np.nextafter(0.5, 0.0)  # one ulp closer: inside
    rp, _ = orc.neighbors(x, y, 1.0, h, "brute")
    assert rp[1] - rp[0] == 1



def test_periodic_copies_tile_the_box():
    """sph_inputs.periodic_copies: n = R^2 n0 particles in [0, L); copy t holds the pattern shrunk
    by R and shifted by (t mod R, t div R) L / R, exactly for R a power of two; the other arrays are
    repeated; every particle of every copy has the nearest-neighbour distance of its original in
    the pattern's own periodic box (the copies meet without overlap or gap)."""
    ic0 = si.jittered_lattice(8, seed=4, jitter=0.3)
    ic0["ux"] = si.uniform53(40, ic0["n"]) - 0.5
    R, n0 = 4, ic0["n"]
    big, pat = si.periodic_copies(ic0, R)
    assert big["n"] == R * R * n0 == len(big["x"]) == len(big["q11"])
    assert np.all((big["x"] >= 0) & (big["x"] < 1) & (big["y"] >= 0) & (big["y"] < 1))
    assert np.array_equal(pat["x"], ic0["x"] / R) and np.array_equal(pat["ux"], ic0["ux"])
    t = np.arange(R * R)
    assert np.array_equal(big["x"].reshape(R * R, n0), pat["x"][None, :] + ((t % R) / R)[:, None])
    assert np.array_equal(big["y"].reshape(R * R, n0), pat["y"][None, :] + ((t // R) / R)[:, None])
    assert np.array_equal(big["ux"].reshape(R * R, n0), np.broadcast_to(ic0["ux"], (R * R, n0)))

    def nearest(x, y, L):
        d = np.stack([x[:, None] - x[None, :], y[:, None] - y[None, :]], axis=-1)
        d = (d + 0.5 * L) % L - 0.5 * L
        r = np.sqrt((d * d).sum(-1))
        np.fill_diagonal(r, np.inf)
        return r.min(axis=1)

    nb = nearest(big["x"], big["y"], 1.0).reshape(R * R, n0)
    npat = nearest(pat["x"], pat["y"], 1.0 / R)
    assert np.allclose(nb, np.broadcast_to(npat, nb.shape), rtol=0, atol=1e-15)
