"""FP64 CPU oracle of the flow diagnostics of the paper's results section -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
module; the product path never does.  Gridding and defect counting are plain C (``sph_diag.c``);
the rest is numpy, with ``numpy.fft.fft2`` as the one library step.

Definitions (the paper gives the quantities, not their discretisation; each reading is listed
with the code that takes it):
  * kinetic energy per unit mass E = 1/2 <u^2> (Eq. 31); its spectrum E(w), w = 2 pi n / L: the
    Shepard-gridded velocity (``grid_shepard``) is Fourier transformed, u_hat = fft2(u) / M^2, and
    E_n = 1/2 sum |u_hat(k)|^2 over the integer wavevectors k with nearest-integer |k| = n, so
    that sum_n E_n = 1/2 mean(|u_grid|^2) (Parseval).  |k| is never a half integer, so the shell
    of every k is decided exactly.
  * vorticity omega = d uy/dx - d ux/dy on the grid by periodic central differences.
  * correlation C(r) = <f(r) f(0)> / f(0)^2 (Eq. 32) along the horizontal centre line
    (row M/2), r = k L/M, k = 0..M/2: with one origin at the centre (the paper's r = 0) or
    averaged over every origin of the line (the box is periodic and homogeneous):
    C(k) = sum_i f(i + k) f(i) / sum_i f(i)^2.  Length scales: the first r where C reaches 0, and
    the first where it falls below 0.2 max C, by linear interpolation between grid points.
  * defects: winding number of (Q11, Q12) around each grid plaquette (``defects``, exact).
  * mixing: the paper colours particles by their initial region and shows the colours mix.  The
    measure taken is Danckwerts' intensity of segregation on a G x G grid of bins, averaged over
    the species present: for species s with overall fraction a_s (0 < a_s < 1),
    I_s = mean over non-empty bins of (f_bs - a_s)^2 / (a_s (1 - a_s)), f_bs = the species
    fraction in bin b; I = mean_s I_s.  Fully segregated at the bin scale gives 1, perfectly mixed
    gives 0.  Bin of a particle: floor(x G / L), clamped to G - 1.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import lib as _orc_lib

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)
_bp = ctypes.POINTER(ctypes.c_int8)
_ready = False


def _lib():
    global _ready
    L = _orc_lib()
    if not _ready:
        args = [ctypes.c_int64, _dp, _dp, ctypes.c_int32, _dp, ctypes.c_double, ctypes.c_double,
                ctypes.c_int32, _dp, _dp]
        L.orc_grid_shepard_brute.argtypes = args
        L.orc_grid_shepard_cells.argtypes = args
        L.orc_grid_nodes.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_int32, _dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int32, ctypes.c_int64, _lp, _dp, _dp]
        L.orc_defects.argtypes = [ctypes.c_int32, _dp, _dp, _bp, _lp]
        for f in (L.orc_grid_shepard_brute, L.orc_grid_shepard_cells, L.orc_grid_nodes, L.orc_defects):
            f.restype = None
        _ready = True
    return L


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def grid_shepard(x, y, fields, L, h, M, mode="cells"):
    """Shepard interpolation of the particle fields onto the M x M nodes (ix L/M, iy L/M).
    Returns (grids [nf, M, M] indexed [q, iy, ix], weight sums [M, M])."""
    x, px = _d(x)
    y, py = _d(y)
    f, pf = _d(np.stack([np.asarray(v, dtype=np.float64) for v in fields]))
    nf = f.shape[0]
    assert nf <= 16
    out = np.zeros((nf, M, M))
    ws = np.zeros((M, M))
    fn = {"brute": _lib().orc_grid_shepard_brute, "cells": _lib().orc_grid_shepard_cells}[mode]
    fn(x.size, px, py, nf, pf, L, h, M, out.ctypes.data_as(_dp), ws.ctypes.data_as(_dp))
    return out, ws


def grid_nodes(x, y, fields, L, h, M, nodes):
    """The same interpolation at selected nodes (index iy M + ix), brute force: ([k, nf], [k])."""
    x, px = _d(x)
    y, py = _d(y)
    f, pf = _d(np.stack([np.asarray(v, dtype=np.float64) for v in fields]))
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((nodes.size, f.shape[0]))
    ws = np.zeros(nodes.size)
    _lib().orc_grid_nodes(x.size, px, py, f.shape[0], pf, L, h, M, nodes.size,
                          nodes.ctypes.data_as(_lp), out.ctypes.data_as(_dp), ws.ctypes.data_as(_dp))
    return out, ws


def n_shells(M):
    return int(round(M / math.sqrt(2.0))) + 1


def shell_index(M):
    """Nearest-integer |k| of every FFT mode [iy, ix] (integer wavevector components)."""
    k = np.fft.fftfreq(M, d=1.0 / M).round().astype(np.int64)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    return np.rint(np.sqrt(k2.astype(np.float64))).astype(np.int64)


def energy_spectrum(ux_g, uy_g, L):
    """(w [nshell], E [nshell]) of the gridded velocity (see the module header)."""
    M = ux_g.shape[0]
    ux_hat = np.fft.fft2(ux_g) / M ** 2
    uy_hat = np.fft.fft2(uy_g) / M ** 2
    e = 0.5 * (np.abs(ux_hat) ** 2 + np.abs(uy_hat) ** 2)
    E = np.bincount(shell_index(M).ravel(), weights=e.ravel(), minlength=n_shells(M))
    w = 2.0 * np.pi * np.arange(E.size) / L
    return w, E


def spectrum_slope(w, E, w1, w2):
    """Least-squares slope of log E against log w over the shells with w1 <= w <= w2, E > 0."""
    m = (w >= w1) & (w <= w2) & (E > 0) & (w > 0)
    if m.sum() < 2:
        return float("nan")
    return float(np.polyfit(np.log(w[m]), np.log(E[m]), 1)[0])


def vorticity(ux_g, uy_g, L):
    """omega[iy, ix] = (uy[ix+1] - uy[ix-1]) / 2D - (ux[iy+1] - ux[iy-1]) / 2D, D = L/M."""
    M = ux_g.shape[0]
    D = L / M
    return ((np.roll(uy_g, -1, axis=1) - np.roll(uy_g, 1, axis=1)) / (2 * D)
            - (np.roll(ux_g, -1, axis=0) - np.roll(ux_g, 1, axis=0)) / (2 * D))


def correlation(f_g, all_origins=True):
    """C[k], k = 0..M/2, along the centre row (see the module header)."""
    M = f_g.shape[0]
    line = f_g[M // 2]
    ks = np.arange(M // 2 + 1)
    if all_origins:
        den = np.sum(line * line)
        return np.array([np.sum(np.roll(line, -k) * line) for k in ks]) / den
    i0 = M // 2
    return np.array([line[(i0 + k) % M] * line[i0] for k in ks]) / (line[i0] * line[i0])


def crossing_length(C, L, level):
    """First r = k L/M where C falls to `level` or below (linear interpolation), NaN if never."""
    M = 2 * (C.size - 1)
    for k in range(C.size - 1):
        if C[k] > level >= C[k + 1]:
            return (k + (C[k] - level) / (C[k] - C[k + 1])) * L / M
    return float("nan")


def length_scales(C, L):
    return crossing_length(C, L, 0.0), crossing_length(C, L, 0.2 * float(np.max(C)))


def defects(q11_g, q12_g):
    """(winding map m [M, M] int8 for the plaquette at lower-left node [iy, ix], counts
    (m = +1, m = -1, |m| >= 2))."""
    M = q11_g.shape[0]
    a, pa = _d(q11_g)
    b, pb = _d(q12_g)
    m = np.zeros((M, M), dtype=np.int8)
    counts = np.zeros(3, dtype=np.int64)
    _lib().orc_defects(M, pa, pb, m.ctypes.data_as(_bp), counts.ctypes.data_as(_lp))
    return m, counts


def mixing_index(x, y, colors, L, G):
    """(I, per-species I_s or NaN where a_s is 0 or 1) of the module header."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    colors = np.asarray(colors, dtype=np.int64)
    bx = np.minimum(np.floor(x * G / L).astype(np.int64), G - 1)
    by = np.minimum(np.floor(y * G / L).astype(np.int64), G - 1)
    b = by * G + bx
    S = int(colors.max()) + 1 if colors.size else 1
    cnt = np.zeros((G * G, S))
    np.add.at(cnt, (b, colors), 1.0)
    nb = cnt.sum(axis=1)
    full = nb > 0
    frac = cnt[full] / nb[full, None]
    a = np.bincount(colors, minlength=S) / colors.size
    Is = np.full(S, np.nan)
    for s in range(S):
        if 0.0 < a[s] < 1.0:
            Is[s] = np.mean((frac[:, s] - a[s]) ** 2) / (a[s] * (1.0 - a[s]))
    ok = ~np.isnan(Is)
    return (float(Is[ok].mean()) if ok.any() else 0.0), Is


def min_image(d, L):
    return d - L * np.round(d / L)


class Unwrapper:
    """Unwrapped trajectories of an oracle run advanced step by step: each step's displacement is
    taken as its minimum image (valid while a particle moves less than L/2 per step)."""

    def __init__(self, x, y, L):
        self.L = L
        self.x = np.array(x, dtype=np.float64)
        self.y = np.array(y, dtype=np.float64)
        self.ux = self.x.copy()
        self.uy = self.y.copy()

    def update(self, x, y):
        self.ux += min_image(np.asarray(x) - self.x, self.L)
        self.uy += min_image(np.asarray(y) - self.y, self.L)
        self.x = np.array(x, dtype=np.float64)
        self.y = np.array(y, dtype=np.float64)
