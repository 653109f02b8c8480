"""FP64 CPU oracle for the SPH active-nematic step (arXiv 2108.08919) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py``
may import this package.  The product path (``paper_2108_08919_gb300``) never imports it, and it
never imports the product path: the two share nothing but the seeded inputs of ``sph_inputs``.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, compiled without fused multiply-add so
that the neighbour decision ``|d|^2 < (3h)^2`` is reproducible).  This module only marshals numpy
arrays through ctypes.  Each wrapper names the equation of the paper it evaluates; see the C file
for the readings taken where the paper is ambiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "sph_diag.c"), os.path.join(_HERE, "sph_oracle3d.c")]
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double), ("h", ctypes.c_double), ("dt", ctypes.c_double),
        ("rho0", ctypes.c_double), ("eta", ctypes.c_double), ("Gamma", ctypes.c_double),
        ("lam", ctypes.c_double), ("A", ctypes.c_double), ("B", ctypes.c_double),
        ("C", ctypes.c_double), ("K", ctypes.c_double), ("zeta", ctypes.c_double),
        ("gamma_eos", ctypes.c_double), ("beta", ctypes.c_double), ("c0_min", ctypes.c_double),
        ("c_shift", ctypes.c_double),
        ("apd", ctypes.c_int32), ("conservative", ctypes.c_int32),
        ("q_new_in_momentum", ctypes.c_int32), ("nbr_mode", ctypes.c_int32),
        ("elastic", ctypes.c_int32),
    ]


class OrcRecord(ctypes.Structure):
    _fields_ = [(name, _dp) for name in (
        "sumW", "V", "B11", "B12", "B22", "gradu", "lapQ11", "lapQ12", "k", "rho_half", "rho_hat",
        "p", "divQx", "divQy", "ax", "ay", "apdx", "apdy", "trace_m", "qrate11", "qrate12")] + [
        ("nnbr", _ip), ("c0", _dp)]


DEFAULTS = dict(L=1.0, h=1.3 / 64, dt=1e-4, rho0=1.0, eta=1.0, Gamma=0.34, lam=0.7, A=0.0,
                B=0.0, C=1.0, K=0.04, zeta=0.05, gamma_eos=7.0, beta=1.0, c0_min=0.0,
                c_shift=1.0 / 3.0, apd=1, conservative=0, q_new_in_momentum=1, elastic=0)

NBR_MODES = {"brute": 0, "ghost": 1, "cells": 2}


def build(force: bool = False) -> str:
    """Compile ``sph_oracle.c``, ``sph_diag.c`` and ``sph_oracle3d.c`` into ``_lib/liborc.so`` with gcc (OpenMP, no FP
    contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and all(os.path.getmtime(_LIB) >= os.path.getmtime(p) for p in _SRCS)):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_W.restype = ctypes.c_double
        L.orc_W.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_dWdb.restype = ctypes.c_double
        L.orc_dWdb.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_kernel_ad.restype = ctypes.c_double
        L.orc_kernel_ad.argtypes = [ctypes.c_double]
        L.orc_eos.restype = ctypes.c_double
        L.orc_eos.argtypes = [ctypes.c_double] * 4
        for fn in ("orc_neighbors_brute", "orc_neighbors_ghost", "orc_neighbors_cells"):
            f = getattr(L, fn)
            f.restype = ctypes.c_int64
            f.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double, _lp, _ip]
        L.orc_volumes.restype = None
        L.orc_volumes.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                  _lp, _ip, _dp, _dp]
        L.orc_correction.restype = ctypes.c_int64
        L.orc_correction.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                     _lp, _ip, _dp, _dp, _dp, _dp]
        for fn in ("orc_gradient", "orc_laplacian"):
            f = getattr(L, fn)
            f.restype = None
            f.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double, _lp, _ip,
                          _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_density_filter.restype = None
        L.orc_density_filter.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double,
                                         ctypes.c_double, _lp, _ip, ctypes.c_double, _dp, _dp]
        L.orc_continuity.restype = None
        L.orc_continuity.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                     _lp, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_q_rate.restype = None
        L.orc_q_rate.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_double, ctypes.c_double,
                                 _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_elastic_stress.restype = None
        L.orc_elastic_stress.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_double, ctypes.c_double,
                                         _dp, _dp]
        L.orc_momentum_paper.restype = None
        L.orc_momentum_paper.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int64, _dp, _dp, _lp,
                                         _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                         _dp, _dp, _dp, _dp, _dp]
        L.orc_momentum_conservative.restype = None
        L.orc_momentum_conservative.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int64, _dp,
                                                _dp, _lp, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                                _dp, _dp]
        L.orc_apd.restype = None
        L.orc_apd.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, _lp, _ip, _dp, _dp, _dp, _dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int64] + [_dp] * 9 + [
            ctypes.c_int64, ctypes.POINTER(OrcRecord)]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


# ---------------------------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------------------------

def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _wd(n, k=1):
    a = np.zeros(n * k, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def make_params(**kw) -> OrcParams:
    p = dict(DEFAULTS)
    mode = kw.pop("nbr_mode", "brute")
    unknown = set(kw) - set(p)
    if unknown:
        raise KeyError(f"unknown oracle parameters: {sorted(unknown)}")
    p.update(kw)
    return OrcParams(p["L"], p["h"], p["dt"], p["rho0"], p["eta"], p["Gamma"], p["lam"], p["A"],
                     p["B"], p["C"], p["K"], p["zeta"], p["gamma_eos"], p["beta"], p["c0_min"],
                     p["c_shift"], int(p["apd"]), int(p["conservative"]),
                     int(p["q_new_in_momentum"]), NBR_MODES[mode] if isinstance(mode, str) else int(mode),
                     int(p["elastic"]))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


# ---------------------------------------------------------------------------------------------
# kernel, §3 Eq. (18)
# ---------------------------------------------------------------------------------------------

def W(b, h):
    f = lib().orc_W
    return np.array([f(float(v), float(h)) for v in np.atleast_1d(b)])


def dWdb(b, h):
    f = lib().orc_dWdb
    return np.array([f(float(v), float(h)) for v in np.atleast_1d(b)])


def kernel_ad(h):
    return lib().orc_kernel_ad(float(h))


def eos(rho, rho0, c0, gamma_eos=7.0):
    f = lib().orc_eos
    return np.array([f(float(r), float(rho0), float(c0), float(gamma_eos)) for r in np.atleast_1d(rho)])


# ---------------------------------------------------------------------------------------------
# neighbours
# ---------------------------------------------------------------------------------------------

def neighbors(x, y, L, h, mode="brute"):
    """CSR neighbour lists (rowptr int64[n+1], cols int32[nnz]); rows in ascending j."""
    x, xp = _d(x)
    y, yp = _d(y)
    n = x.shape[0]
    fn = {"brute": lib().orc_neighbors_brute, "ghost": lib().orc_neighbors_ghost,
          "cells": lib().orc_neighbors_cells}[mode]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    nnz = fn(n, xp, yp, float(L), float(h), rowptr.ctypes.data_as(_lp), None)
    if nnz < 0:
        raise MemoryError("oracle neighbour search failed")
    cols = np.zeros(max(nnz, 1), dtype=np.int32)
    fn(n, xp, yp, float(L), float(h), rowptr.ctypes.data_as(_lp), cols.ctypes.data_as(_ip))
    return rowptr, cols[:nnz]


class Nbrs:
    """Positions plus their neighbour lists, the common input of the operator wrappers."""

    def __init__(self, x, y, L, h, mode="brute"):
        self.x, self.xp = _d(x)
        self.y, self.yp = _d(y)
        self.n = self.x.shape[0]
        self.L, self.h = float(L), float(h)
        self.rowptr, cols = neighbors(self.x, self.y, L, h, mode)
        self.cols = np.ascontiguousarray(cols if cols.size else np.zeros(1, np.int32))
        self.rp = self.rowptr.ctypes.data_as(_lp)
        self.cp = self.cols.ctypes.data_as(_ip)

    def args(self):
        return (self.n, self.xp, self.yp, self.L, self.h, self.rp, self.cp)


# ---------------------------------------------------------------------------------------------
# operators, §3
# ---------------------------------------------------------------------------------------------

def volumes(nb: Nbrs):
    """Eq. (19): (sum_j W_ij including self, V = 1/sum)."""
    s, sp = _wd(nb.n)
    V, Vp = _wd(nb.n)
    lib().orc_volumes(*nb.args(), sp, Vp)
    return s, V


def correction(nb: Nbrs, V):
    """Eq. (22) and its inverse: (B11, B12, B22, number of non-positive det alpha)."""
    V, Vp = _d(V)
    b11, b11p = _wd(nb.n)
    b12, b12p = _wd(nb.n)
    b22, b22p = _wd(nb.n)
    bad = lib().orc_correction(*nb.args(), Vp, b11p, b12p, b22p)
    return b11, b12, b22, bad


def gradient(nb: Nbrs, V, B, f):
    """Eq. (20): corrected gradient of a scalar field, shape (n, 2)."""
    V, Vp = _d(V)
    B = [_d(b) for b in B]
    f, fp = _d(f)
    out, op = _wd(nb.n, 2)
    lib().orc_gradient(*nb.args(), Vp, B[0][1], B[1][1], B[2][1], fp, op)
    return out.reshape(nb.n, 2)


def laplacian(nb: Nbrs, V, B, f):
    """Eq. (21) (scalar corrected reading): Laplacian of a scalar field."""
    V, Vp = _d(V)
    B = [_d(b) for b in B]
    f, fp = _d(f)
    out, op = _wd(nb.n)
    lib().orc_laplacian(*nb.args(), Vp, B[0][1], B[1][1], B[2][1], fp, op)
    return out


def density_filter(nb: Nbrs, rho, beta=1.0):
    """Eq. (28)."""
    rho, rp = _d(rho)
    out, op = _wd(nb.n)
    lib().orc_density_filter(*nb.args(), float(beta), rp, op)
    return out


def continuity(nb: Nbrs, V, B, ux, uy, rho):
    """Eq. (25): k_i."""
    V, Vp = _d(V)
    B = [_d(b) for b in B]
    ux, uxp = _d(ux)
    uy, uyp = _d(uy)
    rho, rp = _d(rho)
    out, op = _wd(nb.n)
    lib().orc_continuity(*nb.args(), Vp, B[0][1], B[1][1], B[2][1], uxp, uyp, rp, op)
    return out


def q_rate(params: OrcParams, q11, q12, D, lapQ, with_H=False):
    """Eq. (24) for one particle: (m11, m12, trace of the unprojected m[, H as 2x2])."""
    D, Dp = _d(np.asarray(D, dtype=np.float64).reshape(4))
    lQ, lQp = _d(np.asarray(lapQ, dtype=np.float64).reshape(4))
    m11 = ctypes.c_double()
    m12 = ctypes.c_double()
    tr = ctypes.c_double()
    H, Hp = _wd(4)
    lib().orc_q_rate(ctypes.byref(params), float(q11), float(q12), Dp, lQp, ctypes.byref(m11),
                     ctypes.byref(m12), ctypes.byref(tr), Hp)
    if with_H:
        return m11.value, m12.value, tr.value, H.reshape(2, 2)
    return m11.value, m12.value, tr.value


def elastic_stress(params: OrcParams, q11, q12, H):
    """Eq. (12) without -p I, for one particle: Pi_el as 2x2."""
    H, Hp = _d(np.asarray(H, dtype=np.float64).reshape(4))
    out, op = _wd(4)
    lib().orc_elastic_stress(ctypes.byref(params), float(q11), float(q12), Hp, op)
    return out.reshape(2, 2)


def momentum_paper(params: OrcParams, nb: Nbrs, V, B, rho, p, ux, uy, q11, q12, pel=None):
    """Eq. (23) with the active term scaled by -zeta/rho: (ax, ay, divQx, divQy).  ``pel``: the
    elastic stress per particle as (n, 3) = (11, 12, 22), used when params.elastic is set."""
    arrs = [_d(a) for a in (V, B[0], B[1], B[2], rho, p, ux, uy, q11, q12)]
    outs = [_wd(nb.n) for _ in range(4)]
    pe = _d(np.zeros(3 * nb.n) if pel is None else np.asarray(pel, dtype=np.float64).reshape(-1))
    lib().orc_momentum_paper(ctypes.byref(params), nb.n, nb.xp, nb.yp, nb.rp, nb.cp,
                             *[a[1] for a in arrs], *[o[1] for o in outs], pe[1])
    return tuple(o[0] for o in outs)


def momentum_conservative(params: OrcParams, nb: Nbrs, rho, p, ux, uy, q11, q12, pel=None):
    arrs = [_d(a) for a in (rho, p, ux, uy, q11, q12)]
    outs = [_wd(nb.n) for _ in range(2)]
    pe = _d(np.zeros(3 * nb.n) if pel is None else np.asarray(pel, dtype=np.float64).reshape(-1))
    lib().orc_momentum_conservative(ctypes.byref(params), nb.n, nb.xp, nb.yp, nb.rp, nb.cp,
                                    *[a[1] for a in arrs], *[o[1] for o in outs], pe[1])
    return tuple(o[0] for o in outs)


def apd(nb: Nbrs, ux, uy, dt):
    """Eq. (29): the displacement (dx, dy)."""
    ux, uxp = _d(ux)
    uy, uyp = _d(uy)
    ox, oxp = _wd(nb.n)
    oy, oyp = _wd(nb.n)
    lib().orc_apd(nb.n, nb.xp, nb.yp, nb.L, nb.h, float(dt), nb.rp, nb.cp, uxp, uyp, oxp, oyp)
    return ox, oy


# ---------------------------------------------------------------------------------------------
# time step, §3.1
# ---------------------------------------------------------------------------------------------

STATE_FIELDS = ("x", "y", "ux", "uy", "q11", "q12", "rho", "ax", "ay")
RECORD_FIELDS = ("sumW", "V", "B11", "B12", "B22", "gradu", "lapQ11", "lapQ12", "k", "rho_half",
                 "rho_hat", "p", "divQx", "divQy", "ax", "ay", "apdx", "apdy", "trace_m", "qrate11", "qrate12")


def step(params: OrcParams, state: dict, nsteps: int = 1, record: bool = False):
    """Advance a copy of ``state`` by ``nsteps`` modified-Euler steps.

    ``state`` holds float64 arrays ``x, y, ux, uy, q11, q12, rho`` and optionally ``ax, ay``
    (a^n, default zero).  Returns ``(new_state, rec)``; ``rec`` holds the last step's
    intermediates when ``record`` is set, else None.
    """
    n = int(np.asarray(state["x"]).shape[0])
    st = {}
    for k in STATE_FIELDS:
        v = state.get(k)
        st[k] = np.array(v, dtype=np.float64, copy=True) if v is not None else np.zeros(n)
    ptrs = [st[k].ctypes.data_as(_dp) for k in STATE_FIELDS]
    rec = None
    recp = None
    if record:
        rec = {k: np.zeros(n * (4 if k == "gradu" else 1)) for k in RECORD_FIELDS}
        rec["nnbr"] = np.zeros(n, dtype=np.int32)
        rec["c0"] = np.zeros(1)
        r = OrcRecord()
        for k in RECORD_FIELDS:
            setattr(r, k, rec[k].ctypes.data_as(_dp))
        r.nnbr = rec["nnbr"].ctypes.data_as(_ip)
        r.c0 = rec["c0"].ctypes.data_as(_dp)
        recp = ctypes.byref(r)
    rc = lib().orc_step(ctypes.byref(params), n, *ptrs, int(nsteps), recp)
    if rc == -1:
        raise MemoryError("oracle step: allocation failed")
    if rec is not None:
        rec["gradu"] = rec["gradu"].reshape(n, 4)
        rec["c0"] = float(rec["c0"][0])
        rec["status"] = rc
    return st, rec
