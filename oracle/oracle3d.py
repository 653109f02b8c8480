"""The three-dimensional FP64 oracle (``sph_oracle3d.c``) from Python -- TEST INFRASTRUCTURE.

Only ``tests/`` and the CPU legs of ``bench.py`` may import this module.  State layout: x, y, z
and rho of length n; u and a as (n, 3); Q as (n, 5) = (Q11, Q12, Q13, Q22, Q23), Q33 = -Q11 - Q22.
The 3D readings of the paper are listed at the top of ``sph_oracle3d.c``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib as _lib

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int32)

DEFAULTS = dict(L=1.0, h=1.3 / 16, dt=1e-4, rho0=1.0, eta=1.0, Gamma=0.34, lam=0.7, A=0.0, B=0.0, C=1.0,
                K=0.04, zeta=0.05, gamma_eos=7.0, beta=1.0, c0_min=0.0, c_shift=1.0 / 3.0, apd=1)
_ORDER = ("L", "h", "dt", "rho0", "eta", "Gamma", "lam", "A", "B", "C", "K", "zeta", "gamma_eos", "beta",
          "c0_min", "c_shift")


class Params3(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in _ORDER] + [("apd", ctypes.c_int32)]


class Nb3(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", _dp), ("y", _dp), ("z", _dp), ("L", ctypes.c_double),
                ("h", ctypes.c_double), ("rp", _lp), ("cols", _ip)]


REC_FIELDS = {"sumW": 1, "V": 1, "Bm": 9, "gradu": 9, "lapQ": 5, "qrate": 5, "k": 1, "rho_half": 1,
              "rho_hat": 1, "p": 1, "a": 3, "apd": 3}


class Rec3(ctypes.Structure):
    _fields_ = [(k, _dp) for k in REC_FIELDS] + [("nnbr", _ip), ("c0", _dp)]


_ready = False


def lib():
    global _ready
    L = _lib()
    if not _ready:
        L.orc3_kernel_ad.restype = ctypes.c_double
        L.orc3_kernel_ad.argtypes = [ctypes.c_double]
        L.orc3_W.restype = ctypes.c_double
        L.orc3_W.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc3_dWdb.restype = ctypes.c_double
        L.orc3_dWdb.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc3_neighbors.restype = ctypes.c_int64
        L.orc3_neighbors.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _lp, _ip]
        nb = ctypes.POINTER(Nb3)
        L.orc3_volumes.restype = None
        L.orc3_volumes.argtypes = [nb, _dp, _dp]
        L.orc3_correction.restype = ctypes.c_int64
        L.orc3_correction.argtypes = [nb, _dp, _dp]
        for fn in ("orc3_gradient", "orc3_laplacian"):
            getattr(L, fn).restype = None
            getattr(L, fn).argtypes = [nb, _dp, _dp, _dp, _dp]
        L.orc3_q_rate.restype = None
        L.orc3_q_rate.argtypes = [ctypes.POINTER(Params3), _dp, _dp, _dp, _dp, _dp]
        L.orc3_momentum.restype = None
        L.orc3_momentum.argtypes = [ctypes.POINTER(Params3), nb, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc3_step.restype = ctypes.c_int
        L.orc3_step.argtypes = [ctypes.POINTER(Params3), ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                ctypes.c_int64, ctypes.POINTER(Rec3)]
        _ready = True
    return L


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def make_params(**kw) -> Params3:
    p = dict(DEFAULTS)
    unknown = set(kw) - set(p)
    if unknown:
        raise KeyError(f"unknown 3D oracle parameters: {sorted(unknown)}")
    p.update(kw)
    return Params3(*[float(p[k]) for k in _ORDER], int(p["apd"]))


def kernel_ad(h):
    return lib().orc3_kernel_ad(float(h))


def W(b, h):
    return np.array([lib().orc3_W(float(v), float(h)) for v in np.atleast_1d(b)])


def dWdb(b, h):
    return np.array([lib().orc3_dWdb(float(v), float(h)) for v in np.atleast_1d(b)])


class Nbrs3:
    """Positions and their neighbour lists (support 3h, minimum image), the input of the operators."""

    def __init__(self, x, y, z, L, h):
        self.x, xp = _d(x)
        self.y, yp = _d(y)
        self.z, zp = _d(z)
        self.n = self.x.shape[0]
        self.rowptr = np.zeros(self.n + 1, dtype=np.int64)
        ne = lib().orc3_neighbors(self.n, xp, yp, zp, L, h, self.rowptr.ctypes.data_as(_lp), None)
        self.cols = np.zeros(max(ne, 1), dtype=np.int32)
        lib().orc3_neighbors(self.n, xp, yp, zp, L, h, self.rowptr.ctypes.data_as(_lp), self.cols.ctypes.data_as(_ip))
        self.s = Nb3(self.n, xp, yp, zp, float(L), float(h), self.rowptr.ctypes.data_as(_lp),
                     self.cols.ctypes.data_as(_ip))

    def ref(self):
        return ctypes.byref(self.s)


def volumes(nb: Nbrs3):
    s, V = np.zeros(nb.n), np.zeros(nb.n)
    lib().orc3_volumes(nb.ref(), s.ctypes.data_as(_dp), V.ctypes.data_as(_dp))
    return s, V


def correction(nb: Nbrs3, V):
    V, Vp = _d(V)
    Bm = np.zeros(9 * nb.n)
    bad = lib().orc3_correction(nb.ref(), Vp, Bm.ctypes.data_as(_dp))
    return Bm.reshape(nb.n, 3, 3), bad


def gradient(nb: Nbrs3, V, Bm, f):
    V, Vp = _d(V)
    Bm, Bp = _d(np.asarray(Bm).reshape(-1))
    f, fp = _d(f)
    out = np.zeros(3 * nb.n)
    lib().orc3_gradient(nb.ref(), Vp, Bp, fp, out.ctypes.data_as(_dp))
    return out.reshape(nb.n, 3)


def laplacian(nb: Nbrs3, V, Bm, f):
    V, Vp = _d(V)
    Bm, Bp = _d(np.asarray(Bm).reshape(-1))
    f, fp = _d(f)
    out = np.zeros(nb.n)
    lib().orc3_laplacian(nb.ref(), Vp, Bp, fp, out.ctypes.data_as(_dp))
    return out


def q_rate(P: Params3, q5, D, lapq5):
    q5, qp = _d(q5)
    D, Dp = _d(np.asarray(D).reshape(9))
    lq, lp = _d(lapq5)
    m = np.zeros(5)
    tr = np.zeros(1)
    lib().orc3_q_rate(ctypes.byref(P), qp, Dp, lp, m.ctypes.data_as(_dp), tr.ctypes.data_as(_dp))
    return m, float(tr[0])


def momentum(P: Params3, nb: Nbrs3, V, Bm, rho, p, u, q):
    args = [_d(v) for v in (V, np.asarray(Bm).reshape(-1), rho, p, np.asarray(u).reshape(-1),
                            np.asarray(q).reshape(-1))]
    a = np.zeros(3 * nb.n)
    dq = np.zeros(3 * nb.n)
    lib().orc3_momentum(ctypes.byref(P), nb.ref(), *[v[1] for v in args], a.ctypes.data_as(_dp),
                        dq.ctypes.data_as(_dp))
    return a.reshape(nb.n, 3), dq.reshape(nb.n, 3)


STATE = ("x", "y", "z", "u", "q", "rho", "a")


def step(P: Params3, state: dict, nsteps: int = 1, record: bool = False):
    """Advance a copy of ``state`` (x, y, z, rho: (n,); u, a: (n, 3); q: (n, 5); a optional, 0)
    by ``nsteps`` modified-Euler steps.  Returns (new_state, rec or None)."""
    n = int(np.asarray(state["x"]).shape[0])
    st = {k: np.array(state[k], dtype=np.float64, copy=True) for k in ("x", "y", "z", "rho")}
    st["u"] = np.array(state["u"], dtype=np.float64, copy=True).reshape(n, 3)
    st["q"] = np.array(state["q"], dtype=np.float64, copy=True).reshape(n, 5)
    st["a"] = (np.zeros((n, 3)) if state.get("a") is None
               else np.array(state["a"], dtype=np.float64, copy=True).reshape(n, 3))
    rec, recp = None, None
    if record:
        rec = {k: np.zeros(n * c) for k, c in REC_FIELDS.items()}
        rec["nnbr"] = np.zeros(n, dtype=np.int32)
        rec["c0"] = np.zeros(1)
        r = Rec3(*[rec[k].ctypes.data_as(_dp) for k in REC_FIELDS], rec["nnbr"].ctypes.data_as(_ip),
                 rec["c0"].ctypes.data_as(_dp))
        recp = ctypes.byref(r)
    ptr = [st[k].ctypes.data_as(_dp) for k in ("x", "y", "z", "u", "q", "rho", "a")]
    rc = lib().orc3_step(ctypes.byref(P), n, *ptr, int(nsteps), recp)
    if rc == -1:
        raise MemoryError("3D oracle step: allocation failed")
    if rec is not None:
        for k, c in REC_FIELDS.items():
            if c > 1:
                rec[k] = rec[k].reshape(n, c)
        rec["c0"] = float(rec["c0"][0])
        rec["status"] = rc
    return st, rec
