"""FP64 CPU oracle of the learned coarse-step surrogate -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
module.  It states the network that the GPU trains and evaluates, in plain numpy FP64, with the
backward pass derived by hand (the pins check it against finite differences).

The paper has no learned component; the surrogate is the project's: a message-passing MLP over
the SPH neighbour graph that maps the state at step t to the increments of Q and u over k = 8
steps.

Graphs and weights.  N(i): the neighbours of particle i closer than a radius R, and SPH weights
normalised per row with the particle itself included (Eqs. 18, 19):
    w_ii = W(0) / S_i,  w_ij = W(|x_i - x_j|) / S_i,  S_i = W(0) + sum_{j in N(i)} W(|x_i - x_j|)
    agg(f)_i = w_ii f_i + sum_{j in N(i)} w_ij f_j          (an SPH mean; agg(const) = const)
Two graphs: the SPH support R = 3h (as in the step) for the features' mean and the explicit
increment, and R = 2h for the network's message passing (about 21 neighbours instead of 48; the
quintic kernel puts about 99 % of its weight inside 2h).
Features (16 per particle, agg on the 3h graph): r_i = (Q11, Q12, ux / us, uy / us) and the
method's own tendencies at
the last step -- the acceleration a (Eq. 23), the projected Q rate m (Eq. 24), the corrected
Laplacian of Q11, Q12 (Eq. 21), and from the corrected velocity gradient D (Eq. 20) the divergence
D_xx + D_yy and the vorticity D_yx - D_xy -- scaled to increments over the k steps it spans:
    x_i = (r_i, agg(r)_i - r_i, a k dt / ys_u, m k dt / ys_q, (lap Q) Gamma K k dt / ys_q,
           (div u, vort u) k dt)
Prediction: an explicit k-step increment plus the network's correction,
    (dQ11, dQ12, dux, duy) = k dt (m11, m12, agg(agg(a))) + (ys_q y0, ys_q y1, ys_u y2, ys_u y3),
so an untrained network (y = 0) reproduces that macro-step and training learns what it misses.
Only the velocity rate is smoothed.  The step's dt sits at the explicit viscous limit, so over k dt
the plain Euler factor of a velocity mode, 1 - k dt lambda(kappa), falls well below -1 away from
the longest waves; the compressive modes of the viscous term of Eq. 23 have about three times the
lambda of the shear modes.  agg multiplies a mode by its SPH transform sigma(kappa), which falls
from 1 at long waves to ~0 at the lattice scale; one pass still leaves compressive modes near a
fifth of the lattice wavenumber at |1 - k dt lambda sigma| > 1, two passes (sigma^2) bring every
lattice mode inside the unit circle once a plain step follows (a pin checks this on a lattice).
The Q rate is dominated by the local bulk term of H (Eq. 25 with A, C) and by Gamma K lap Q, whose
k dt is far from its own limit; smoothing it would erase the particle-local part of the rate.
Layers (relu, width 128, messages of width 32; agg on the 2h graph):
    h1 = relu(W1 [x ; agg(x)] + b1)                 W1: 128 x 32
    z1 = P1 h1,  h2 = relu(W2 [h1 ; agg(z1)] + b2)  P1: 32 x 128, W2: 128 x 160
    z2 = P2 h2,  h3 = relu(W3 [h2 ; agg(z2)] + b3)  P2: 32 x 128, W3: 128 x 160
    y = Wo h3 + bo                                   Wo: 4 x 128
Loss: mean over particles and the 4 outputs of (y - t)^2, t = the normalised residual
(true increment - Euler increment) / ys.
"""
from __future__ import annotations

import numpy as np

F0 = 16      # input features
WIDTH = 128  # hidden width
MSG = 32     # message width
NOUT = 4

SHAPES = {"W1": (WIDTH, 2 * F0), "b1": (WIDTH,), "P1": (MSG, WIDTH), "W2": (WIDTH, WIDTH + MSG),
          "b2": (WIDTH,), "P2": (MSG, WIDTH), "W3": (WIDTH, WIDTH + MSG), "b3": (WIDTH,),
          "Wo": (NOUT, WIDTH), "bo": (NOUT,)}
ORDER = ["W1", "b1", "P1", "W2", "b2", "P2", "W3", "b3", "Wo", "bo"]


def init_params(seed: int):
    """He-style initialisation from the seeded generator of ``sph_inputs`` (Box-Muller)."""
    import sph_inputs as si

    out = {}
    off = 0
    for k in ORDER:
        shape = SHAPES[k]
        size = int(np.prod(shape))
        if k.startswith("b"):
            out[k] = np.zeros(shape)
            continue
        u = si.uniform53(seed, 2 * size, offset=off)
        off += 2 * size
        u1 = np.maximum(u[:size], 1e-300)
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[size:])
        fan_in = shape[1]
        out[k] = g.reshape(shape) * np.sqrt(2.0 / fan_in) * (0.5 if k == "Wo" else 1.0)
    return out


class Graph:
    """Neighbour rows (CSR, self excluded) and the normalised weights of the module header.
    rowptr, cols: the neighbours within the support 3h; radius (in units of h) keeps those closer."""

    def __init__(self, x, y, L, h, rowptr, cols, radius=3.0):
        from . import lib as _lib

        lib = _lib()
        self.n = len(x)
        rowptr = np.asarray(rowptr, dtype=np.int64)
        self.cols = np.asarray(cols, dtype=np.int64)[: rowptr[-1]]
        rows = np.repeat(np.arange(self.n), np.diff(rowptr))
        dx = x[rows] - x[self.cols]
        dy = y[rows] - y[self.cols]
        dx -= L * np.round(dx / L)
        dy -= L * np.round(dy / L)
        r = np.sqrt(dx * dx + dy * dy)
        keep = r < radius * h
        rows, r = rows[keep], r[keep]
        self.cols = self.cols[keep]
        import ctypes

        bq = np.ascontiguousarray(r / h)
        W = np.zeros(bq.size)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_W_array.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp]
        lib.orc_W_array.restype = None
        if bq.size:
            lib.orc_W_array(bq.size, bq.ctypes.data_as(dp), h, W.ctypes.data_as(dp))
        w0 = lib.orc_W(0.0, h)
        S = w0 + np.bincount(rows, weights=W, minlength=self.n)
        self.rows = rows
        self.w_self = w0 / S
        self.w = W / S[rows]

    def agg(self, f):
        """agg(f) for f of shape (n, c)."""
        out = self.w_self[:, None] * f
        np.add.at(out, self.rows, self.w[:, None] * f[self.cols])
        return out

    def agg_T(self, g):
        """The adjoint of agg: sum over rows i of w_ij g_i into j (and w_ii g_i into i)."""
        out = self.w_self[:, None] * g
        np.add.at(out, self.cols, self.w[:, None] * g[self.rows])
        return out


TENDENCIES = ("ax", "ay", "m11", "m12", "lapQ11", "lapQ12", "div_u", "vort_u")


def features(G: Graph, q11, q12, ux, uy, tend, us, kdt, gamma_k, ys_q, ys_u):
    """tend: (n, 8) tendencies of the last step in the order of TENDENCIES."""
    r = np.stack([q11, q12, ux / us, uy / us], axis=1)
    tend = np.asarray(tend, dtype=np.float64)
    x = np.zeros((G.n, F0))
    x[:, :4] = r
    x[:, 4:8] = G.agg(r) - r
    x[:, 8:10] = tend[:, 0:2] * (kdt / ys_u)
    x[:, 10:12] = tend[:, 2:4] * (kdt / ys_q)
    x[:, 12:14] = tend[:, 4:6] * (gamma_k * kdt / ys_q)
    x[:, 14:16] = tend[:, 6:8] * kdt
    return x


def euler_increment(G: Graph, tend, kdt):
    """k dt (m11, m12, agg(agg(a))): the explicit k-step increment the network corrects."""
    tend = np.asarray(tend, dtype=np.float64)
    return kdt * np.concatenate([tend[:, 2:4], G.agg(G.agg(tend[:, 0:2]))], axis=1)


def tendencies_from_record(rec):
    """The 8 tendencies of TENDENCIES from an oracle step record (``step(..., record=True)``)."""
    gu = rec["gradu"].reshape(-1, 4)
    return np.stack([rec["ax"], rec["ay"], rec["qrate11"], rec["qrate12"], rec["lapQ11"], rec["lapQ12"],
                     gu[:, 0] + gu[:, 3], gu[:, 2] - gu[:, 1]], axis=1)


def relu(a):
    return np.maximum(a, 0.0)


def forward(p, G: Graph, x):
    """Output y (n, 4) and the cache the backward pass needs; G is the network's (2h) graph."""
    c = {"x": x}
    c["ax"] = G.agg(x)
    c["in1"] = np.concatenate([x, c["ax"]], axis=1)
    c["a1"] = c["in1"] @ p["W1"].T + p["b1"]
    c["h1"] = relu(c["a1"])
    c["z1"] = c["h1"] @ p["P1"].T
    c["az1"] = G.agg(c["z1"])
    c["in2"] = np.concatenate([c["h1"], c["az1"]], axis=1)
    c["a2"] = c["in2"] @ p["W2"].T + p["b2"]
    c["h2"] = relu(c["a2"])
    c["z2"] = c["h2"] @ p["P2"].T
    c["az2"] = G.agg(c["z2"])
    c["in3"] = np.concatenate([c["h2"], c["az2"]], axis=1)
    c["a3"] = c["in3"] @ p["W3"].T + p["b3"]
    c["h3"] = relu(c["a3"])
    y = c["h3"] @ p["Wo"].T + p["bo"]
    return y, c


def loss(y, t):
    return float(np.mean((y - t) ** 2))


def backward(p, G: Graph, c, y, t):
    """Gradients of ``loss`` with respect to every parameter (same keys as p)."""
    g = {}
    dy = 2.0 * (y - t) / y.size
    g["Wo"] = dy.T @ c["h3"]
    g["bo"] = dy.sum(axis=0)
    dh3 = dy @ p["Wo"]
    da3 = dh3 * (c["a3"] > 0)
    g["W3"] = da3.T @ c["in3"]
    g["b3"] = da3.sum(axis=0)
    din3 = da3 @ p["W3"]
    dh2 = din3[:, :WIDTH].copy()
    dz2 = G.agg_T(din3[:, WIDTH:])
    g["P2"] = dz2.T @ c["h2"]
    dh2 += dz2 @ p["P2"]
    da2 = dh2 * (c["a2"] > 0)
    g["W2"] = da2.T @ c["in2"]
    g["b2"] = da2.sum(axis=0)
    din2 = da2 @ p["W2"]
    dh1 = din2[:, :WIDTH].copy()
    dz1 = G.agg_T(din2[:, WIDTH:])
    g["P1"] = dz1.T @ c["h1"]
    dh1 += dz1 @ p["P1"]
    da1 = dh1 * (c["a1"] > 0)
    g["W1"] = da1.T @ c["in1"]
    g["b1"] = da1.sum(axis=0)
    return g


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected, in place; step counts from 1."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
