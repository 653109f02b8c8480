"""Qualitative trends of the paper's results (§5) on short GPU runs: statistics, not pointwise
parity (the oracle pins the pointwise step; these check that the flow statistics respond to the
parameters the way the paper reports).

* The rms velocity grows with |zeta| for extensile (zeta > 0) and contractile (zeta < 0) activity
  alike.  From rest the flow is driven by the active force -zeta div Q, so at early times it is
  linear in zeta: four times the activity gives about four times the rms velocity, and reversing
  the sign of zeta reverses the flow and keeps its rms.
* A larger elastic constant K orders the director faster: the +-1/2 defects of a random initial
  director field annihilate sooner (the paper's elastic constant acts against the activity).
"""
import numpy as np
import pytest

import sph_inputs as si
from _sph import GpuRun, params, stable_dt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding


def _vrms(run):
    s = run.state()
    return float(np.sqrt(np.mean(s["ux"] ** 2 + s["uy"] ** 2)))


def test_rms_velocity_grows_with_activity_of_either_sign(B):
    nx, steps = 64, 300
    ic = si.jittered_lattice(nx, seed=31)
    base = params(nx, K=0.04, eta=0.1, c0_min=0.5)
    dt = stable_dt(base)
    v = {}
    for zeta in (0.05, 0.2, -0.05, -0.2):
        p = dict(base, zeta=zeta, dt=dt)
        run = GpuRun(B, p, ic)
        try:
            run.step(steps)
            v[zeta] = _vrms(run)
            assert B.ann_get_diagnostics(run.ctx)["error_bits"] == 0
        finally:
            run.close()
    print({k: f"{x:.3e}" for k, x in v.items()})
    for s in (1.0, -1.0):
        ratio = v[0.2 * s] / v[0.05 * s]
        assert 3.6 < ratio < 4.4, v          # monotone in |zeta|, linear from rest (measured 4.00)
    assert abs(v[-0.2] / v[0.2] - 1.0) < 0.02, v  # extensile and contractile alike (measured 0.2 %)


def test_defects_annihilate_faster_with_larger_elastic_constant(B):
    nx, M, steps = 96, 64, 1500
    ic = si.jittered_lattice(nx, seed=32)
    stiff = params(nx, zeta=0.05, K=0.08, c0_min=0.5)
    dt = stable_dt(stiff)                     # the smaller dt of the two: the same times for both
    counts = {}
    for K in (0.02, 0.08):
        run = GpuRun(B, dict(stiff, K=K, dt=dt), ic)
        try:
            c0, _ = B.ann_defects(run.ctx, M)
            run.step(steps)
            c1, _ = B.ann_defects(run.ctx, M)
            counts[K] = (int(c0[0] + c0[1]), int(c1[0] + c1[1]))
            assert c1[0] == c1[1]              # +1/2 and -1/2 in pairs on a periodic box
        finally:
            run.close()
    print(counts)
    assert counts[0.02][0] == counts[0.08][0] > 0     # the same random initial director field
    assert counts[0.08][1] < counts[0.02][1] < counts[0.02][0]
