"""Long-run statistics (results section) against the oracle's diagnostics, through the C-ABI.

`paper_2108_08919_gb300.longrun` records, every few thousand steps, the statistics the results
section judges active turbulence by: the energy spectrum and its slope (Eq. 31), the vorticity
correlation lengths (Eq. 32), the defect counts, the rms velocity and the order.  Here a short run
(two members, 128^2, the scaled-viscosity reading) is stopped at each snapshot and the recorded
numbers are recomputed by the FP64 oracle from the state they were taken from: the Shepard grid of
the particles (FP32 sums against FP64: 1e-5), and, on the GPU's own grid, the spectrum, slope and
correlation lengths (1e-12) and the defect counts (exact).  The rms velocity and order follow from
the particle state in FP64.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding


def test_long_run_statistics_match_the_oracle(B):
    from oracle import diagnostics as D
    from paper_2108_08919_gb300 import longrun

    nx, M = 128, 128
    checked = []

    def check(k, ctx, s):
        n = nx * nx
        st = B.ann_get_state(ctx, n)
        x, y = st["X"], st["Y"]
        ux, uy = st["UX"].astype(np.float64), st["UY"].astype(np.float64)
        q11, q12 = st["Q11"].astype(np.float64), st["Q12"].astype(np.float64)
        assert s["vrms"] == pytest.approx(math.sqrt(np.mean(ux * ux + uy * uy)), rel=1e-12, abs=1e-300)
        assert s["mean_q"] == pytest.approx(np.mean(np.hypot(q11, q12)), rel=1e-6)
        g = B.ann_grid_fields(ctx, M)
        h = 1.3 / nx
        og, _ = D.grid_shepard(x, y, [ux, uy, q11, q12], 1.0, h, M)
        for c in range(4):
            scale = np.abs(og[c]).max()
            assert np.abs(g[c] - og[c]).max() <= 1e-5 * scale + 1e-30, c
        w, E = D.energy_spectrum(g[0], g[1], 1.0)
        # FP64 FFT round-off is relative to the whole spectrum, not to each (possibly tiny) shell
        np.testing.assert_allclose(s["spectrum"], E, rtol=0, atol=1e-12 * E.max())
        slope = D.spectrum_slope(w, E, 2 * math.pi * 3, 2 * math.pi * 20)
        if math.isfinite(slope):
            assert s["slope"] == pytest.approx(slope, rel=1e-10)
        C = D.correlation(D.vorticity(g[0], g[1], 1.0))
        l0, l02 = D.length_scales(C, 1.0)
        for got, want in ((s["corr_zero"], l0), (s["corr_02"], l02)):
            assert (math.isnan(got) and math.isnan(want)) or got == pytest.approx(want, rel=1e-10)
        _, counts = D.defects(g[2], g[3])
        assert (s["defects_plus"], s["defects_minus"]) == (int(counts[0]), int(counts[1]))
        checked.append((k, s["step"]))

    res = longrun.run([(0.1, 0.02), (0.05, 0.04)], nx=nx, steps=6000, every=3000, M=M, eta=0.03, dt=1e-4,
                      keep_spectra=True, initial="random_director", on_snapshot=check)
    assert sorted(checked) == [(0, 0), (0, 3000), (0, 6000), (1, 0), (1, 3000), (1, 6000)]
    assert all(m["failed"] is None for m in res["members"])
    # the first snapshot is the seeded random director: thousands of defects; they anneal
    for m in res["members"]:
        d = [s["defect_density"] for s in m["snapshots"]]
        assert d[0] > 1000 and d[-1] < d[0] / 10
    # the more active member moves faster
    v = [m["snapshots"][-1]["vrms"] for m in res["members"]]
    assert v[0] > v[1] > 0.0
