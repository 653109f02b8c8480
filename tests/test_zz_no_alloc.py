"""Velocity moments without any device allocation.

Some callers cannot call cudaMalloc: a host framework that owns a fixed device memory pool (or a
hard memory budget) and forbids allocations after start-up, or a real-time loop that cannot afford
the device synchronisation cudaMalloc may cause.  ``ann_velocity_moments_noalloc`` serves them from
a fixed device array inside the library.  These tests call it through the C-ABI and check it
against ``ann_get_diagnostics``, which computes the same momentum, mean kinetic energy and peak
speed with scratch memory the context allocated, on two calls in a row (the array keeps the last
call's contents, so the second call checks that nothing stale leaks in).

The file is named to be collected last: if it fails, a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from _sph import gpu_params, params, random_velocity_ic, relerr, stable_dt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding, torch


def test_noalloc_moments_match_diagnostics_twice(env):
    B, torch = env
    nx = 128
    ic = random_velocity_ic(nx, 7)
    p = params(nx, conservative=1, c0_min=0.05)
    p["dt"] = stable_dt(p)
    n = ic["n"]
    ctx = B.ann_create(gpu_params(B, p, n))
    try:
        B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])
        m0 = float(np.float32(p["rho0"] * p["L"] ** 2 / n))   # the context's fixed particle mass
        for call in range(2):
            B.ann_step(ctx, 3)
            d = B.ann_get_diagnostics(ctx)
            ux = torch.empty(n, dtype=torch.float32, device="cuda")
            uy = torch.empty(n, dtype=torch.float32, device="cuda")
            B.ann_get_field(ctx, "UX", n, out=ux)
            B.ann_get_field(ctx, "UY", n, out=uy)
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            B.ann_velocity_moments_noalloc(ux, uy, out, m0=m0, stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert relerr(got[:2], np.array(d["momentum"])) <= 1e-5, (call, got, d["momentum"])
            assert relerr([got[2]], [d["kinetic_energy"]]) <= 1e-5, (call, got, d)
            # both sides take |u| of the same FP32 components in FP64; a tight relative bound
            # keeps the check valid if either reduction changes its order
            assert got[3] == pytest.approx(d["max_speed"], rel=1e-12), (call, got, d)
            assert d["kinetic_energy"] > 0.0
    finally:
        B.ann_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    B, torch = env
    big = B.NOALLOC_MAX_N + 1
    u = torch.zeros(big, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AnnError) as e:
        B.ann_velocity_moments_noalloc(u, u, out)
    assert e.value.status == -11
    # NULL arguments are rejected before any device work
    st = B.lib().ann_velocity_moments_noalloc(None, None, None, ctypes.c_double(1.0), 10, None, None)
    assert st == -1
    # the largest allowed size still works, with per-particle masses
    u = torch.full((B.NOALLOC_MAX_N,), 0.5, dtype=torch.float32, device="cuda")
    m = torch.full((B.NOALLOC_MAX_N,), 2.0, dtype=torch.float32, device="cuda")
    B.ann_velocity_moments_noalloc(u, u, out, mass=m)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == pytest.approx(2.0 * 0.5 * B.NOALLOC_MAX_N, rel=1e-12)
    assert got[2] == pytest.approx(0.25, rel=1e-12)
    assert got[3] == pytest.approx(np.float32(np.sqrt(0.5)), rel=1e-7)


def test_noalloc_rejects_mismatched_arguments_on_the_host(env):
    B, torch = env
    n = 1000
    ux = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    bad = [
        (ux, torch.zeros(n - 1, dtype=torch.float32, device="cuda"), out, None),   # short uy
        (ux, ux, out, torch.zeros(n - 1, dtype=torch.float32, device="cuda")),     # short mass
        (ux, ux, torch.zeros(4, dtype=torch.float32, device="cuda"), None),        # FP32 out
        (ux, ux, torch.zeros(1, dtype=torch.float64, device="cuda"), None),        # 1-element out
        (ux, torch.zeros(n, dtype=torch.float64, device="cuda"), out, None),       # FP64 uy
        (ux, torch.zeros(2 * n, dtype=torch.float32, device="cuda")[::2], out, None),   # strided
        (ux, torch.zeros(n, dtype=torch.float32), out, None),                      # host tensor
    ]
    for a in bad:
        with pytest.raises(ValueError):
            B.ann_velocity_moments_noalloc(a[0], a[1], a[2], mass=a[3])
    # the C entry point itself refuses host memory before any launch
    host = np.zeros(n, dtype=np.float32)
    st = B.lib().ann_velocity_moments_noalloc(
        ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(host.ctypes.data), None, ctypes.c_double(1.0), n,
        ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1
    torch.cuda.synchronize()
    assert torch.all(out == 0)
