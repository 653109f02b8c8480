"""Batched ensemble through the C-ABI: members of uneven size and parameters, advanced by one
graph launch per step, end bit-identical to the same members advanced alone, under every grouping
of members into graph branches and after autotuning; a failing member is reported by index while
the others advance."""
import numpy as np
import pytest

import sph_inputs as si
from _sph import gpu_params, params, random_velocity_ic, stable_dt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding


def _members():
    """(params dict, initial condition) of five uneven members: extensile and contractile activity,
    several K, one fast enough to re-sort every few steps, one in the conservative mode."""
    out = []
    for k, (nx, zeta, K, u) in enumerate(((32, 0.05, 0.04, 1e-3), (48, -0.08, 0.02, 1e-3),
                                          (64, 0.12, 0.06, 1e-3), (40, 0.02, 0.01, 2.0),
                                          (56, -0.01, 0.08, 1e-3))):
        p = params(nx, zeta=zeta, K=K, c0_min=0.5)
        if u > 1.0:
            p["eta"] = 0.1
        p["dt"] = stable_dt(p)
        if k == 4:
            p["conservative"] = 1
        out.append((p, random_velocity_ic(nx, 40 + k, u_scale=u, rho_scale=1e-4)))
    return out


def _load(B, ctx, ic):
    B.ann_set_particles(ctx, ic["x"], ic["y"], ic["ux"], ic["uy"], ic["q11"], ic["q12"], ic["rho"])


def _state(B, ctx, n):
    return {f: B.ann_get_field(ctx, f, n) for f in ("X", "Y", "UX", "UY", "Q11", "Q12", "DRHO", "AX", "AY")}


def test_members_match_solo_runs_bitwise(B):
    mem = _members()
    ens = B.ann_ensemble_create([gpu_params(B, p, ic["n"]) for p, ic in mem])
    try:
        for k, (p, ic) in enumerate(mem):
            _load(B, B.ann_ensemble_member(ens, k), ic)
        B.ann_ensemble_step(ens, 6)           # all members in parallel branches
        B.ann_ensemble_set_groups(ens, 2)     # two branches, members in sequence within each
        B.ann_ensemble_step(ens, 5)
        B.ann_ensemble_set_groups(ens, 1)
        B.ann_ensemble_step(ens, 3)
        groups, ms = B.ann_ensemble_autotune(ens, 3)
        assert 1 <= groups <= len(mem) and ms > 0.0
        B.ann_ensemble_step(ens, 4)
        resorts = []
        for k, (p, ic) in enumerate(mem):
            ctx = B.ann_ensemble_member(ens, k)
            d = B.ann_get_diagnostics(ctx)
            resorts.append(d["resorts"])
            got = _state(B, ctx, ic["n"])
            solo = B.ann_create(gpu_params(B, p, ic["n"]))
            try:
                _load(B, solo, ic)
                B.ann_step(solo, d["step"])
                want = _state(B, solo, ic["n"])
            finally:
                B.ann_destroy(solo)
            for f in got:
                assert np.array_equal(got[f], want[f]), (k, f)
        assert resorts[3] >= 4 and resorts[0] == 1, resorts   # the fast member re-sorted on its own
    finally:
        B.ann_ensemble_destroy(ens)


def test_failing_member_is_named_and_others_advance(B):
    mem = _members()[:3]
    ens = B.ann_ensemble_create([gpu_params(B, p, ic["n"]) for p, ic in mem])
    try:
        for k, (p, ic) in enumerate(mem):
            _load(B, B.ann_ensemble_member(ens, k), ic)
        with pytest.raises(B.AnnError):
            B.ann_ensemble_step(ens, -1)
        # member 1: a velocity beyond FP32 range (accepted on load as FP64) makes its positions
        # non-finite in the first step; its kernels stop, the other members' do not
        ic = dict(mem[1][1])
        ic["ux"] = np.full(ic["n"], 1e300)
        _load(B, B.ann_ensemble_member(ens, 1), ic)
        with pytest.raises(B.AnnError) as e:
            B.ann_ensemble_step(ens, 2)
        assert e.value.status == -6 and "member 1" in str(e.value)
        for k in (0, 2):
            d = B.ann_get_diagnostics(B.ann_ensemble_member(ens, k))
            assert d["step"] == 2 and d["error_bits"] == 0
        # a member whose load was rejected holds no particles: the ensemble refuses to step
        bad = dict(mem[1][1])
        bad["x"] = bad["x"].copy()
        bad["x"][0] = np.nan
        with pytest.raises(B.AnnError):
            _load(B, B.ann_ensemble_member(ens, 1), bad)
        with pytest.raises(B.AnnError) as e:
            B.ann_ensemble_step(ens, 1)
        assert e.value.status == -9 and "member 1" in str(e.value)
        _load(B, B.ann_ensemble_member(ens, 1), mem[1][1])
        B.ann_ensemble_step(ens, 2)
        steps = [B.ann_get_diagnostics(B.ann_ensemble_member(ens, k))["step"] for k in range(3)]
        assert steps == [4, 2, 4], steps
    finally:
        B.ann_ensemble_destroy(ens)


def test_benchmark_ensemble_members_match_solo_runs(B):
    """The benchmark's 64-member ensemble (sides uniform in [128, 512], 7.4M particles, autotuned
    grouping) after a few steps: sampled members, the smallest and the largest among them, are
    bit-identical to the same members stepped alone."""
    import math

    import sph_inputs as si

    u = si.uniform53(2021, 3 * 64).reshape(64, 3)   # the benchmark's member recipe
    spec = [(int(round(128 + 384 * u[k, 0])), math.exp(math.log(0.01) + u[k, 1] * (math.log(0.2) - math.log(0.01))),
             0.01 + 0.07 * u[k, 2]) for k in range(64)]
    plist = [B.ann_default_params(n=nx * nx, h=1.3 / nx, zeta=z, K=K, dt_mode=1) for nx, z, K in spec]
    ics = [si.jittered_lattice(nx, seed=100 + k) for k, (nx, _, _) in enumerate(spec)]
    ens = B.ann_ensemble_create(plist)
    try:
        for k, ic in enumerate(ics):
            _load(B, B.ann_ensemble_member(ens, k), ic)
        B.ann_ensemble_autotune(ens, 2)
        B.ann_ensemble_step(ens, 3)
        sides = [s[0] for s in spec]
        sample = sorted({sides.index(min(sides)), sides.index(max(sides)), 0, 17, 33, 50, 63})
        for k in sample:
            ctx = B.ann_ensemble_member(ens, k)
            steps = B.ann_get_diagnostics(ctx)["step"]
            got = _state(B, ctx, ics[k]["n"])
            solo = B.ann_create(plist[k])
            try:
                _load(B, solo, ics[k])
                B.ann_step(solo, steps)
                want = _state(B, solo, ics[k]["n"])
            finally:
                B.ann_destroy(solo)
            for f in got:
                assert np.array_equal(got[f], want[f]), (k, f)
    finally:
        B.ann_ensemble_destroy(ens)
