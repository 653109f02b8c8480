"""The C-ABI library loads and exports every entry point ``include/ann.h`` declares; host-only
calls (defaults, validation, grid sizing) behave as the header states.  No GPU needed: nothing
here launches a kernel."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ann.h")


@pytest.fixture(scope="module")
def B():
    from paper_2108_08919_gb300 import build, binding

    build.build()
    return binding


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ann_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(B):
    names = _declared()
    assert len(names) >= 18
    lib = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert all(hasattr(B, n) for n in names)


def test_struct_layouts_match_header(B, tmp_path):
    """ctypes mirrors of the header structs have the C compiler's sizes and field offsets."""
    import subprocess
    structs = {"ann_params": B.ann_params, "ann_grid": B.ann_grid, "ann_diag": B.ann_diag,
               "ann_allocator": B.ann_allocator}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ann.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {cname}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in structs.items():
        assert got[(sname, "sizeof")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_version_and_status_strings(B):
    assert B.ann_version() == 1
    assert B.ann_status_string(0) == "ok"
    assert "neighbour" in B.ann_status_string(-5)
    assert B.ann_status_string(-999) == "unknown status"
    assert B.ann_kernel_count() == 10
    names = [B.ann_kernel_name(k) for k in range(10)]
    assert names == ["predict", "cell_keys", "cell_scan", "cell_scatter", "cell_order",
                     "pass_a_resort", "pass_a", "pass_b", "pass_c", "pass_d"]


def test_default_params_are_the_paper_setup(B):
    p = B.ann_default_params()
    assert p.n == 4096 and p.L == 1.0 and p.h == pytest.approx(1.3 / 64)
    assert (p.dt, p.rho0, p.eta, p.Gamma, p.lambda_, p.A, p.C, p.K, p.zeta) == \
        (1e-4, 1.0, 1.0, 0.34, 0.7, 0.0, 1.0, 0.04, 0.05)
    assert p.gamma_eos == 7.0 and p.beta == 1.0 and p.c_shift == pytest.approx(1 / 3)
    assert B.ann_validate_params(p) == 0


@pytest.mark.parametrize("field,value", [
    ("n", 0), ("L", -1.0), ("h", 0.0), ("dt", float("nan")), ("rho0", 0.0), ("eta", -1.0),
    ("beta", 1.5), ("apd", 2), ("momentum_mode", 7), ("dt_mode", 3), ("zeta", float("inf")),
    ("h", 0.2),   # 3h = 0.6: fewer than three cells across the box
])
def test_validation_rejects(B, field, value):
    p = B.ann_default_params()
    setattr(p, field, value)
    assert B.ann_validate_params(p) == -1


def test_particle_count_limit(B):
    """n up to 2^29 (every per-particle index of the kernels stays in int32); one more is refused."""
    for n, status in ((1 << 29, 0), ((1 << 29) + 1, -1)):
        p = B.ann_default_params(n=n, h=1.3 / math.sqrt(n))
        assert B.ann_validate_params(p) == status, n


def test_validation_rejects_crowded_support(B):
    p = B.ann_default_params()
    p.h = 2.0 / 64   # pi (6 dx)^2 = 113 expected neighbours > list capacity
    assert B.ann_validate_params(p) == -1


def test_grid_info(B):
    # cells are at least 3h (1 + 0.02) wide, the radius of the candidate lists
    for nx, nc in ((64, 16), (256, 64), (1024, 257)):
        p = B.ann_default_params(n=nx * nx, h=1.3 / nx)
        g = B.ann_grid_info(p)
        assert g.cells_per_side == nc
        assert g.cell_size >= 3 * p.h * 1.02
        assert g.tiles_per_side == math.ceil(nc / 4)
        assert g.expected_neighbors == pytest.approx(math.pi * 3.9 ** 2)
        assert g.device_bytes > nx * nx * 200


def test_stable_dt(B):
    p = B.ann_default_params(n=256 * 256, h=1.3 / 256, dt_mode=1)
    g = B.ann_grid_info(p)
    assert g.dt_effective == pytest.approx(0.125 * (1.3 / 256) ** 2 / 1.0)
    p.dt_mode = 0
    assert B.ann_grid_info(p).dt_effective == 1e-4


def test_dt_check_mode_and_new_status_codes(B):
    p = B.ann_default_params(dt_mode=2)   # ANN_DT_CHECK: dt as given, checked every step
    assert B.ann_validate_params(p) == 0
    assert B.ann_grid_info(p).dt_effective == p.dt
    assert "timed out" in B.ann_status_string(-12)
    assert "CFL" in B.ann_status_string(-13)


def test_allocator_callbacks_are_validated_before_any_device_call(B):
    a = B.ann_allocator()   # both callbacks NULL
    with pytest.raises(B.AnnError) as e:
        B.ann_create_with_allocator(B.ann_default_params(), a)
    assert e.value.status == -1
    with pytest.raises(B.AnnError) as e:   # bad parameters are reported first
        B.ann_create_with_allocator(B.ann_default_params(n=0), None)
    assert e.value.status == -1


def test_bounded_wait_self_test_rejects_bad_limits(B):
    assert B.ann_check_bounded_wait(0) == -1
    assert B.ann_check_bounded_wait(1 << 21) == -1


def test_create_without_gpu_reports_not_available(B):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(B.AnnError) as e:
        B.ann_create(B.ann_default_params())
    assert e.value.status == -10


def test_state_transfer_arguments_are_checked_on_the_host(B):
    """The binding rejects state arrays of the wrong dtype, length or mixture before any call."""
    import numpy as np

    n = 16
    good = {"X": np.zeros(n), "Y": np.zeros(n), "UX": np.zeros(n, np.float32), "UY": np.zeros(n, np.float32),
            "Q11": np.zeros(n, np.float32), "Q12": np.zeros(n, np.float32)}
    for bad in ({**good, "UX": np.zeros(n)},                     # float64 where float32 is kept
                {**good, "Q12": np.zeros(n - 1, np.float32)},   # short
                {k: v for k, v in good.items() if k != "Y"}):   # a required field missing
        with pytest.raises(ValueError):
            B.ann_update_state(None, bad)
        with pytest.raises(ValueError):
            B.ann_set_state(None, bad)
    with pytest.raises(ValueError):
        B.ann_get_state(None, n, out={"X": np.zeros(n, np.float32)})
