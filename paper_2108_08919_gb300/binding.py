"""Python binding of the C-ABI in ``include/ann.h`` (ctypes, argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but convert
arguments: numpy arrays are passed as host pointers, CUDA tensors (anything with ``data_ptr()`` and
``is_cuda``) as device pointers.  All arithmetic of the method runs in the CUDA library
``_lib/libann.so``; if that library is missing this module raises instead of falling back to any
other implementation.  Negative status codes raise :class:`AnnError`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libann.so")

MAX_NEIGHBORS = 64
MOMENTUM_PAPER, MOMENTUM_CONSERVATIVE = 0, 1
DT_FIXED, DT_STABLE = 0, 1

FIELDS = ["X", "Y", "UX", "UY", "Q11", "Q12", "DRHO", "AX", "AY", "SUMW", "V", "B11", "B12", "B22",
          "K", "DRHO_HALF", "DRHO_HAT", "P", "DIVQX", "DIVQY", "NNBR", "GRADU_XX", "GRADU_XY",
          "GRADU_YX", "GRADU_YY", "LAPQ11", "LAPQ12", "APDX", "APDY", "QRATE11", "QRATE12"]
FIELD_ID = {name: k for k, name in enumerate(FIELDS)}


def field_dtype(name: str):
    if name in ("X", "Y"):
        return np.float64
    if name == "NNBR":
        return np.int32
    return np.float32


class ann_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_double) for k in (
        "L", "h", "dt", "rho0", "eta", "Gamma", "lambda_", "A", "B", "C", "K", "zeta", "gamma_eos",
        "beta", "c0_min", "c_shift")] + [(k, ctypes.c_int32) for k in (
        "apd", "momentum_mode", "q_new_in_momentum", "dt_mode", "elastic_stress")] + [
        ("reserved", ctypes.c_int32 * 3)]


class ann_grid(ctypes.Structure):
    _fields_ = [("cells_per_side", ctypes.c_int32), ("tiles_per_side", ctypes.c_int32),
                ("cell_size", ctypes.c_double), ("dt_effective", ctypes.c_double),
                ("expected_neighbors", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class ann_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_int64), ("momentum", ctypes.c_double * 2),
                ("kinetic_energy", ctypes.c_double), ("max_speed", ctypes.c_double),
                ("c0", ctypes.c_double), ("mass", ctypes.c_double), ("mean_q", ctypes.c_double),
                ("nbr_mean", ctypes.c_double), ("nbr_min", ctypes.c_int32),
                ("nbr_max", ctypes.c_int32), ("min_det_alpha", ctypes.c_double),
                ("error_bits", ctypes.c_uint32), ("resorts", ctypes.c_int32),
                ("band_checks", ctypes.c_uint64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "momentum"}
        d["momentum"] = (self.momentum[0], self.momentum[1])
        return d


class ann3_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_double) for k in (
        "L", "h", "dt", "rho0", "eta", "Gamma", "lambda_", "A", "B", "C", "K", "zeta", "gamma_eos",
        "beta", "c0_min", "c_shift")] + [("apd", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


FIELDS3 = {"POS": (0, 3), "U": (1, 3), "Q": (2, 5), "RHO": (3, 1), "A": (4, 3), "SUMW": (5, 1),
           "GRADU": (6, 9), "LAPQ": (7, 5), "QRATE": (8, 5), "P": (9, 1), "NNBR": (10, 1)}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class ann_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("user", ctypes.c_void_p)]


class AnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_P = ctypes.POINTER


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with "
                           "paper_2108_08919_gb300.build.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    sig = {
        "ann_version": (i32, []),
        "ann_status_string": (ctypes.c_char_p, [i32]),
        "ann_default_params": (i32, [_P(ann_params)]),
        "ann_validate_params": (i32, [_P(ann_params)]),
        "ann_grid_info": (i32, [_P(ann_params), _P(ann_grid)]),
        "ann_create": (i32, [_P(ann_params), _P(vp)]),
        "ann_create_with_allocator": (i32, [_P(ann_params), _P(ann_allocator), _P(vp)]),
        "ann_check_bounded_wait": (i32, [ctypes.c_uint32]),
        "ann_destroy": (None, [vp]),
        "ann_set_stream": (i32, [vp, vp]),
        "ann_set_particles": (i32, [vp, i64, dp, dp, dp, dp, dp, dp, dp, i32]),
        "ann_step": (i32, [vp, i64]),
        "ann_step_profile": (i32, [vp, i64, _P(ctypes.c_double)]),
        "ann_kernel_count": (i32, []),
        "ann_kernel_name": (ctypes.c_char_p, [i32]),
        "ann_set_record": (i32, [vp, i32]),
        "ann_get_field": (i32, [vp, i32, vp, i64, i32]),
        "ann_get_state": (i32, [vp] * 10 + [i32]),
        "ann_update_state": (i32, [vp] * 10 + [i32]),
        "ann_set_state": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, vp, i32]),
        "ann_get_diagnostics": (i32, [vp, _P(ann_diag)]),
        "ann_get_neighbors": (i32, [vp, _P(ctypes.c_int64), _P(ctypes.c_int32), i64]),
        "ann_save_state": (i32, [vp, ctypes.c_char_p]),
        "ann_load_state": (i32, [vp, ctypes.c_char_p]),
        "ann_last_error": (ctypes.c_char_p, [vp]),
        "ann_velocity_moments_noalloc": (i32, [vp, vp, vp, ctypes.c_double, i64, vp, vp]),
        "ann_fp32_fma_peak": (i32, [vp, _P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_int32)]),
        "ann_grid_fields": (i32, [vp, i32, vp, i32]),
        "ann_spectrum_shells": (i32, [i32]),
        "ann_energy_spectrum": (i32, [vp, i32, _P(ctypes.c_double), i32]),
        "ann_spectrum_slope": (i32, [_P(ctypes.c_double), i32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _P(ctypes.c_double)]),
        "ann_vorticity_correlation": (i32, [vp, i32, i32, _P(ctypes.c_double), _P(ctypes.c_double)]),
        "ann_defects": (i32, [vp, i32, _P(ctypes.c_int64), _P(ctypes.c_int8)]),
        "ann_set_colors": (i32, [vp, vp, i64, i32]),
        "ann_mixing_index": (i32, [vp, i32, _P(ctypes.c_double), _P(ctypes.c_double)]),
        "ann_get_unwrapped": (i32, [vp, _P(ctypes.c_int64), i64, _P(ctypes.c_double)]),
        "ann_bf16_gemm": (i32, [vp, i32, vp, i32, vp, i32, i64, vp, i32, vp, i32, i32, vp]),
        "ann_bf16_gemm_tn": (i32, [vp, i32, vp, i32, i64, vp, vp]),
        "ann_surrogate_create": (i32, [i64, _P(vp)]),
        "ann_surrogate_destroy": (None, [vp]),
        "ann_surrogate_set_params": (i32, [vp, _P(ctypes.c_float)]),
        "ann_surrogate_init": (i32, [vp, ctypes.c_uint64]),
        "ann_surrogate_get_params": (i32, [vp, _P(ctypes.c_float)]),
        "ann_surrogate_set_scales": (i32, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32]),
        "ann_surrogate_load": (i32, [vp, vp, _P(ctypes.c_float)]),
        "ann_surrogate_forward": (i32, [vp, _P(ctypes.c_float)]),
        "ann_surrogate_euler": (i32, [vp, _P(ctypes.c_float)]),
        "ann_surrogate_gradients": (i32, [vp, _P(ctypes.c_float), _P(ctypes.c_double), _P(ctypes.c_float)]),
        "ann_surrogate_adam": (i32, [vp, ctypes.c_double]),
        "ann_surrogate_jump": (i32, [vp, vp, _P(ctypes.c_float)]),
        "ann_surrogate_advance": (i32, [vp, vp, vp, i32, i32, ctypes.c_double, vp]),
        "ann_surrogate_set_velocity_correction": (i32, [vp, i32]),
        "ann_surrogate_last_error": (ctypes.c_char_p, [vp]),
        "ann_ensemble_create": (i32, [_P(ann_params), i32, _P(vp)]),
        "ann_ensemble_destroy": (None, [vp]),
        "ann_ensemble_member": (i32, [vp, i32, _P(vp)]),
        "ann_ensemble_step": (i32, [vp, i64]),
        "ann_ensemble_set_groups": (i32, [vp, i32]),
        "ann_ensemble_autotune": (i32, [vp, i32, _P(ctypes.c_int32), _P(ctypes.c_double)]),
        "ann_ensemble_last_error": (ctypes.c_char_p, [vp]),
        "ann3_default_params": (i32, [_P(ann3_params)]),
        "ann3_create": (i32, [_P(ann3_params), _P(vp)]),
        "ann3_destroy": (None, [vp]),
        "ann3_set_particles": (i32, [vp, i64, dp, dp, dp, dp, dp, dp]),
        "ann3_step": (i32, [vp, i64]),
        "ann3_get_field": (i32, [vp, i32, dp]),
        "ann3_get_status": (i32, [vp, _P(ctypes.c_int64), _P(ctypes.c_uint32), _P(ctypes.c_int64)]),
        "ann3_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, ctx=None, what: str = ""):
    if status < 0:
        detail = ""
        if ctx is not None:
            detail = lib().ann_last_error(ctx).decode()
        text = lib().ann_status_string(status).decode()
        raise AnnError(status, f"{what}: {text}" + (f" ({detail})" if detail else ""))
    return status


def _ptr(a):
    """(pointer, is_device, keepalive) of a numpy array or CUDA tensor; None passes NULL."""
    if a is None:
        return None, None, None
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        return ctypes.c_void_p(a.data_ptr()), True, a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data_as(ctypes.c_void_p), False, arr


# ------------------------------------------------------------------------------------------------
# entry points
# ------------------------------------------------------------------------------------------------

def ann_version() -> int:
    return lib().ann_version()


def ann_status_string(status: int) -> str:
    return lib().ann_status_string(status).decode()


def ann_default_params(**overrides) -> ann_params:
    p = ann_params()
    _check(lib().ann_default_params(ctypes.byref(p)), what="ann_default_params")
    names = {f[0] for f in ann_params._fields_}
    for k, v in overrides.items():
        k = "lambda_" if k == "lambda" else k
        if k not in names or k == "reserved":
            raise TypeError(f"ann_params has no field {k!r}")
        setattr(p, k, v)
    return p


def ann_validate_params(p: ann_params) -> int:
    return lib().ann_validate_params(ctypes.byref(p))


def ann_grid_info(p: ann_params) -> ann_grid:
    g = ann_grid()
    _check(lib().ann_grid_info(ctypes.byref(p), ctypes.byref(g)), what="ann_grid_info")
    return g


def ann_create(p: ann_params) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().ann_create(ctypes.byref(p), ctypes.byref(ctx)), what="ann_create")
    return ctx


# allocators handed to ann_create_with_allocator, kept alive (with their ctypes callbacks) until
# the context that uses them is destroyed
_ctx_allocators = {}


def ann_create_with_allocator(p: ann_params, a) -> ctypes.c_void_p:
    """``a``: an ann_allocator (see torch_allocator), or None for cudaMalloc."""
    ctx = ctypes.c_void_p()
    _check(lib().ann_create_with_allocator(ctypes.byref(p), ctypes.byref(a) if a is not None else None,
                                           ctypes.byref(ctx)), what="ann_create_with_allocator")
    if a is not None:
        _ctx_allocators[ctx.value] = a
    return ctx


def torch_allocator() -> ann_allocator:
    """An ann_allocator that takes device memory from PyTorch's CUDA caching allocator, on the
    context's own stream (memory then counts in torch.cuda.memory_allocated)."""
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except RuntimeError:
            return None

    def release(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ann_allocator(_ALLOC_FN(alloc), _RELEASE_FN(release), None)


def ann_destroy(ctx) -> None:
    if ctx:
        lib().ann_destroy(ctx)
        _ctx_allocators.pop(getattr(ctx, "value", ctx), None)


def ann_set_stream(ctx, stream) -> None:
    """``stream``: an integer cudaStream_t handle or an object with ``cuda_stream``."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().ann_set_stream(ctx, ctypes.c_void_p(int(handle) if handle else 0)), ctx, "ann_set_stream")


def ann_set_particles(ctx, x, y, ux, uy, q11, q12, rho=None) -> None:
    """FP64 arrays (numpy on the host, or CUDA tensors on the device) in particle-ID order."""
    arrs = [_ptr(a) for a in (x, y, ux, uy, q11, q12, rho)]
    dev = {d for _, d, _ in arrs if d is not None}
    if len(dev) != 1:
        raise ValueError("inputs must all be host arrays or all CUDA tensors")
    n = int(len(arrs[0][2]) if not hasattr(arrs[0][2], "numel") else arrs[0][2].numel())
    _check(lib().ann_set_particles(ctx, n, *[a[0] for a in arrs], int(dev.pop())), ctx,
           "ann_set_particles")


def ann_set_state(ctx, state: dict) -> None:
    """Load the state as ann_get_state returns it: a dict with X, Y (float64) and UX, UY, Q11, Q12
    and optionally DRHO (float32), all numpy arrays or all CUDA tensors, in particle-ID order."""
    ptrs, dev, n = _state_ptrs(state, STATE_FIELDS, ("X", "Y", "UX", "UY", "Q11", "Q12"), "state")
    _check(lib().ann_set_state(ctx, n, *ptrs, 1 if dev else 0), ctx, "ann_set_state")


def ann_step(ctx, nsteps: int) -> None:
    _check(lib().ann_step(ctx, int(nsteps)), ctx, "ann_step")


def ann_kernel_count() -> int:
    return lib().ann_kernel_count()


def ann_kernel_name(k: int) -> str:
    return lib().ann_kernel_name(k).decode()


def ann_step_profile(ctx, nsteps: int) -> dict:
    """Per-kernel device time (ms, summed over the steps), from CUDA events around each kernel."""
    k = ann_kernel_count()
    ms = (ctypes.c_double * k)()
    _check(lib().ann_step_profile(ctx, int(nsteps), ms), ctx, "ann_step_profile")
    return {ann_kernel_name(i): ms[i] for i in range(k)}


def ann_set_record(ctx, on: bool) -> None:
    _check(lib().ann_set_record(ctx, int(bool(on))), ctx, "ann_set_record")


def ann_get_field(ctx, field: str, n: int, out=None):
    """Field ``field`` (a name of FIELDS) in particle-ID order: a new numpy array, or written into
    ``out`` (numpy array or CUDA tensor of the field's dtype and length n)."""
    dt = field_dtype(field)
    if out is None:
        out = np.empty(n, dtype=dt)
    if hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
        ptr, dev, nbytes = out.data_ptr(), 1, out.numel() * out.element_size()
    else:
        if out.dtype != dt or not out.flags.c_contiguous:
            raise ValueError(f"out must be a contiguous {np.dtype(dt).name} array")
        ptr, dev, nbytes = out.ctypes.data, 0, out.nbytes
    _check(lib().ann_get_field(ctx, FIELD_ID[field], ctypes.c_void_p(ptr), nbytes, dev), ctx,
           f"ann_get_field({field})")
    return out


STATE_FIELDS = ("X", "Y", "UX", "UY", "Q11", "Q12", "DRHO")
FULL_STATE = STATE_FIELDS + ("AX", "AY")   # with the last step's acceleration


def _state_ptrs(arrays: dict, names, required, what: str):
    """Pointers (None where absent) of host arrays or CUDA tensors of the fields' dtypes, and whether
    they are on the device; every array holds the same number of values, which is returned."""
    ptrs, dev, n = [], None, None
    for f in names:
        a = arrays.get(f)
        if a is None:
            if f in required:
                raise ValueError(f"{what}[{f!r}] is required")
            ptrs.append(None)
            continue
        is_dev = bool(getattr(a, "is_cuda", False))
        dev = is_dev if dev is None else dev
        if is_dev != dev:
            raise ValueError(f"{what} must be all host arrays or all CUDA tensors")
        size = a.numel() if is_dev else a.size
        n = size if n is None else n
        want = np.dtype(field_dtype(f))
        if is_dev:
            if a.element_size() != want.itemsize or size != n or not a.is_contiguous():
                raise ValueError(f"{what}[{f!r}] must be a contiguous {want.name} tensor of n values")
            ptrs.append(ctypes.c_void_p(a.data_ptr()))
        else:
            if a.dtype != want or size != n or not a.flags.c_contiguous:
                raise ValueError(f"{what}[{f!r}] must be a contiguous {want.name} array of n values")
            ptrs.append(ctypes.c_void_p(a.ctypes.data))
    return ptrs, bool(dev), n


def ann_get_state(ctx, n: int, out=None) -> dict:
    """The state fields X, Y (float64), UX, UY, Q11, Q12, DRHO and the last step's AX, AY (float32)
    in particle-ID order, in one call: new numpy arrays, or written into ``out`` (a dict of numpy
    arrays, or of CUDA tensors, with some or all of those names).  Numpy arrays in page-locked
    memory (e.g. ``torch.empty(n).pin_memory().numpy()``) are written by the device directly."""
    if out is None:
        out = {f: np.empty(n, dtype=field_dtype(f)) for f in FULL_STATE}
    ptrs, dev, m = _state_ptrs(out, FULL_STATE, (), "out")
    if m is not None and m < n:
        raise ValueError("out arrays must hold n values")
    _check(lib().ann_get_state(ctx, *ptrs, 1 if dev else 0), ctx, "ann_get_state")
    return out


def ann_update_state(ctx, state: dict) -> None:
    """Replace the present state, keeping the step count and the cell structure (see the header): a
    dict with the names of ann_get_state (DRHO, AX, AY optional), all numpy arrays or all CUDA
    tensors, in particle-ID order.  Page-locked numpy arrays are read by the device directly."""
    ptrs, dev, _ = _state_ptrs(state, FULL_STATE, ("X", "Y", "UX", "UY", "Q11", "Q12"), "state")
    _check(lib().ann_update_state(ctx, *ptrs, 1 if dev else 0), ctx, "ann_update_state")


def ann_get_diagnostics(ctx) -> dict:
    d = ann_diag()
    _check(lib().ann_get_diagnostics(ctx, ctypes.byref(d)), ctx, "ann_get_diagnostics")
    return d.as_dict()


def ann_get_neighbors(ctx, n: int):
    """CSR neighbour lists of the current positions: (rowptr int64[n+1], cols int32[nnz])."""
    rowptr = np.zeros(n + 1, dtype=np.int64)
    L = lib()
    _check(L.ann_get_neighbors(ctx, rowptr.ctypes.data_as(_P(ctypes.c_int64)), None, 0), ctx,
           "ann_get_neighbors")
    cols = np.zeros(max(int(rowptr[-1]), 1), dtype=np.int32)
    _check(L.ann_get_neighbors(ctx, rowptr.ctypes.data_as(_P(ctypes.c_int64)),
                               cols.ctypes.data_as(_P(ctypes.c_int32)), cols.size), ctx,
           "ann_get_neighbors")
    return rowptr, cols[: int(rowptr[-1])]


def ann_save_state(ctx, path: str) -> None:
    _check(lib().ann_save_state(ctx, os.fsencode(path)), ctx, "ann_save_state")


def ann_load_state(ctx, path: str) -> None:
    _check(lib().ann_load_state(ctx, os.fsencode(path)), ctx, "ann_load_state")


def ann_last_error(ctx) -> str:
    return lib().ann_last_error(ctx).decode()


def ann_fp32_fma_peak(stream=None) -> dict:
    """Measured FP32 FMA throughput of the current device: {"scalar": TFLOP/s, "pair": TFLOP/s,
    "sms": SM count}."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
    _check(lib().ann_fp32_fma_peak(ctypes.c_void_p(int(handle) if handle else 0), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(n)), None, "ann_fp32_fma_peak")
    return {"scalar": a.value, "pair": b.value, "sms": n.value}


NOALLOC_MAX_N = 2097152


def ann_velocity_moments_noalloc(ux, uy, out, mass=None, m0=1.0, stream=None) -> None:
    """Momentum, mean kinetic energy and peak speed of a device velocity field, written into the
    CUDA tensor ``out`` (4 float64) without any device allocation; ``ux``, ``uy`` (and ``mass``)
    are contiguous float32 CUDA tensors of one length n, all on one device.  Asynchronous on
    ``stream`` (default: the legacy default stream).  The arguments are checked here, before any
    C call: a shorter ``uy`` or ``mass`` or a smaller ``out`` would make the kernel read or write
    past the end of an allocation."""
    import torch

    named = [("ux", ux), ("uy", uy), ("out", out)] + ([("mass", mass)] if mass is not None else [])
    for name, a in named:
        if not (isinstance(a, torch.Tensor) and a.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    n = ux.numel()
    for name, a in named:
        if name == "out":
            if a.dtype != torch.float64 or a.numel() < 4:
                raise ValueError("out must be a float64 tensor of at least 4 elements")
        elif a.dtype != torch.float32 or a.numel() != n:
            raise ValueError(f"{name} must be a float32 tensor of {n} elements (the length of ux)")
    if len({a.device for _, a in named}) != 1:
        raise ValueError("ux, uy, out and mass must be on one device")
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
    with torch.cuda.device(ux.device):
        st = lib().ann_velocity_moments_noalloc(
            ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(uy.data_ptr()),
            ctypes.c_void_p(mass.data_ptr()) if mass is not None else None, float(m0), int(n),
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(int(handle) if handle else 0))
    _check(st, None, "ann_velocity_moments_noalloc")


# ------------------------------------------------------------------ flow diagnostics (§5)

GRID_MAX = 2048
MAX_COLORS = 16
_dptr = lambda a: a.ctypes.data_as(_P(ctypes.c_double))  # noqa: E731


def ann_grid_fields(ctx, M: int, out=None):
    """Gridded present state, shape (5, M, M): ux, uy, q11, q12, Shepard weight sum ([iy, ix]).
    ``out``: optional float64 numpy array or CUDA tensor of 5 M^2 elements."""
    if out is None:
        out = np.empty((5, M, M), dtype=np.float64)
    if hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
        ptr, dev = out.data_ptr(), 1
    else:
        if out.dtype != np.float64 or out.size != 5 * M * M or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of 5 M^2 elements")
        ptr, dev = out.ctypes.data, 0
    _check(lib().ann_grid_fields(ctx, int(M), ctypes.c_void_p(ptr), dev), ctx, "ann_grid_fields")
    return out


def ann_spectrum_shells(M: int) -> int:
    return _check(lib().ann_spectrum_shells(int(M)), None, "ann_spectrum_shells")


def ann_energy_spectrum(ctx, M: int):
    """Shell energies E_n of the gridded velocity, n = 0 .. shells - 1; shell n is the wavenumber
    w_n = 2 pi n / L."""
    ns = ann_spectrum_shells(M)
    E = np.zeros(ns)
    _check(lib().ann_energy_spectrum(ctx, int(M), _dptr(E), ns), ctx, "ann_energy_spectrum")
    return E


def ann_spectrum_slope(E, L: float, w1: float, w2: float) -> float:
    E = np.ascontiguousarray(E, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib().ann_spectrum_slope(_dptr(E), E.size, float(L), float(w1), float(w2), ctypes.byref(out)),
           None, "ann_spectrum_slope")
    return out.value


def ann_vorticity_correlation(ctx, M: int, all_origins: bool = True):
    """(C[0..M/2], (zero-crossing length, 0.2-max length))."""
    C = np.zeros(M // 2 + 1)
    lengths = np.zeros(2)
    _check(lib().ann_vorticity_correlation(ctx, int(M), int(bool(all_origins)), _dptr(C), _dptr(lengths)), ctx,
           "ann_vorticity_correlation")
    return C, (float(lengths[0]), float(lengths[1]))


def ann_defects(ctx, M: int, with_map: bool = False):
    """(counts [m = +1, m = -1, |m| >= 2], winding map int8 [M, M] or None)."""
    counts = np.zeros(3, dtype=np.int64)
    m = np.zeros((M, M), dtype=np.int8) if with_map else None
    _check(lib().ann_defects(ctx, int(M), counts.ctypes.data_as(_P(ctypes.c_int64)),
                             m.ctypes.data_as(_P(ctypes.c_int8)) if with_map else None), ctx, "ann_defects")
    return counts, m


def ann_set_colors(ctx, colors) -> None:
    """Colour of each particle by ID: uint8 numpy array or CUDA tensor of n values."""
    if hasattr(colors, "data_ptr") and getattr(colors, "is_cuda", False):
        ptr, dev, n = colors.data_ptr(), 1, colors.numel()
    else:
        colors = np.ascontiguousarray(colors, dtype=np.uint8)
        ptr, dev, n = colors.ctypes.data, 0, colors.size
    _check(lib().ann_set_colors(ctx, ctypes.c_void_p(ptr), int(n), dev), ctx, "ann_set_colors")


def ann_mixing_index(ctx, G: int):
    """(intensity of segregation I, per-colour I_s with NaN for absent or sole colours)."""
    I = ctypes.c_double()
    per = np.zeros(MAX_COLORS)
    _check(lib().ann_mixing_index(ctx, int(G), ctypes.byref(I), _dptr(per)), ctx, "ann_mixing_index")
    return I.value, per


def ann_get_unwrapped(ctx, ids):
    """Unwrapped positions (k, 2) of the particles with the given IDs."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    xy = np.zeros((ids.size, 2))
    _check(lib().ann_get_unwrapped(ctx, ids.ctypes.data_as(_P(ctypes.c_int64)), ids.size, _dptr(xy)), ctx,
           "ann_get_unwrapped")
    return xy


# ------------------------------------------------------------------ batched ensemble

ENSEMBLE_MAX = 256


def _echeck(status: int, ens, what: str):
    if status < 0:
        detail = lib().ann_ensemble_last_error(ens).decode() if ens is not None else ""
        text = lib().ann_status_string(status).decode()
        raise AnnError(status, f"{what}: {text}" + (f" ({detail})" if detail else ""))
    return status


def ann_ensemble_create(params) -> ctypes.c_void_p:
    """An ensemble of len(params) members (a list of ann_params)."""
    arr = (ann_params * len(params))(*params)
    ens = ctypes.c_void_p()
    _echeck(lib().ann_ensemble_create(arr, len(params), ctypes.byref(ens)), None, "ann_ensemble_create")
    return ens


def ann_ensemble_destroy(ens) -> None:
    lib().ann_ensemble_destroy(ens)


def ann_ensemble_member(ens, k: int) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _echeck(lib().ann_ensemble_member(ens, int(k), ctypes.byref(ctx)), ens, "ann_ensemble_member")
    return ctx


def ann_ensemble_step(ens, nsteps: int) -> None:
    _echeck(lib().ann_ensemble_step(ens, int(nsteps)), ens, "ann_ensemble_step")


def ann_ensemble_set_groups(ens, groups: int) -> None:
    _echeck(lib().ann_ensemble_set_groups(ens, int(groups)), ens, "ann_ensemble_set_groups")


def ann_ensemble_autotune(ens, trial_steps: int):
    """(chosen grouping, ms per ensemble step)."""
    g = ctypes.c_int32()
    ms = ctypes.c_double()
    _echeck(lib().ann_ensemble_autotune(ens, int(trial_steps), ctypes.byref(g), ctypes.byref(ms)), ens,
            "ann_ensemble_autotune")
    return g.value, ms.value


def ann_ensemble_last_error(ens) -> str:
    return lib().ann_ensemble_last_error(ens).decode()


# ------------------------------------------------------------------ BF16 tensor-core GEMMs


def _dev(t):
    if t is None:
        return None
    if not (hasattr(t, "data_ptr") and getattr(t, "is_cuda", False)):
        raise ValueError("GEMM operands must be CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def ann_bf16_gemm(A1, B, C, A2=None, bias=None, relu=False, accumulate=False, stream=None) -> None:
    """C = act([A1 | A2] B^T + bias) with bfloat16 CUDA tensors A1 (rows x K1), A2 (rows x K2),
    B (N x K); C (rows x N) bfloat16 or float32 (accumulate adds to a float32 C)."""
    rows, K1 = A1.shape
    K2 = A2.shape[1] if A2 is not None else 0
    N = B.shape[0]
    c_bf16 = int(str(C.dtype).endswith("bfloat16"))
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
    st = lib().ann_bf16_gemm(_dev(A1), K1, _dev(A2), K2, _dev(B), N, rows, _dev(bias), int(bool(relu)), _dev(C),
                             c_bf16, int(bool(accumulate)), ctypes.c_void_p(int(handle) if handle else 0))
    _check(st, None, "ann_bf16_gemm")


def ann_bf16_gemm_tn(A, B, C, stream=None) -> None:
    """C += A^T B with bfloat16 CUDA tensors A (rows x K), B (rows x N) and float32 C (K x N)."""
    rows, K = A.shape
    N = B.shape[1]
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
    st = lib().ann_bf16_gemm_tn(_dev(A), K, _dev(B), N, rows, _dev(C), ctypes.c_void_p(int(handle) if handle else 0))
    _check(st, None, "ann_bf16_gemm_tn")


def ann_check_bounded_wait(spin_limit: int = 4096) -> int:
    """Status of the bounded-wait self-test: ANN_ERR_TIMEOUT (-12) is the expected result."""
    return lib().ann_check_bounded_wait(spin_limit)


# ------------------------------------------------------------------ learned surrogate

SG_PARAMS = 54148
_fp = lambda a: a.ctypes.data_as(_P(ctypes.c_float))  # noqa: E731


def _scheck(status: int, sg, what: str):
    if status < 0:
        detail = lib().ann_surrogate_last_error(sg).decode() if sg is not None else ""
        text = lib().ann_status_string(status).decode()
        raise AnnError(status, f"{what}: {text}" + (f" ({detail})" if detail else ""))
    return status


def ann_surrogate_create(n_max: int) -> ctypes.c_void_p:
    sg = ctypes.c_void_p()
    _scheck(lib().ann_surrogate_create(int(n_max), ctypes.byref(sg)), None, "ann_surrogate_create")
    return sg


def ann_surrogate_destroy(sg) -> None:
    lib().ann_surrogate_destroy(sg)


def ann_surrogate_set_params(sg, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != SG_PARAMS:
        raise ValueError(f"expected {SG_PARAMS} parameters")
    _scheck(lib().ann_surrogate_set_params(sg, _fp(p)), sg, "ann_surrogate_set_params")


def ann_surrogate_get_params(sg):
    p = np.zeros(SG_PARAMS, dtype=np.float32)
    _scheck(lib().ann_surrogate_get_params(sg, _fp(p)), sg, "ann_surrogate_get_params")
    return p


def ann_surrogate_set_scales(sg, us: float, ys_q: float, ys_u: float, k: int = 8) -> None:
    _scheck(lib().ann_surrogate_set_scales(sg, float(us), float(ys_q), float(ys_u), int(k)), sg,
            "ann_surrogate_set_scales")


def _tend(tend):
    if tend is None:
        return None, None
    t = np.ascontiguousarray(np.asarray(tend, dtype=np.float32).T if np.ndim(tend) == 2 and np.shape(tend)[1] == 8
                             else tend, dtype=np.float32)
    return _fp(t), t


def ann_surrogate_load(sg, ctx, tend=None) -> None:
    """tend: None (the context's last recorded step) or (n, 8) tendencies in ID order."""
    ptr, keep = _tend(tend)
    _scheck(lib().ann_surrogate_load(sg, ctx, ptr), sg, "ann_surrogate_load")


def ann_surrogate_forward(sg, n: int):
    y = np.zeros((n, 4), dtype=np.float32)
    _scheck(lib().ann_surrogate_forward(sg, _fp(y)), sg, "ann_surrogate_forward")
    return y


def ann_surrogate_gradients(sg, target):
    """(loss, gradients float32[SG_PARAMS]) against targets (n x 4)."""
    t = np.ascontiguousarray(target, dtype=np.float32)
    g = np.zeros(SG_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _scheck(lib().ann_surrogate_gradients(sg, _fp(t), ctypes.byref(loss), _fp(g)), sg, "ann_surrogate_gradients")
    return loss.value, g


def ann_surrogate_adam(sg, lr: float) -> None:
    _scheck(lib().ann_surrogate_adam(sg, float(lr)), sg, "ann_surrogate_adam")


def ann_surrogate_jump(sg, ctx, tend=None) -> None:
    ptr, keep = _tend(tend)
    _scheck(lib().ann_surrogate_jump(sg, ctx, ptr), sg, "ann_surrogate_jump")


class ann_guard_report(ctypes.Structure):
    _fields_ = [("cycles_done", ctypes.c_int32), ("checks", ctypes.c_int32), ("fell_back", ctypes.c_int32),
                ("fallback_cycle", ctypes.c_int32), ("plain_steps", ctypes.c_int64),
                ("max_err_q", ctypes.c_double), ("max_err_u", ctypes.c_double),
                ("last_err_q", ctypes.c_double), ("last_err_u", ctypes.c_double)]


def ann_surrogate_advance(sg, ctx, shadow, cycles: int, check_every: int, tol: float = 0.05) -> dict:
    """Guarded surrogate cycles (recorded plain step + jump), checked against plain SPH on `shadow`
    every `check_every` cycles; falls back to plain SPH when an error exceeds `tol`.  The report as
    a dict."""
    r = ann_guard_report()
    _scheck(lib().ann_surrogate_advance(sg, ctx, shadow, int(cycles), int(check_every), float(tol), ctypes.byref(r)),
            sg, "ann_surrogate_advance")
    return {k: getattr(r, k) for k, _ in r._fields_}


def ann_surrogate_set_velocity_correction(sg, on) -> None:
    _scheck(lib().ann_surrogate_set_velocity_correction(sg, int(on)), sg,
            "ann_surrogate_set_velocity_correction")


def ann_surrogate_last_error(sg) -> str:
    return lib().ann_surrogate_last_error(sg).decode()


def ann_surrogate_init(sg, seed: int) -> None:
    _scheck(lib().ann_surrogate_init(sg, int(seed)), sg, "ann_surrogate_init")


def ann_surrogate_euler(sg, n: int):
    """The explicit increment (n x 4: dQ11, dQ12, dux, duy; acceleration smoothed) of the loaded state."""
    inc = np.zeros((n, 4), dtype=np.float32)
    _scheck(lib().ann_surrogate_euler(sg, _fp(inc)), sg, "ann_surrogate_euler")
    return inc


# ---------------------------------------------------------------------------------------------
# three-dimensional variant
# ---------------------------------------------------------------------------------------------

def _check3(status: int, ctx, what: str):
    if status < 0:
        detail = lib().ann3_last_error(ctx).decode() if ctx is not None else ""
        text = lib().ann_status_string(status).decode()
        raise AnnError(status, f"{what}: {text}" + (f" ({detail})" if detail else ""))
    return status


def ann3_default_params(**overrides) -> ann3_params:
    p = ann3_params()
    _check(lib().ann3_default_params(ctypes.byref(p)), what="ann3_default_params")
    names = {f[0] for f in ann3_params._fields_}
    for k, v in overrides.items():
        k = "lambda_" if k == "lambda" else k
        if k not in names or k == "reserved":
            raise TypeError(f"ann3_params has no field {k!r}")
        setattr(p, k, v)
    return p


def ann3_create(p: ann3_params) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().ann3_create(ctypes.byref(p), ctypes.byref(ctx)), what="ann3_create")
    return ctx


def ann3_destroy(ctx) -> None:
    if ctx:
        lib().ann3_destroy(ctx)


def ann3_set_particles(ctx, x, y, z, u, q, rho=None) -> None:
    """Host FP64 state in ID order: x, y, z (n), u (n, 3), q (n, 5), rho (n) or None."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (x, y, z, u, q)]
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    n = arrs[0].size
    ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
    _check3(lib().ann3_set_particles(ctx, n, *ptrs, None if r is None else r.ctypes.data_as(ctypes.c_void_p)),
            ctx, "ann3_set_particles")


def ann3_step(ctx, nsteps: int = 1) -> None:
    _check3(lib().ann3_step(ctx, int(nsteps)), ctx, "ann3_step")


def ann3_get_field(ctx, name: str, n: int) -> np.ndarray:
    """Field `name` (a key of FIELDS3) in ID order as an (n, components) FP64 array."""
    fid, comps = FIELDS3[name]
    out = np.zeros(n * comps, dtype=np.float64)
    _check3(lib().ann3_get_field(ctx, fid, out.ctypes.data_as(ctypes.c_void_p)), ctx, "ann3_get_field")
    return out.reshape(n, comps)


def ann3_get_status(ctx):
    """(steps, error bits, re-sorting steps) since the particles were loaded."""
    steps = ctypes.c_int64()
    bits = ctypes.c_uint32()
    rs = ctypes.c_int64()
    _check3(lib().ann3_get_status(ctx, ctypes.byref(steps), ctypes.byref(bits), ctypes.byref(rs)), ctx,
            "ann3_get_status")
    return steps.value, bits.value, rs.value


def ann3_last_error(ctx) -> str:
    return lib().ann3_last_error(ctx).decode()
