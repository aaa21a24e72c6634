"""ctypes binding of ``libbrahmap.so`` (include/brahmap.h), same names as the C-ABI.

Argument marshalling only: device arrays are passed as torch CUDA tensors
(their ``data_ptr()``), host arrays as numpy arrays, and a non-OK status is
raised as :class:`BrahmapError` carrying ``bm_last_error()``.  Every step of
the computation runs in the library's CUDA kernels; there is no Python or
CPU fallback, and importing this module fails if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbrahmap.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "brahmap.h")

BM_OK, BM_ERR_INVALID, BM_ERR_OOM, BM_ERR_CUDA = 0, 1, 2, 3
BM_ERR_NOT_CONVERGED, BM_ERR_BREAKDOWN, BM_ERR_TIMEOUT, BM_ERR_BUSY, BM_ERR_NOT_FOUND = 4, 5, 6, 7, 8
BM_SOLVER_I, BM_SOLVER_QU, BM_SOLVER_IQU = 1, 2, 3
BM_F32, BM_F64 = 0, 1
BM_PREC_FP64, BM_PREC_MIXED = 0, 1


class BrahmapError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {status_string(status)} ({status}): {msg}")
        self.status = status


class bm_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


BM_NOISE_WHITE, BM_NOISE_TOEPLITZ = 0, 1


class bm_request(ctypes.Structure):
    _fields_ = [("npix", ctypes.c_int64), ("nsamples", ctypes.c_int64), ("solver", ctypes.c_int),
                ("pix", ctypes.c_void_p), ("cos2psi", ctypes.c_void_p), ("sin2psi", ctypes.c_void_p),
                ("psi", ctypes.c_void_p), ("psi_dtype", ctypes.c_int), ("ndet", ctypes.c_int32),
                ("det_offsets", ctypes.c_void_p), ("noise", ctypes.c_int), ("inv_var", ctypes.c_void_p),
                ("chunk_len", ctypes.c_int64), ("nlags", ctypes.c_int32), ("coeffs", ctypes.c_void_p),
                ("tod", ctypes.c_void_p), ("tod_dtype", ctypes.c_int), ("min_hits", ctypes.c_int32),
                ("max_cond", ctypes.c_double), ("tol", ctypes.c_double), ("maxiter", ctypes.c_int32),
                ("precision", ctypes.c_int), ("map_out", ctypes.c_void_p), ("pointing_key", ctypes.c_uint64)]


class bm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("message", ctypes.c_char * 256), ("batch_size", ctypes.c_int32), ("resident", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["message"] = d["message"].decode(errors="replace")
        return d


class bm_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "rejected", "cancelled", "running", "queued")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "samples_per_s")] + \
               [(n, ctypes.c_int64) for n in ("budget_bytes", "reserved_bytes", "peak_reserved_bytes",
                                              "resident_bytes", "resident_hits", "batches", "batched_requests",
                                              "evictions", "oom_requeues")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2501_16122_gb300.build.build()")
lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double

_SIGS = {
    "bm_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "bm_last_error": ([], ctypes.c_char_p),
    "bm_version": ([], ctypes.c_char_p),
    "bm_context_create": ([ctypes.c_int, _P, _PP], ctypes.c_int),
    "bm_context_destroy": ([_P], None),
    "bm_context_set_timing": ([_P, ctypes.c_int], ctypes.c_int),
    "bm_context_set_graphs": ([_P, ctypes.c_int], ctypes.c_int),
    "bm_context_kernel_time": ([_P, ctypes.c_char_p, ctypes.POINTER(_f64), ctypes.POINTER(_i64)], ctypes.c_int),
    "bm_kernel_launches": ([], _i64),
    "bm_ang2pix_ring": ([_P, _i64, _i64, _P, _P, _P], ctypes.c_int),
    "bm_pointing_create": ([_P, _i64, _i64, _P, _P, ctypes.c_int, ctypes.c_int, _PP], ctypes.c_int),
    "bm_pointing_create_trig": ([_P, _i64, _i64, _P, _P, _P, ctypes.c_int, _PP], ctypes.c_int),
    "bm_pointing_create_hwp": ([_P, _i64, _i64, _P, _i32, _P, _P, _f64, _f64, ctypes.c_int, _PP], ctypes.c_int),
    "bm_pointing_create_with_tod": ([_P, _i64, _i64, _P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _PP],
                                    ctypes.c_int),
    "bm_pointing_destroy": ([_P], None),
    "bm_pointing_get_hits": ([_P, _P], ctypes.c_int),
    "bm_pointing_get_order": ([_P, _P, _P], ctypes.c_int),
    "bm_pointing_apply": ([_P, _P, _P], ctypes.c_int),
    "bm_pointing_apply_transpose": ([_P, _P, _P], ctypes.c_int),
    "bm_inv_noise_create_diag": ([_P, _i32, _P, _P, _PP], ctypes.c_int),
    "bm_inv_noise_create_toeplitz": ([_P, _i32, _P, _i64, _i32, _P, _P, _PP], ctypes.c_int),
    "bm_inv_noise_create_sample_weights": ([_P, _i64, _P, _PP], ctypes.c_int),
    "bm_inv_noise_create_offset_filter": ([_P, _i32, _P, _P, _i64, _PP], ctypes.c_int),
    "bm_inv_noise_destroy": ([_P], None),
    "bm_inv_noise_apply": ([_P, _P, _P], ctypes.c_int),
    "bm_blockdiag_precond_create": ([_P, _P, _i32, _f64, _PP], ctypes.c_int),
    "bm_precond_destroy": ([_P], None),
    "bm_precond_get_mask": ([_P, _P, _P], ctypes.c_int),
    "bm_precond_get_blocks": ([_P, _P, _P], ctypes.c_int),
    "bm_precond_apply": ([_P, _P, _P], ctypes.c_int),
    "bm_rhs": ([_P, _P, _P, _P, ctypes.c_int, _i32, _P], ctypes.c_int),
    "bm_matvec": ([_P, _P, _P, _P, _P, ctypes.c_int], ctypes.c_int),
    "bm_matvec_white_static": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bm_measure_fma_peak": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "bm_context_set_allreduce": ([_P, _P, _P], ctypes.c_int),
    "bm_pcg_solve": ([_P, _P, _P, _P, ctypes.c_int, _i32, _P, _f64, _i32, ctypes.c_int,
                      ctypes.POINTER(bm_solve_info)], ctypes.c_int),
    "bm_serve_create": ([_P, ctypes.c_size_t, _i32, _PP], ctypes.c_int),
    "bm_serve_submit": ([_P, ctypes.POINTER(bm_request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bm_serve_poll": ([_P, ctypes.c_uint64, _i32, ctypes.POINTER(bm_result)], ctypes.c_int),
    "bm_serve_cancel": ([_P, ctypes.c_uint64], ctypes.c_int),
    "bm_serve_get_stats": ([_P, ctypes.POINTER(bm_serve_stats)], ctypes.c_int),
    "bm_serve_destroy": ([_P], None),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def header_functions() -> list[str]:
    """Names of the functions declared in include/brahmap.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"typedef[^;]*;", "", text)  # function-pointer types are not functions
    return sorted(set(re.findall(r"\b(bm_[a-z0-9_]+)\s*\(", text)))


def status_string(s: int) -> str:
    return lib.bm_status_string(int(s)).decode()


def bm_last_error() -> str:
    return lib.bm_last_error().decode()


def bm_version() -> str:
    return lib.bm_version().decode()


def _check(status: int, func: str):
    if status != BM_OK:
        raise BrahmapError(status, func, bm_last_error())


def _dev(t, dtype=None, name="array"):
    """Device pointer of a contiguous CUDA tensor (optionally of a given dtype)."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _in(t, dtype=None, name="array"):
    """Pointer of an input the library may read from the host: a contiguous
    CUDA tensor, or a contiguous page-locked (pinned) CPU tensor."""
    if t is None:
        return None
    if getattr(t, "is_cuda", False):
        return _dev(t, dtype, name)
    if not (hasattr(t, "is_pinned") and t.is_pinned()):
        raise TypeError(f"{name} must be a CUDA tensor or a pinned CPU tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return BM_F32
    if t.dtype == torch.float64:
        return BM_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


# ---------------------------------------------------------------- context
def bm_context_create(device: int = 0, stream=None):
    """stream: a torch.cuda.Stream (default: the current stream of `device`)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    out = ctypes.c_void_p()
    _check(lib.bm_context_create(int(device), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out)),
           "bm_context_create")
    return out


def bm_context_destroy(ctx):
    _REDUCERS.pop(ctx.value, None)
    lib.bm_context_destroy(ctx)


# bm_allreduce_fn: bm_status (*)(double* buf, int64_t count, void* user)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)
_REDUCERS = {}  # context -> the ctypes callback object (kept alive while set)


def bm_context_set_allreduce(ctx, fn):
    """Make ctx one rank of a detector-sharded solve: fn(ptr, count) sums the
    FP64 device array at ptr over every rank in place and returns a bm_status
    (0 = BM_OK); None makes the context unsharded again."""
    if fn is None:
        _check(lib.bm_context_set_allreduce(ctx, None, None), "bm_context_set_allreduce")
        _REDUCERS.pop(ctx.value, None)
        return

    def call(ptr, count, _user):
        try:
            return int(fn(ptr, count) or 0)
        except Exception as exc:  # no exception may cross the C-ABI
            import sys
            print(f"allreduce callback failed: {exc!r}", file=sys.stderr)
            return BM_ERR_CUDA

    cb = ALLREDUCE_FN(call)
    _check(lib.bm_context_set_allreduce(ctx, ctypes.cast(cb, ctypes.c_void_p), None), "bm_context_set_allreduce")
    _REDUCERS[ctx.value] = cb


class _DeviceArray:
    """A view of count FP64 values at a device address, for torch.as_tensor."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def torch_allreduce(group=None):
    """A reduction for bm_context_set_allreduce over a torch.distributed
    process group: NCCL sums the device array in place; another backend
    (gloo) sums a host copy, which is copied back."""
    import torch
    import torch.distributed as dist

    def reduce(ptr, count):
        t = torch.as_tensor(_DeviceArray(ptr, count), device="cuda")
        if dist.get_backend(group) == "nccl":
            dist.all_reduce(t, group=group)
        else:
            h = t.cpu()
            dist.all_reduce(h, group=group)
            t.copy_(h)
        torch.cuda.current_stream().synchronize()
        return BM_OK

    return reduce


from .shard import detector_shard  # noqa: E402,F401  (host-side partition of a sharded solve)


def bm_context_set_timing(ctx, enable: bool):
    _check(lib.bm_context_set_timing(ctx, int(bool(enable))), "bm_context_set_timing")


def bm_context_set_graphs(ctx, enable: bool):
    _check(lib.bm_context_set_graphs(ctx, int(bool(enable))), "bm_context_set_graphs")


def bm_kernel_launches() -> int:
    return int(lib.bm_kernel_launches())


def bm_context_kernel_time(ctx, name: str):
    ms, n = _f64(), _i64()
    _check(lib.bm_context_kernel_time(ctx, name.encode(), ctypes.byref(ms), ctypes.byref(n)),
           "bm_context_kernel_time")
    return ms.value, n.value


# ------------------------------------------------------------ pixelisation
def bm_ang2pix_ring(ctx, nside: int, z, phi, pix):
    import torch
    _check(lib.bm_ang2pix_ring(ctx, int(nside), z.numel(), _dev(z, torch.float64, "z"),
                               _dev(phi, torch.float64, "phi"), _dev(pix, torch.int32, "pix")),
           "bm_ang2pix_ring")


# ---------------------------------------------------------------- pointing
def bm_pointing_create(ctx, npix: int, pix, psi, solver: int = BM_SOLVER_IQU):
    import torch
    out = ctypes.c_void_p()
    _check(lib.bm_pointing_create(ctx, int(npix), pix.numel(), _in(pix, torch.int32, "pix"),
                                  _in(psi, None, "psi"), _dtype_code(psi), int(solver), ctypes.byref(out)),
           "bm_pointing_create")
    return out


def bm_pointing_create_trig(ctx, npix: int, pix, cos2psi, sin2psi, solver: int = BM_SOLVER_IQU):
    import torch
    out = ctypes.c_void_p()
    _check(lib.bm_pointing_create_trig(ctx, int(npix), pix.numel(), _in(pix, torch.int32, "pix"),
                                       _in(cos2psi, torch.float32, "cos2psi"), _in(sin2psi, torch.float32, "sin2psi"),
                                       int(solver), ctypes.byref(out)), "bm_pointing_create_trig")
    return out


def bm_pointing_create_hwp(ctx, npix: int, pix, det_offsets, psi_det, hwp_turns_per_sample: float,
                           hwp_phase0: float, solver: int = BM_SOLVER_IQU):
    """Pointing whose angle follows a rotating half-wave plate: sample k of
    detector d has theta = psi_det[d] + 2 (2 pi hwp_turns_per_sample k +
    hwp_phase0).  pix: int32 device or pinned host tensor; det_offsets and
    psi_det: host arrays."""
    import torch
    off, offp = _host(det_offsets, np.int64)
    pd, pdp = _host(psi_det, np.float64)
    out = ctypes.c_void_p()
    _check(lib.bm_pointing_create_hwp(ctx, int(npix), pix.numel(), _in(pix, torch.int32, "pix"), off.size - 1, offp,
                                      pdp, float(hwp_turns_per_sample), float(hwp_phase0), int(solver),
                                      ctypes.byref(out)), "bm_pointing_create_hwp")
    return out


def bm_pointing_create_with_tod(ctx, npix: int, pix, tod, psi=None, cos2psi=None, sin2psi=None,
                                solver: int = BM_SOLVER_IQU):
    """A pointing that also carries one FP32 TOD in pixel-sorted order: give
    psi, or cos2psi and sin2psi.  bm_rhs / bm_pcg_solve with tod=None use it."""
    import torch
    out = ctypes.c_void_p()
    _check(lib.bm_pointing_create_with_tod(
        ctx, int(npix), pix.numel(), _in(pix, torch.int32, "pix"),
        _in(psi, None, "psi") if psi is not None else None, _dtype_code(psi) if psi is not None else 0,
        _in(cos2psi, torch.float32, "cos2psi") if cos2psi is not None else None,
        _in(sin2psi, torch.float32, "sin2psi") if sin2psi is not None else None,
        _in(tod, torch.float32, "tod"), int(solver), ctypes.byref(out)), "bm_pointing_create_with_tod")
    return out


def bm_pointing_destroy(p):
    lib.bm_pointing_destroy(p)


def bm_pointing_get_hits(p, hits):
    import torch
    _check(lib.bm_pointing_get_hits(p, _dev(hits, torch.int32, "hits")), "bm_pointing_get_hits")


def bm_pointing_get_order(p):
    """The time indices of the non-flagged samples in pixel order, ties in
    time order (a device int32 tensor holding the uint32 indices)."""
    import torch
    nv = ctypes.c_int64(0)
    _check(lib.bm_pointing_get_order(p, None, ctypes.byref(nv)), "bm_pointing_get_order")
    order = torch.zeros(max(nv.value, 1), dtype=torch.int32, device="cuda")
    _check(lib.bm_pointing_get_order(p, ctypes.c_void_p(order.data_ptr()), None), "bm_pointing_get_order")
    return order[: nv.value]


def bm_pointing_apply(p, x, y):
    import torch
    _check(lib.bm_pointing_apply(p, _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y")),
           "bm_pointing_apply")


def bm_pointing_apply_transpose(p, y, x):
    import torch
    _check(lib.bm_pointing_apply_transpose(p, _dev(y, torch.float64, "y"), _dev(x, torch.float64, "x")),
           "bm_pointing_apply_transpose")


# ----------------------------------------------------------- inverse noise
def bm_inv_noise_create_diag(ctx, det_offsets, inv_var):
    off, offp = _host(det_offsets, np.int64)
    iv, ivp = _host(inv_var, np.float64)
    out = ctypes.c_void_p()
    _check(lib.bm_inv_noise_create_diag(ctx, off.size - 1, offp, ivp, ctypes.byref(out)),
           "bm_inv_noise_create_diag")
    return out


def bm_inv_noise_create_toeplitz(ctx, det_offsets, chunk_len: int, coeffs, white_inv_var):
    off, offp = _host(det_offsets, np.int64)
    c, cp = _host(coeffs, np.float64)
    wv, wvp = _host(white_inv_var, np.float64)
    out = ctypes.c_void_p()
    _check(lib.bm_inv_noise_create_toeplitz(ctx, off.size - 1, offp, int(chunk_len), c.shape[-1], cp, wvp,
                                            ctypes.byref(out)), "bm_inv_noise_create_toeplitz")
    return out


def bm_inv_noise_create_sample_weights(ctx, weights):
    """Diagonal N^-1 with a weight per sample (FP64 device or pinned host tensor)."""
    import torch
    out = ctypes.c_void_p()
    _check(lib.bm_inv_noise_create_sample_weights(ctx, weights.numel(), _in(weights, torch.float64, "weights"),
                                                  ctypes.byref(out)), "bm_inv_noise_create_sample_weights")
    return out


def bm_inv_noise_create_offset_filter(ctx, det_offsets, inv_var, baseline_len: int):
    """White N^-1 with a baseline offset per interval of baseline_len samples marginalised out."""
    off, offp = _host(det_offsets, np.int64)
    iv, ivp = _host(inv_var, np.float64)
    out = ctypes.c_void_p()
    _check(lib.bm_inv_noise_create_offset_filter(ctx, off.size - 1, offp, ivp, int(baseline_len),
                                                 ctypes.byref(out)), "bm_inv_noise_create_offset_filter")
    return out


def bm_inv_noise_destroy(n):
    lib.bm_inv_noise_destroy(n)


def bm_inv_noise_apply(n, y, z):
    import torch
    _check(lib.bm_inv_noise_apply(n, _dev(y, torch.float64, "y"), _dev(z, torch.float64, "z")),
           "bm_inv_noise_apply")


# ---------------------------------------------------------- preconditioner
def bm_blockdiag_precond_create(p, n, min_hits: int = 3, max_cond: float = 1e3):
    out = ctypes.c_void_p()
    _check(lib.bm_blockdiag_precond_create(p, n, int(min_hits), float(max_cond), ctypes.byref(out)),
           "bm_blockdiag_precond_create")
    return out


def bm_precond_destroy(pc):
    lib.bm_precond_destroy(pc)


def bm_precond_get_mask(pc, mask=None, hits=None):
    import torch
    _check(lib.bm_precond_get_mask(pc, _dev(mask, torch.uint8, "mask"), _dev(hits, torch.int32, "hits")),
           "bm_precond_get_mask")


def bm_precond_get_blocks(pc, blocks=None, cond=None):
    import torch
    _check(lib.bm_precond_get_blocks(pc, _dev(blocks, torch.float64, "blocks"), _dev(cond, torch.float64, "cond")),
           "bm_precond_get_blocks")


def bm_precond_apply(pc, r, z):
    import torch
    _check(lib.bm_precond_apply(pc, _dev(r, torch.float64, "r"), _dev(z, torch.float64, "z")), "bm_precond_apply")


# ---------------------------------------------------------------- system
def bm_rhs(p, n, pc, tod, nrhs: int, b):
    import torch
    # tod=None: the TOD the pointing was created with
    _check(lib.bm_rhs(p, n, pc, _dev(tod, None, "tod") if tod is not None else None,
                      _dtype_code(tod) if tod is not None else BM_F32, int(nrhs), _dev(b, torch.float64, "b")),
           "bm_rhs")


def bm_matvec(p, n, pc, x, q, prec: int = BM_PREC_FP64):
    import torch
    _check(lib.bm_matvec(p, n, pc, _dev(x, torch.float64, "x"), _dev(q, torch.float64, "q"), int(prec)),
           "bm_matvec")


def bm_matvec_white_static(p, n, pc, x, q):
    """White-noise FP32-product matvec that allocates no device memory (its
    scratch is a fixed array inside the library)."""
    import torch
    _check(lib.bm_matvec_white_static(p, n, pc, _dev(x, torch.float64, "x"), _dev(q, torch.float64, "q")),
           "bm_matvec_white_static")


def bm_measure_fma_peak(ctx, dtype: int) -> float:
    """Measured FMA rate of the device in flop/s: dtype BM_F32 or BM_F64."""
    v = ctypes.c_double()
    _check(lib.bm_measure_fma_peak(ctx, int(dtype), ctypes.byref(v)), "bm_measure_fma_peak")
    return v.value


def bm_pcg_solve(p, n, pc, tod, nrhs: int, map_out, tol: float, maxiter: int, prec: int = BM_PREC_FP64,
                 raise_on_error: bool = True):
    """Returns (status, [info dict per RHS])."""
    import torch
    infos = (bm_solve_info * int(nrhs))()
    st = lib.bm_pcg_solve(p, n, pc, _in(tod, None, "tod") if tod is not None else None,
                          _dtype_code(tod) if tod is not None else BM_F32, int(nrhs),
                          _dev(map_out, torch.float64, "map_out"), float(tol), int(maxiter), int(prec), infos)
    if raise_on_error and st not in (BM_OK, BM_ERR_NOT_CONVERGED):
        _check(st, "bm_pcg_solve")
    return st, [i.as_dict() for i in infos]


# ------------------------------------------------------------------ serving
def bm_serve_create(ctx, hbm_budget_bytes: int, max_slots: int):
    out = ctypes.c_void_p()
    _check(lib.bm_serve_create(ctx, int(hbm_budget_bytes), int(max_slots), ctypes.byref(out)), "bm_serve_create")
    return out


def make_request(npix, pix, tod, map_out, det_offsets, inv_var, solver=BM_SOLVER_IQU, cos2psi=None, sin2psi=None,
                 psi=None, coeffs=None, chunk_len=0, min_hits=3, max_cond=1e3, tol=1e-6, maxiter=500,
                 precision=BM_PREC_MIXED, pointing_key=0):
    """Build a bm_request from torch device tensors and host arrays.  Returns
    (request, keepalive) -- keep the second object alive until submitted.
    pointing_key: 0, or the caller's name of a pointing shared by several
    requests (kept resident by the server between them)."""
    import torch
    off, offp = _host(det_offsets, np.int64)
    iv, ivp = _host(inv_var, np.float64)
    keep = [off, iv]
    r = bm_request()
    r.npix, r.nsamples, r.solver = int(npix), pix.numel(), int(solver)
    r.pix = _dev(pix, torch.int32, "pix")
    if cos2psi is not None:
        r.cos2psi = _dev(cos2psi, torch.float32, "cos2psi")
        r.sin2psi = _dev(sin2psi, torch.float32, "sin2psi")
    else:
        r.psi = _dev(psi, None, "psi")
        r.psi_dtype = _dtype_code(psi)
    r.ndet = off.size - 1
    r.det_offsets, r.inv_var = offp, ivp
    if coeffs is not None:
        c, cp = _host(coeffs, np.float64)
        keep.append(c)
        r.noise, r.coeffs, r.nlags, r.chunk_len = BM_NOISE_TOEPLITZ, cp, c.shape[-1], int(chunk_len)
    else:
        r.noise = BM_NOISE_WHITE
    r.tod, r.tod_dtype = _dev(tod, None, "tod"), _dtype_code(tod)
    r.min_hits, r.max_cond, r.tol, r.maxiter, r.precision = int(min_hits), float(max_cond), float(tol), int(maxiter), int(precision)
    r.map_out = _dev(map_out, torch.float64, "map_out")
    r.pointing_key = int(pointing_key)
    return r, keep


def bm_serve_submit(server, req) -> int:
    t = ctypes.c_uint64()
    _check(lib.bm_serve_submit(server, ctypes.byref(req), ctypes.byref(t)), "bm_serve_submit")
    return t.value


def bm_serve_poll(server, ticket: int, timeout_ms: int):
    """Returns (status, result dict or None); status is BM_OK, BM_ERR_TIMEOUT or BM_ERR_NOT_FOUND."""
    res = bm_result()
    st = lib.bm_serve_poll(server, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res))
    if st not in (BM_OK, BM_ERR_TIMEOUT, BM_ERR_NOT_FOUND):
        _check(st, "bm_serve_poll")
    return st, (res.as_dict() if st == BM_OK else None)


def bm_serve_cancel(server, ticket: int) -> int:
    return lib.bm_serve_cancel(server, ctypes.c_uint64(ticket))


def bm_serve_get_stats(server):
    s = bm_serve_stats()
    _check(lib.bm_serve_get_stats(server, ctypes.byref(s)), "bm_serve_get_stats")
    return s.as_dict()


def bm_serve_destroy(server):
    lib.bm_serve_destroy(server)
