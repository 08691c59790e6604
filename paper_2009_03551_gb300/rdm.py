"""Thin ctypes binding of the C ABI in include/rdm.h.

Argument marshalling only: every step of the solve runs in the CUDA kernels
of ``librdm.so``.  The functions keep the C names (``rdm_create``,
``rdm_upload_h0``, ``rdm_solve``, ...); ``Solver`` wraps a handle for
convenience.  Matrices are passed as any object with ``nb, b, n, row_ptr,
col_idx, vals`` attributes (NumPy arrays: host upload) or as CUDA torch
tensors (device upload, ``on_device = 1``).  There is no CPU fallback: if
the library is missing this module raises ImportError.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from pathlib import Path
from typing import Optional

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "librdm.so"

RDM_OK = 0
RDM_NOT_CONVERGED = 1
RDM_EINVAL = -1
RDM_EBADBSR = -2
RDM_ENOMEM = -3
RDM_ECUDA = -4
RDM_ECAPACITY = -5
RDM_ETIMEOUT = -6
RDM_ESTATE = -7

MODE_FP64 = 0
MODE_FP32 = 1
MODE_MIXED_BF16 = 2
MODE_MIXED_FP16 = 3
MODES = {"fp64": 0, "fp32": 1, "mixed_bf16": 2, "mixed_fp16": 3}
PRODUCT_SLICES = 8      # rdm_block_product: the tensor-core slice product (FP64-class)
REFINE_SLICES = 5       # rdm_params.refine_x0: X0^2 of the final tier as tensor-core slice products

EXPORTED = (
    "rdm_create", "rdm_destroy", "rdm_last_error", "rdm_default_params", "rdm_set_params",
    "rdm_batch_create", "rdm_upload_h0", "rdm_upload_h1", "rdm_solve", "rdm_force_branches",
    "rdm_get_info", "rdm_get_p0_nnzb", "rdm_get_p1_nnzb", "rdm_get_p0", "rdm_get_p1",
    "rdm_get_alpha", "rdm_get_log", "rdm_block_product", "rdm_version", "rdm_bsr_dot_noalloc",
    "rdm_set_test_knobs", "rdm_solve_async", "rdm_sync", "rdm_upload_s",
)


class rdm_bsr(C.Structure):
    _fields_ = [("nb", C.c_int32), ("b", C.c_int32), ("n", C.c_int32), ("on_device", C.c_int32),
                ("nnzb", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("vals", C.c_void_p)]


class rdm_bsr_out(C.Structure):
    _fields_ = [("nb", C.c_int32), ("b", C.c_int32), ("n", C.c_int32), ("nnzb", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p)]


class rdm_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("tau_x1", C.c_double), ("tau_refine", C.c_double),
                ("tol", C.c_double), ("stall_tol", C.c_double), ("spin_factor", C.c_double),
                ("max_iter", C.c_int32), ("mode", C.c_int32), ("min_iter", C.c_int32),
                ("use_graphs", C.c_int32), ("verbose", C.c_int32), ("refine_x1", C.c_int32),
                ("symbolic_hash", C.c_int32), ("chunk_mb", C.c_int32), ("refine_x0", C.c_int32),
                ("stall_window", C.c_int32), ("block_size", C.c_int32), ("autotune", C.c_int32),
                ("split_directions", C.c_int32), ("correct", C.c_int32),
                ("correct_tau", C.c_double)]


class rdm_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("tier_iters", C.c_int32 * 4),
                ("eps_min", C.c_double), ("eps_max", C.c_double), ("trace_error", C.c_double),
                ("idempotency", C.c_double), ("band_energy0", C.c_double),
                ("nnzb_p0", C.c_int64), ("nnzb_p1", C.c_int64 * 3), ("time_ms", C.c_double),
                ("useful_flops", C.c_double), ("issued_flops", C.c_double),
                ("kernel_ms", C.c_double * 8), ("kernel_flops", C.c_double * 5),
                ("kernel_launches", C.c_int64), ("tc_launches", C.c_int32), ("simt_launches", C.c_int32),
                ("numeric_bytes", C.c_double), ("device_bytes_peak", C.c_int64),
                ("product_groups", C.c_int32), ("block_size", C.c_int32), ("autotune_ms", C.c_double),
                ("probe_ms", C.c_double * 3), ("lowdin_iterations", C.c_int32), ("oz_launches", C.c_int32),
                ("correction_ms", C.c_double)]


class rdm_test_knobs(C.Structure):
    _fields_ = [("tc_wait_cycles", C.c_int64), ("tc_hold", C.c_int32), ("tc_window_cols", C.c_int32),
                ("tc_block_copies", C.c_int32), ("pad0", C.c_int32)]


class rdm_iter_log(C.Structure):
    _fields_ = [("iter", C.c_int32), ("branch", C.c_int32), ("tier", C.c_int32), ("sys", C.c_int32),
                ("trace", C.c_double), ("idempotency", C.c_double), ("eb0", C.c_double),
                ("eb1", C.c_double * 3), ("nnzb0", C.c_int64), ("nnzb1", C.c_int64 * 3),
                ("ms", C.c_double)]


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"{_LIB_PATH.name} is not built; run `python -m paper_2009_03551_gb300.build` "
                          "(requires nvcc)")
    lib = C.CDLL(str(_LIB_PATH))
    H = C.c_void_p
    sig = {
        "rdm_create": (C.c_int, [C.POINTER(H), C.c_int, C.c_void_p]),
        "rdm_destroy": (C.c_int, [H]),
        "rdm_last_error": (C.c_char_p, [H]),
        "rdm_default_params": (C.c_int, [C.POINTER(rdm_params)]),
        "rdm_set_params": (C.c_int, [H, C.POINTER(rdm_params)]),
        "rdm_batch_create": (C.c_int, [H, C.c_int]),
        "rdm_upload_h0": (C.c_int, [H, C.c_int, C.POINTER(rdm_bsr), C.c_int64]),
        "rdm_upload_h1": (C.c_int, [H, C.c_int, C.c_int, C.POINTER(rdm_bsr)]),
        "rdm_upload_s": (C.c_int, [H, C.c_int, C.POINTER(rdm_bsr)]),
        "rdm_solve": (C.c_int, [H, C.POINTER(rdm_info)]),
        "rdm_solve_async": (C.c_int, [H]),
        "rdm_sync": (C.c_int, [H, C.POINTER(rdm_info)]),
        "rdm_force_branches": (C.c_int, [H, C.POINTER(C.c_uint8), C.c_int]),
        "rdm_get_info": (C.c_int, [H, C.c_int, C.POINTER(rdm_info)]),
        "rdm_get_p0_nnzb": (C.c_int, [H, C.c_int, C.POINTER(C.c_int64)]),
        "rdm_get_p1_nnzb": (C.c_int, [H, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
        "rdm_get_p0": (C.c_int, [H, C.c_int, C.POINTER(rdm_bsr_out)]),
        "rdm_get_p1": (C.c_int, [H, C.c_int, C.c_int, C.POINTER(rdm_bsr_out)]),
        "rdm_get_alpha": (C.c_int, [H, C.c_int, C.POINTER(C.c_double)]),
        "rdm_get_log": (C.c_int, [H, C.POINTER(rdm_iter_log), C.c_int, C.POINTER(C.c_int)]),
        "rdm_block_product": (C.c_int, [H, C.POINTER(rdm_bsr), C.POINTER(rdm_bsr), C.POINTER(rdm_bsr),
                                        C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                                        C.POINTER(rdm_bsr_out), C.POINTER(C.c_int64)]),
        "rdm_version": (C.c_char_p, []),
        "rdm_set_test_knobs": (C.c_int, [H, C.POINTER(rdm_test_knobs)]),
        "rdm_bsr_dot_noalloc": (C.c_int, [C.POINTER(rdm_bsr), C.POINTER(rdm_bsr), C.c_void_p, C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


class RdmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rdm status {code}: {msg}")
        self.code = code


# ---- C names, one-to-one --------------------------------------------------

def rdm_version() -> str:
    return _lib.rdm_version().decode()


def rdm_last_error(h) -> str:
    return (_lib.rdm_last_error(h) or b"").decode()


def _check(h, code: int, allow_warn: bool = False) -> int:
    if code < 0 or (code > 0 and not allow_warn):
        raise RdmError(code, rdm_last_error(h))
    return code


def rdm_create(device: int = 0, stream=None):
    h = C.c_void_p()
    code = _lib.rdm_create(C.byref(h), device, stream)
    if code != RDM_OK:
        raise RdmError(code, rdm_last_error(None))
    return h


def rdm_destroy(h) -> None:
    _lib.rdm_destroy(h)


def rdm_default_params() -> rdm_params:
    p = rdm_params()
    _lib.rdm_default_params(C.byref(p))
    return p


def rdm_set_params(h, p: rdm_params) -> None:
    _check(h, _lib.rdm_set_params(h, C.byref(p)))


def rdm_batch_create(h, n: int) -> None:
    _check(h, _lib.rdm_batch_create(h, n))


class _Keep:
    """Keeps the arrays behind an rdm_bsr alive for the duration of a call."""

    def __init__(self, *objs):
        self.objs = objs


def to_bsr(m):
    """Marshal a matrix object (NumPy or CUDA torch tensors) into rdm_bsr."""
    rp, ci, va = m.row_ptr, m.col_idx, m.vals
    on_dev = 0
    if hasattr(va, "is_cuda"):
        import torch
        if va.is_cuda:
            on_dev = 1
            rp = rp.to(device=va.device, dtype=torch.int32).contiguous()
            ci = ci.to(device=va.device, dtype=torch.int32).contiguous()
            va = va.to(dtype=torch.float64).contiguous()
            ptrs = (rp.data_ptr(), ci.data_ptr(), va.data_ptr())
        else:
            rp, ci, va = rp.numpy(), ci.numpy(), va.numpy()
    if not on_dev:
        rp = np.ascontiguousarray(rp, dtype=np.int32)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        va = np.ascontiguousarray(va, dtype=np.float64)
        ptrs = (rp.ctypes.data, ci.ctypes.data if ci.size else 0, va.ctypes.data if va.size else 0)
    s = rdm_bsr(int(m.nb), int(m.b), int(m.n), on_dev, int(ci.shape[0]), *ptrs)
    return s, _Keep(rp, ci, va)


def rdm_upload_h0(h, sys: int, m, n_electrons: int) -> None:
    s, keep = to_bsr(m)
    _check(h, _lib.rdm_upload_h0(h, sys, C.byref(s), int(n_electrons)))
    del keep


def rdm_upload_h1(h, sys: int, direction: int, m) -> None:
    s, keep = to_bsr(m)
    _check(h, _lib.rdm_upload_h1(h, sys, direction, C.byref(s)))
    del keep


def rdm_upload_s(h, sys: int, m) -> None:
    """Overlap matrix of system `sys` (non-orthogonal basis, see include/rdm.h)."""
    b, keep = to_bsr(m)
    _check(h, _lib.rdm_upload_s(h, sys, C.byref(b)))
    del keep


def rdm_force_branches(h, seq) -> None:
    arr = (C.c_uint8 * len(seq))(*[int(x) for x in seq])
    _check(h, _lib.rdm_force_branches(h, arr, len(seq)))


def rdm_solve(h) -> tuple:
    info = rdm_info()
    code = _check(h, _lib.rdm_solve(h, C.byref(info)), allow_warn=True)
    return code, info


def rdm_solve_async(h) -> None:
    """Start the solve; it runs while the caller continues (rdm_sync waits)."""
    _check(h, _lib.rdm_solve_async(h))


def rdm_sync(h) -> tuple:
    """Wait for the solve started by rdm_solve_async: (status, rdm_info)."""
    info = rdm_info()
    code = _lib.rdm_sync(h, C.byref(info))
    _check(h, code, allow_warn=True)
    return code, info


def rdm_get_info(h, sys: int = 0) -> rdm_info:
    info = rdm_info()
    _check(h, _lib.rdm_get_info(h, sys, C.byref(info)))
    return info


@dataclass
class BsrResult:
    nb: int
    b: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    def to_dense(self, padded: bool = False) -> np.ndarray:
        b = self.b
        a = np.zeros((self.nb * b, self.nb * b))
        rows = np.repeat(np.arange(self.nb), np.diff(self.row_ptr))
        for p in range(self.nnzb):
            i, j = rows[p], self.col_idx[p]
            a[i * b:(i + 1) * b, j * b:(j + 1) * b] = self.vals[p]
        return a if padded else a[: self.n, : self.n]


def _fetch(h, getter, *idx, out=None) -> BsrResult:
    """Size query, then one copy into host arrays: fresh ones, or the
    caller's ``out = (row_ptr, col_idx, vals)`` (e.g. views of pinned
    memory reused across solves; C-contiguous int32 / int32 / float64, with
    room for nb + 1, nnzb and nnzb*b*b entries).  The result's arrays are
    views of exactly nb + 1, nnzb and (nnzb, b, b) entries."""
    q = rdm_bsr_out()                      # size query (row_ptr = NULL)
    _check(h, getter(h, *idx, C.byref(q)))
    nb, b, nnz = int(q.nb), int(q.b), int(q.nnzb)
    if out is None:
        rp = np.empty(nb + 1, dtype=np.int32)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        va = np.empty((max(nnz, 1), b, b), dtype=np.float64)
    else:
        rp, ci, va = out
        for a, dt, need in ((rp, np.int32, nb + 1), (ci, np.int32, nnz), (va, np.float64, nnz * b * b)):
            if a.dtype != dt or not a.flags.c_contiguous or a.size < need:
                raise ValueError(f"output buffer: need a C-contiguous {np.dtype(dt).name} array of "
                                 f">= {need} elements")
        va = va.reshape(-1)[: max(nnz, 1) * b * b].reshape(max(nnz, 1), b, b) if va.size else va
    o = rdm_bsr_out(nb, b, 0, nnz, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    _check(h, getter(h, *idx, C.byref(o)))
    return BsrResult(nb, b, int(o.n), rp[: nb + 1], ci[:nnz], va[:nnz])


def rdm_get_p0_nnzb(h, sys: int = 0) -> int:
    n = C.c_int64()
    _check(h, _lib.rdm_get_p0_nnzb(h, sys, C.byref(n)))
    return int(n.value)


def rdm_get_p1_nnzb(h, sys: int = 0, direction: int = 0) -> int:
    n = C.c_int64()
    _check(h, _lib.rdm_get_p1_nnzb(h, sys, direction, C.byref(n)))
    return int(n.value)


def rdm_get_p0(h, sys: int = 0, out=None) -> BsrResult:
    return _fetch(h, _lib.rdm_get_p0, sys, out=out)


def rdm_get_p1(h, sys: int = 0, direction: int = 0, out=None) -> BsrResult:
    return _fetch(h, _lib.rdm_get_p1, sys, direction, out=out)


def rdm_get_alpha(h, sys: int = 0) -> np.ndarray:
    a = (C.c_double * 9)()
    _check(h, _lib.rdm_get_alpha(h, sys, a))
    return np.array(list(a)).reshape(3, 3)


def rdm_get_log(h) -> list:
    n = C.c_int()
    _check(h, _lib.rdm_get_log(h, None, 0, C.byref(n)))
    buf = (rdm_iter_log * max(n.value, 1))()
    _check(h, _lib.rdm_get_log(h, buf, n.value, C.byref(n)))
    out = []
    for r in buf[: n.value]:
        out.append({"iter": r.iter, "branch": r.branch, "tier": r.tier, "sys": r.sys,
                    "trace": r.trace, "idempotency": r.idempotency, "eb0": r.eb0,
                    "eb1": list(r.eb1), "nnzb0": r.nnzb0, "nnzb1": list(r.nnzb1), "ms": r.ms})
    return out


def rdm_block_product(h, A, B, X, c_lin: float, c_sq: float, terms: int, tau: float,
                      mode: int = MODE_FP64) -> BsrResult:
    sa, ka = to_bsr(A)
    sb, kb = to_bsr(B) if B is not None else (None, None)
    sx, kx = to_bsr(X) if X is not None else (None, None)
    pa = C.byref(sa)
    pb = C.byref(sb) if sb is not None else None
    px = C.byref(sx) if sx is not None else None
    need = C.c_int64()
    _check(h, _lib.rdm_block_product(h, pa, pb, px, c_lin, c_sq, terms, tau, mode, None, C.byref(need)))
    nnz = int(need.value)
    nb, b = int(A.nb), int(A.b)
    rp = np.zeros(nb + 1, dtype=np.int32)
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    va = np.zeros((max(nnz, 1), b, b), dtype=np.float64)
    out = rdm_bsr_out(nb, b, 0, nnz, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    _check(h, _lib.rdm_block_product(h, pa, pb, px, c_lin, c_sq, terms, tau, mode, C.byref(out), None))
    del ka, kb, kx
    return BsrResult(nb, b, int(A.n), rp, ci[:nnz].copy(), va[:nnz].copy())


def rdm_bsr_dot_noalloc(A, B, out_ptr: int, stream=None) -> None:
    """<A, B> of two device BSR matrices into the device double at out_ptr,
    without any device allocation (see include/rdm.h)."""
    sa, ka = to_bsr(A)
    sb, kb = to_bsr(B)
    code = _lib.rdm_bsr_dot_noalloc(C.byref(sa), C.byref(sb), C.c_void_p(out_ptr), stream)
    del ka, kb
    if code != RDM_OK:
        raise RdmError(code, "rdm_bsr_dot_noalloc failed (device matrices with equal nb, b required; "
                             "nb <= 262144)")


def rdm_set_test_knobs(h, tc_wait_cycles: int = 0, tc_hold: int = 0, tc_window_cols: int = 0,
                       tc_block_copies: int = 0) -> None:
    """Test settings of the tensor-core path (see include/rdm.h); all zeros
    restore production behaviour."""
    k = rdm_test_knobs(tc_wait_cycles, tc_hold, tc_window_cols, tc_block_copies, 0)
    _check(h, _lib.rdm_set_test_knobs(h, C.byref(k)))


# ---- convenience wrapper ---------------------------------------------------

class Solver:
    """One library handle.  ``Solver(device, stream)``; the stream defaults
    to torch's current CUDA stream when torch is importable."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = None
        self.h = rdm_create(device, stream)

    def close(self):
        if self.h:
            rdm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        p = rdm_default_params()
        for k, v in kw.items():
            if k == "mode" and isinstance(v, str):
                v = MODES[v]
            setattr(p, k, v)
        rdm_set_params(self.h, p)
        return p

    def load(self, systems, n_electrons=None):
        """Upload one system (or a list: a batch).  Each entry needs h0, h1
        (list of matrices for directions ``dirs``) and n_electrons."""
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        rdm_batch_create(self.h, len(systems))
        for s, y in enumerate(systems):
            ne = n_electrons if n_electrons is not None else y.n_electrons
            rdm_upload_h0(self.h, s, y.h0, ne)
            dirs = getattr(y, "dirs", ("x", "y", "z")[: len(y.h1)])
            for d, m in zip(dirs, y.h1):
                rdm_upload_h1(self.h, s, "xyz".index(d), m)
            if getattr(y, "s", None) is not None:
                rdm_upload_s(self.h, s, y.s)

    def solve(self):
        code, info = rdm_solve(self.h)
        return code, info

    def solve_async(self):
        rdm_solve_async(self.h)

    def sync(self):
        return rdm_sync(self.h)

    def p0(self, sys: int = 0, out=None) -> BsrResult:
        return rdm_get_p0(self.h, sys, out=out)

    def p1(self, sys: int = 0, direction: int = 0, out=None) -> BsrResult:
        return rdm_get_p1(self.h, sys, direction, out=out)

    def alpha(self, sys: int = 0) -> np.ndarray:
        return rdm_get_alpha(self.h, sys)

    def log(self) -> list:
        return rdm_get_log(self.h)

    def info(self, sys: int = 0) -> rdm_info:
        return rdm_get_info(self.h, sys)
