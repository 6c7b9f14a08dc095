"""Thin Python binding of libpbspgemm (ctypes over the C ABI in include/pb_spgemm.h).

Only argument marshalling lives here: torch tensors become device pointers,
the current torch stream becomes the cudaStream_t, and torch's caching
allocator provides the plan's device memory.  Every step of the product runs
in the CUDA library; there is no CPU path.  If the library cannot be built or
loaded the calls raise.

Names follow the C ABI: ``symbolic`` / ``numeric`` / ``plan_status`` mirror
``pb_spgemm_symbolic`` / ``pb_spgemm_numeric`` / ``pb_plan_status``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import build as _build

PB_F64, PB_F32, PB_F64_F32TUPLE = 0, 1, 2
STATUS_NAMES = {0: "PB_OK", 1: "PB_ERR_INVALID_ARG", 2: "PB_ERR_SHAPE", 3: "PB_ERR_UNSUPPORTED_DTYPE",
                4: "PB_ERR_OOM", 5: "PB_ERR_OVERFLOW", 6: "PB_ERR_CUDA", 7: "PB_ERR_TIMEOUT", 8: "PB_ERR_BUSY",
                9: "PB_ERR_UNSUPPORTED", 10: "PB_ERR_WORKSPACE"}
_IN_DTYPE = {PB_F64: torch.float64, PB_F32: torch.float32, PB_F64_F32TUPLE: torch.float64}
_OUT_DTYPE = _IN_DTYPE


class PBError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


class _CSC(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _CSR(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _CSROut(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("cap", ctypes.c_int64),
                ("rowptr64", ctypes.c_void_p), ("rowptr32", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("nnz_dev", ctypes.c_void_p)]


class _Config(ctypes.Structure):
    _fields_ = [("bin_capacity", ctypes.c_int32), ("sort_threads", ctypes.c_int32),
                ("expand_chunk", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("max_tuple_bytes", ctypes.c_int64), ("min_panels", ctypes.c_int64)]


class _CSRHost(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("cap", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("nnz", ctypes.c_int64)]


class _BatchTune(ctypes.Structure):
    _fields_ = [("log2n", ctypes.c_int32), ("dclass", ctypes.c_int32), ("bin_capacity", ctypes.c_int32),
                ("rmax_log2", ctypes.c_int32), ("expand_chunk", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("A", _CSC), ("B", _CSR)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

# Exported symbols of the library with their C signatures (kept in step with the header).
_VP, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "pb_version": (_I32, []),
    "pb_create": (ctypes.c_int, [ctypes.POINTER(_VP)]),
    "pb_destroy": (ctypes.c_int, [_VP]),
    "pb_set_allocator": (ctypes.c_int, [_VP, _ALLOC_FN, _FREE_FN, _VP]),
    "pb_last_error": (ctypes.c_char_p, [_VP]),
    "pb_spgemm_symbolic": (ctypes.c_int, [_VP, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR), ctypes.c_int,
                                          ctypes.POINTER(_Config), _VP, ctypes.POINTER(_VP)]),
    "pb_plan_query": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_SZ),
                                     ctypes.POINTER(_I64), ctypes.POINTER(_I32)]),
    "pb_spgemm_numeric": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR),
                                         ctypes.POINTER(_CSROut), _VP, _SZ, _VP]),
    "pb_plan_status": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int)]),
    "pb_plan_export": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "pb_debug_expand": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR), _VP, _SZ, _VP]),
    "pb_debug_values_offset": (_SZ, [_VP]),
    "pb_debug_tuple_layout": (ctypes.c_int32, [_VP]),
    "pb_plan_destroy": (ctypes.c_int, [_VP]),
    "pb_set_phase_events": (ctypes.c_int, [_VP, _VP]),
    "pb_kernel_launches": (_I64, []),
    "pb_spgemm_host": (ctypes.c_int, [_VP, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR), ctypes.c_int,
                                      ctypes.POINTER(_Config), ctypes.POINTER(_CSRHost), _VP,
                                      ctypes.POINTER(ctypes.c_int)]),
    "pb_validate_operands": (ctypes.c_int, [_VP, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR), _VP,
                                            ctypes.POINTER(ctypes.c_int)]),
    "pb_spgemm_noalloc": (ctypes.c_int, [ctypes.POINTER(_CSC), ctypes.POINTER(_CSR), ctypes.c_int,
                                         ctypes.POINTER(_CSROut), _VP, ctypes.POINTER(ctypes.c_int)]),
    "pb_spgemm_batch_query": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR), ctypes.c_int,
                                             _VP, ctypes.POINTER(_SZ), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "pb_spgemm_batch": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR),
                                       ctypes.POINTER(_CSROut), ctypes.c_int, _VP, _SZ, _VP, _VP]),
    "pb_batch_autotune": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_CSC), ctypes.POINTER(_CSR),
                                         ctypes.POINTER(_CSROut), ctypes.c_int, _VP, _SZ, _VP, _I32]),
    "pb_batch_get_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(_BatchTune), _I32, ctypes.POINTER(_I32)]),
    "pb_batch_set_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(_BatchTune), _I32]),
    "pb_server_create": (ctypes.c_int, [_VP, _SZ, _I32, ctypes.POINTER(_VP)]),
    "pb_server_destroy": (ctypes.c_int, [_VP]),
    "pb_serve_submit": (ctypes.c_int, [_VP, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]),
    "pb_serve_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_int)]),
    "pb_serve_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "pb_serve_result": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(_CSROut)]),
    "pb_serve_timing": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "pb_serve_release": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "pb_serve_stats": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_SZ),
                                      ctypes.POINTER(_SZ)]),
    "pb_server_set_batching": (ctypes.c_int, [_VP, _I32, ctypes.c_double]),
    "pb_serve_batch_stats": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
}

_lib = None
_lib_lock = threading.Lock()


def load_library(path: Optional[str] = None):
    """Build (if stale) and load libpbspgemm.so; declare every exported symbol."""
    global _lib
    with _lib_lock:
        if _lib is None:
            lib = ctypes.CDLL(path or os.environ.get("PB_LIBRARY") or _build.build())
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


# ---------------------------------------------------------------------------
# Device-memory provider: torch's caching allocator.
# ---------------------------------------------------------------------------
@_ALLOC_FN
def _torch_alloc(nbytes, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # noqa: BLE001 - an allocation failure becomes PB_ERR_OOM in the library
        return None


@_FREE_FN
def _torch_free(ptr, nbytes, stream, ctx):
    if ptr:
        torch.cuda.caching_allocator_delete(int(ptr))


# ---------------------------------------------------------------------------
# Matrices on the device.
# ---------------------------------------------------------------------------
@dataclass
class CscMatrix:
    nrows: int
    ncols: int
    colptr: torch.Tensor  # int32 [ncols+1]
    rowidx: torch.Tensor  # int32 [nnz]
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.rowidx.numel())

    def _c(self) -> _CSC:
        return _CSC(self.nrows, self.ncols, self.nnz, self.colptr.data_ptr(), self.rowidx.data_ptr() or None,
                    self.val.data_ptr() or None)


@dataclass
class CsrMatrix:
    nrows: int
    ncols: int
    rowptr: torch.Tensor  # int32 or int64 [nrows+1]
    colidx: torch.Tensor  # int32 [nnz]
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def _c(self) -> _CSR:
        if self.rowptr.dtype != torch.int32:
            raise PBError(1, "input CSR row pointers must be int32")
        return _CSR(self.nrows, self.ncols, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr() or None,
                    self.val.data_ptr() or None)


def _dev(a: np.ndarray, device, dtype=None) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def csc_to_device(A, device="cuda", val_dtype=None) -> CscMatrix:
    """Copy a host CSC (any object with nrows/ncols/colptr/rowidx/val) to the device."""
    return CscMatrix(A.nrows, A.ncols, _dev(A.colptr, device, torch.int32), _dev(A.rowidx, device, torch.int32),
                     _dev(A.val, device, val_dtype))


def csr_to_device(B, device="cuda", val_dtype=None) -> CsrMatrix:
    return CsrMatrix(B.nrows, B.ncols, _dev(B.rowptr, device, torch.int32), _dev(B.colidx, device, torch.int32),
                     _dev(B.val, device, val_dtype))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def _check(lib, h, status: int):
    if status != 0:
        msg = lib.pb_last_error(h).decode() if h else ""
        raise PBError(status, msg)


class Handle:
    """pb_handle bound to the current device; plan memory comes from torch."""

    def __init__(self, use_torch_allocator: bool = True):
        self.lib = load_library()
        h = ctypes.c_void_p()
        _check(self.lib, None, self.lib.pb_create(ctypes.byref(h)))
        self.ptr = h
        if use_torch_allocator:
            _check(self.lib, h, self.lib.pb_set_allocator(h, _torch_alloc, _torch_free, None))

    def __del__(self):
        if getattr(self, "ptr", None):
            self.lib.pb_destroy(self.ptr)
            self.ptr = None


def set_phase_events(handle: "Handle", events) -> None:
    """Record four torch.cuda.Event objects around the numeric phases (None disables)."""
    if events is None:
        _check(handle.lib, handle.ptr, handle.lib.pb_set_phase_events(handle.ptr, None))
        return
    for e in events:
        if not e.cuda_event:
            e.record()  # torch creates the CUDA event lazily, on first record
    arr = (ctypes.c_void_p * 4)(*[int(e.cuda_event) for e in events])
    handle._events = (events, arr)  # keep alive
    _check(handle.lib, handle.ptr, handle.lib.pb_set_phase_events(handle.ptr, arr))


def kernel_launches() -> int:
    return int(load_library().pb_kernel_launches())


_default_handle = None


def default_handle() -> Handle:
    global _default_handle
    if _default_handle is None:
        _default_handle = Handle()
    return _default_handle


def make_config(bin_capacity: int = 0, expand_chunk: int = 0, max_tuple_bytes: int = 0,
                deterministic: bool = False, min_panels: int = 0, sort_threads: int = 0) -> _Config:
    return _Config(bin_capacity, sort_threads, expand_chunk, 1 if deterministic else 0, max_tuple_bytes,
                   min_panels)


class Plan:
    """Result of the symbolic phase; owns plan arrays on the device."""

    def __init__(self, handle: Handle, ptr: ctypes.c_void_p, dtype: int, A: CscMatrix, B: CsrMatrix):
        self.handle, self.ptr, self.dtype = handle, ptr, dtype
        self.m, self.k, self.n = A.nrows, A.ncols, B.ncols
        flop, ccap, nbins = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ws, npan = ctypes.c_size_t(), ctypes.c_int32()
        _check(handle.lib, handle.ptr, handle.lib.pb_plan_query(ptr, ctypes.byref(flop), ctypes.byref(ccap),
                                                                 ctypes.byref(ws), ctypes.byref(nbins),
                                                                 ctypes.byref(npan)))
        self.flop, self.c_cap, self.workspace_bytes = flop.value, ccap.value, ws.value
        self.nbins, self.npanels = nbins.value, npan.value

    def __del__(self):
        if getattr(self, "ptr", None):
            self.handle.lib.pb_plan_destroy(self.ptr)
            self.ptr = None

    def status(self, stream=None) -> int:
        st = ctypes.c_int()
        _check(self.handle.lib, self.handle.ptr,
               self.handle.lib.pb_plan_status(self.ptr, _stream_ptr(stream), ctypes.byref(st)))
        return st.value

    def export(self, stream=None):
        """(F, R, bin_row, bin_off) device tensors copied out of the plan."""
        dev = torch.device("cuda")
        F = torch.empty(self.k + 1, dtype=torch.int64, device=dev)
        R = torch.empty(self.m + 1, dtype=torch.int64, device=dev)
        br = torch.empty(self.nbins + 1, dtype=torch.int32, device=dev)
        bo = torch.empty(self.nbins + 1, dtype=torch.int64, device=dev)
        _check(self.handle.lib, self.handle.ptr,
               self.handle.lib.pb_plan_export(self.ptr, F.data_ptr(), R.data_ptr(), br.data_ptr(), bo.data_ptr(),
                                              _stream_ptr(stream)))
        return F, R, br, bo

    def workspace(self) -> torch.Tensor:
        return torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device="cuda")


def symbolic(A: CscMatrix, B: CsrMatrix, dtype: int = PB_F64, config: Optional[_Config] = None,
             handle: Optional[Handle] = None, stream=None) -> Plan:
    h = handle or default_handle()
    for t, want in ((A.val, _IN_DTYPE.get(dtype)), (B.val, _IN_DTYPE.get(dtype))):
        if want is not None and t.dtype != want:
            raise PBError(3, f"values must be {want} for dtype {dtype}")
    cA, cB = A._c(), B._c()
    out = ctypes.c_void_p()
    cfg = ctypes.byref(config) if config is not None else None
    _check(h.lib, h.ptr, h.lib.pb_spgemm_symbolic(h.ptr, ctypes.byref(cA), ctypes.byref(cB), dtype, cfg,
                                                  _stream_ptr(stream), ctypes.byref(out)))
    return Plan(h, out, dtype, A, B)


def numeric(plan: Plan, A: CscMatrix, B: CsrMatrix, C: CsrMatrix, workspace: torch.Tensor,
            nnz_out: Optional[torch.Tensor] = None, stream=None) -> None:
    """Run expand + sort + compress into C (C.colidx / C.val sized to its capacity)."""
    h = plan.handle
    cA, cB = A._c(), B._c()
    r64 = C.rowptr.data_ptr() if C.rowptr.dtype == torch.int64 else None
    r32 = C.rowptr.data_ptr() if C.rowptr.dtype == torch.int32 else None
    cC = _CSROut(C.nrows, C.ncols, C.colidx.numel(), r64, r32, C.colidx.data_ptr() or None,
                 C.val.data_ptr() or None, nnz_out.data_ptr() if nnz_out is not None else None)
    _check(h.lib, h.ptr, h.lib.pb_spgemm_numeric(h.ptr, plan.ptr, ctypes.byref(cA), ctypes.byref(cB),
                                                 ctypes.byref(cC), workspace.data_ptr(), workspace.numel(),
                                                 _stream_ptr(stream)))


def numeric_count(plan: Plan, A: CscMatrix, B: CsrMatrix, workspace: torch.Tensor, nnz_out: torch.Tensor,
                  stream=None) -> None:
    """Counting run: only nnz(C) is computed (into nnz_out), nothing is written to C."""
    h = plan.handle
    cA, cB = A._c(), B._c()
    cC = _CSROut(plan.m, plan.n, 0, None, None, None, None, nnz_out.data_ptr())
    _check(h.lib, h.ptr, h.lib.pb_spgemm_numeric(h.ptr, plan.ptr, ctypes.byref(cA), ctypes.byref(cB),
                                                 ctypes.byref(cC), workspace.data_ptr(), workspace.numel(),
                                                 _stream_ptr(stream)))


def debug_expand(plan: Plan, A: CscMatrix, B: CsrMatrix, workspace: torch.Tensor, stream=None):
    """Run only the expand phase; returns (keys uint32-as-int32 view, values) views of the workspace."""
    h = plan.handle
    cA, cB = A._c(), B._c()
    _check(h.lib, h.ptr, h.lib.pb_debug_expand(h.ptr, plan.ptr, ctypes.byref(cA), ctypes.byref(cB),
                                               workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)))
    return workspace, int(h.lib.pb_debug_values_offset(plan.ptr))


def debug_tuple_layout(plan: Plan) -> int:
    """1 when the plan's tuples are packed {key, value bits} pairs of uint32, 0 for separate arrays."""
    return int(plan.handle.lib.pb_debug_tuple_layout(plan.ptr))


def spgemm_noalloc(A: CscMatrix, B: CsrMatrix, C: CsrMatrix, dtype: int = PB_F64,
                   nnz_out: Optional[torch.Tensor] = None, stream=None) -> int:
    """C = A * B through pb_spgemm_noalloc (no device allocation by the library).

    C must be sized by the caller (capacity = C.colidx.numel()).  Returns the
    device-side status (0 = PB_OK); raises PBError for argument/size errors.
    """
    lib = load_library()
    cA, cB = A._c(), B._c()
    r64 = C.rowptr.data_ptr() if C.rowptr.dtype == torch.int64 else None
    r32 = C.rowptr.data_ptr() if C.rowptr.dtype == torch.int32 else None
    cC = _CSROut(C.nrows, C.ncols, C.colidx.numel(), r64, r32, C.colidx.data_ptr() or None,
                 C.val.data_ptr() or None, nnz_out.data_ptr() if nnz_out is not None else None)
    dev = ctypes.c_int()
    st = lib.pb_spgemm_noalloc(ctypes.byref(cA), ctypes.byref(cB), dtype, ctypes.byref(cC), _stream_ptr(stream),
                               ctypes.byref(dev))
    if st != 0:
        raise PBError(st, "pb_spgemm_noalloc")
    return dev.value


def alloc_output(plan: Plan, rowptr64: bool = True, cap: Optional[int] = None) -> CsrMatrix:
    cap = plan.c_cap if cap is None else cap
    dev = torch.device("cuda")
    return CsrMatrix(plan.m, plan.n,
                     torch.empty(plan.m + 1, dtype=torch.int64 if rowptr64 else torch.int32, device=dev),
                     torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
                     torch.empty(max(cap, 1), dtype=_OUT_DTYPE[plan.dtype], device=dev))


def spgemm_exact(A: CscMatrix, B: CsrMatrix, dtype: int = PB_F64, config: Optional[_Config] = None,
                 rowptr64: bool = True, handle: Optional[Handle] = None):
    """C = A * B with C allocated at exactly nnz(C) (a counting run first); returns (C, plan).

    For products whose flop-sized output would not fit in device memory.
    """
    plan = symbolic(A, B, dtype, config, handle)
    ws = plan.workspace()
    nnz = torch.zeros(1, dtype=torch.int64, device="cuda")
    numeric_count(plan, A, B, ws, nnz)
    if plan.status() != 0:
        raise PBError(plan.status(), "device-side error in the counting run")
    C = alloc_output(plan, rowptr64, cap=int(nnz.item()))
    numeric(plan, A, B, C, ws)
    st = plan.status()
    if st != 0:
        raise PBError(st, "device-side error in the numeric phase")
    k = int(nnz.item())
    return CsrMatrix(C.nrows, C.ncols, C.rowptr, C.colidx[:k], C.val[:k]), plan


def spgemm(A: CscMatrix, B: CsrMatrix, dtype: int = PB_F64, config: Optional[_Config] = None,
           rowptr64: bool = True, handle: Optional[Handle] = None) -> CsrMatrix:
    """C = A * B on the current stream; returns C trimmed to nnz(C).  Synchronises."""
    plan = symbolic(A, B, dtype, config, handle)
    C = alloc_output(plan, rowptr64)
    ws = plan.workspace()
    numeric(plan, A, B, C, ws)
    st = plan.status()
    if st != 0:
        raise PBError(st, "device-side error in the numeric phase")
    nnz = int(C.rowptr[-1].item())
    return CsrMatrix(C.nrows, C.ncols, C.rowptr, C.colidx[:nnz], C.val[:nnz])


# ---------------------------------------------------------------------------
# Batched products (pb_spgemm_batch).
# ---------------------------------------------------------------------------
class Batch:
    """A batch of independent products C[i] = A[i] * B[i] with its workspace.

    The struct arrays handed to the library are built once, so repeated
    run() calls (or a CUDA graph captured around one) cost only the launches.
    query() sizes the workspace and gives each product's flop (the C capacity
    that always suffices) and its largest per-row flop.
    """

    def __init__(self, As, Bs, dtype: int = PB_F64, handle: Optional[Handle] = None, rowptr64: bool = True,
                 caps=None, stream=None):
        self.handle = handle or default_handle()
        self.lib = self.handle.lib
        self.dtype = dtype
        self.As, self.Bs = list(As), list(Bs)
        n = len(self.As)
        if len(self.Bs) != n:
            raise PBError(1, "A and B lists differ in length")
        self.count = n
        self._cA = (_CSC * max(n, 1))(*[a._c() for a in self.As])
        self._cB = (_CSR * max(n, 1))(*[b._c() for b in self.Bs])
        ws = _SZ()
        self.flop = np.zeros(max(n, 1), dtype=np.int64)
        self.max_row = np.zeros(max(n, 1), dtype=np.int64)
        _check(self.lib, self.handle.ptr, self.lib.pb_spgemm_batch_query(
            self.handle.ptr, n, self._cA, self._cB, dtype, _stream_ptr(stream), ctypes.byref(ws),
            self.flop.ctypes.data_as(ctypes.POINTER(_I64)), self.max_row.ctypes.data_as(ctypes.POINTER(_I64))))
        self.flop, self.max_row = self.flop[:n], self.max_row[:n]
        self.workspace_bytes = int(ws.value) + 256
        dev = torch.device("cuda")
        self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=dev)
        self.device_status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.nnz = torch.zeros(max(n, 1), dtype=torch.int64, device=dev)
        caps = self.flop if caps is None else caps
        self.C = []
        outs = []
        for i in range(n):
            cap = max(int(caps[i]), 1)
            C = CsrMatrix(self.As[i].nrows, self.Bs[i].ncols,
                          torch.empty(self.As[i].nrows + 1, dtype=torch.int64 if rowptr64 else torch.int32,
                                      device=dev),
                          torch.empty(cap, dtype=torch.int32, device=dev),
                          torch.empty(cap, dtype=_OUT_DTYPE[dtype], device=dev))
            self.C.append(C)
            outs.append(_CSROut(C.nrows, C.ncols, cap, C.rowptr.data_ptr() if rowptr64 else None,
                                None if rowptr64 else C.rowptr.data_ptr(), C.colidx.data_ptr(), C.val.data_ptr(),
                                self.nnz.data_ptr() + 8 * i))
        self._cC = (_CSROut * max(n, 1))(*outs)

    def run(self, stream=None) -> None:
        """Launch the batch on `stream` (asynchronous; no allocation, no host sync)."""
        _check(self.lib, self.handle.ptr, self.lib.pb_spgemm_batch(
            self.handle.ptr, self.count, self._cA, self._cB, self._cC, self.dtype, self.workspace.data_ptr(),
            self.workspace_bytes, _stream_ptr(stream), self.device_status.data_ptr()))

    def status(self) -> int:
        """Device status of the last run (synchronises)."""
        return int(self.device_status.item())

    def autotune(self, reps: int = 3, stream=None) -> None:
        _check(self.lib, self.handle.ptr, self.lib.pb_batch_autotune(
            self.handle.ptr, self.count, self._cA, self._cB, self._cC, self.dtype, self.workspace.data_ptr(),
            self.workspace_bytes, _stream_ptr(stream), reps))

    def result(self, i: int) -> CsrMatrix:
        """Product i trimmed to its nnz (synchronises)."""
        C = self.C[i]
        k = int(self.nnz[i].item())
        return CsrMatrix(C.nrows, C.ncols, C.rowptr, C.colidx[:k], C.val[:k])


def get_tuning(handle: Optional[Handle] = None):
    """The handle's batch tuning table as a list of dicts."""
    h = handle or default_handle()
    n = _I32()
    _check(h.lib, h.ptr, h.lib.pb_batch_get_tuning(h.ptr, None, 0, ctypes.byref(n)))
    arr = (_BatchTune * max(n.value, 1))()
    _check(h.lib, h.ptr, h.lib.pb_batch_get_tuning(h.ptr, arr, n.value, ctypes.byref(n)))
    keys = ("log2n", "dclass", "bin_capacity", "rmax_log2", "expand_chunk")
    return [{k: int(getattr(arr[i], k)) for k in keys} for i in range(n.value)]


def set_tuning(entries, handle: Optional[Handle] = None) -> None:
    h = handle or default_handle()
    arr = (_BatchTune * max(len(entries), 1))(
        *[_BatchTune(e["log2n"], e["dclass"], e["bin_capacity"], e["rmax_log2"], e["expand_chunk"], 0)
          for e in entries])
    _check(h.lib, h.ptr, h.lib.pb_batch_set_tuning(h.ptr, arr, len(entries)))


# ---------------------------------------------------------------------------
# Serving (pb_server_*): continuous batching of product and Galerkin requests.
# ---------------------------------------------------------------------------
PB_REQ_PRODUCT = 0
PB_REQ_GALERKIN = 1


class _DevView:
    """A device array the server owns, exposed to torch without a copy."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def _view(ptr, n, dtype):
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device="cuda")
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_DevView(int(ptr), int(n), typestr), device="cuda")


class Server:
    """pb_server: requests are admitted as slots and HBM budget free up and overlap on the GPU."""

    def __init__(self, budget_bytes: int, max_slots: int = 4, handle: Optional[Handle] = None):
        self.handle = handle or default_handle()
        self.lib = self.handle.lib
        s = ctypes.c_void_p()
        _check(self.lib, self.handle.ptr, self.lib.pb_server_create(self.handle.ptr, budget_bytes, max_slots,
                                                                     ctypes.byref(s)))
        self.ptr = s
        self._keep = {}  # request id -> operands kept alive until release

    def _submit(self, kind, A: CscMatrix, B: CsrMatrix, dtype: int) -> int:
        req = _Request(kind, dtype, A._c(), B._c())
        rid = ctypes.c_uint64()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_submit(self.ptr, ctypes.byref(req), ctypes.byref(rid)))
        self._keep[rid.value] = (A, B, dtype, kind)
        return rid.value

    def submit_product(self, A: CscMatrix, B: CsrMatrix, dtype: int = PB_F64) -> int:
        """C = A * B."""
        return self._submit(PB_REQ_PRODUCT, A, B, dtype)

    def submit_galerkin(self, A: CscMatrix, P: CsrMatrix, dtype: int = PB_F64) -> int:
        """C = P^T (A P)."""
        return self._submit(PB_REQ_GALERKIN, A, P, dtype)

    def poll(self, rid: int):
        done, st = _I32(), ctypes.c_int()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_poll(self.ptr, rid, ctypes.byref(done), ctypes.byref(st)))
        return bool(done.value), int(st.value)

    def wait(self, rid: int) -> int:
        st = ctypes.c_int()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_wait(self.ptr, rid, ctypes.byref(st)))
        return int(st.value)

    def result(self, rid: int, copy: bool = True) -> CsrMatrix:
        """The finished request's C (cloned into torch memory unless copy=False)."""
        C = _CSROut()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_result(self.ptr, rid, ctypes.byref(C)))
        dtype = self._keep[rid][2]
        vt = _OUT_DTYPE[dtype]
        rp = _view(C.rowptr64, C.nrows + 1, torch.int64)
        ci = _view(C.colidx, C.cap, torch.int32)
        va = _view(C.val, C.cap, vt)
        if copy:
            rp, ci, va = rp.clone(), ci.clone(), va.clone()
        return CsrMatrix(C.nrows, C.ncols, rp, ci, va)

    def timing(self, rid: int):
        """(queued_ms, total_ms) of a finished request."""
        q, t = ctypes.c_double(), ctypes.c_double()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_timing(self.ptr, rid, ctypes.byref(q), ctypes.byref(t)))
        return q.value, t.value

    def release(self, rid: int) -> None:
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_release(self.ptr, rid))
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        c, p, u, k = _I64(), _I64(), _SZ(), _SZ()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_stats(self.ptr, ctypes.byref(c), ctypes.byref(p),
                                                                  ctypes.byref(u), ctypes.byref(k)))
        br, bl = _I64(), _I64()
        _check(self.lib, self.handle.ptr, self.lib.pb_serve_batch_stats(self.ptr, ctypes.byref(br), ctypes.byref(bl)))
        return {"completed": c.value, "preempted": p.value, "bytes_in_use": u.value, "peak_bytes": k.value,
                "batched_requests": br.value, "batch_launches": bl.value}

    def set_batching(self, max_requests: int, max_request_work: float) -> None:
        """Coalesce up to max_requests queued requests of at most max_request_work estimated work per launch."""
        _check(self.lib, self.handle.ptr, self.lib.pb_server_set_batching(self.ptr, max_requests,
                                                                          float(max_request_work)))

    def close(self) -> None:
        if getattr(self, "ptr", None):
            self.lib.pb_server_destroy(self.ptr)
            self.ptr = None
            self._keep.clear()

    def __del__(self):
        self.close()


def validate(A: CscMatrix, B: CsrMatrix, handle: Optional[Handle] = None, stream=None):
    """Device check of the operands' preconditions: (status, message); status 0 = valid."""
    h = handle or default_handle()
    cA, cB = A._c(), B._c()
    res = ctypes.c_int()
    _check(h.lib, h.ptr, h.lib.pb_validate_operands(h.ptr, ctypes.byref(cA), ctypes.byref(cB), _stream_ptr(stream),
                                                    ctypes.byref(res)))
    return int(res.value), (h.lib.pb_last_error(h.ptr).decode() if res.value else "")


def host_tensors(M, val_dtype=None, pin: bool = True):
    """Host (optionally pinned) torch copies of a host CSC/CSR, for pb_spgemm_host."""
    def t(a, dt=None):
        x = torch.from_numpy(np.ascontiguousarray(a))
        if dt is not None:
            x = x.to(dt)
        return x.pin_memory() if pin else x
    if hasattr(M, "colptr"):
        return CscMatrix(M.nrows, M.ncols, t(M.colptr, torch.int32), t(M.rowidx, torch.int32), t(M.val, val_dtype))
    return CsrMatrix(M.nrows, M.ncols, t(M.rowptr, torch.int32), t(M.colidx, torch.int32), t(M.val, val_dtype))


def spgemm_host(A: CscMatrix, B: CsrMatrix, C: CsrMatrix, dtype: int = PB_F64, config: Optional[_Config] = None,
                handle: Optional[Handle] = None, stream=None):
    """pb_spgemm_host: A, B and C in host memory (C preallocated: rowptr int64, colidx/val of any
    capacity).  Returns (nnz, device_status)."""
    h = handle or default_handle()
    cA, cB = A._c(), B._c()
    out = _CSRHost(A.nrows, B.ncols, int(C.colidx.numel()), C.rowptr.data_ptr(), C.colidx.data_ptr() or None,
                   C.val.data_ptr() or None, 0)
    dev = ctypes.c_int()
    cfg = ctypes.byref(config) if config is not None else None
    _check(h.lib, h.ptr, h.lib.pb_spgemm_host(h.ptr, ctypes.byref(cA), ctypes.byref(cB), dtype, cfg,
                                              ctypes.byref(out), _stream_ptr(stream), ctypes.byref(dev)))
    return int(out.nnz), int(dev.value)
