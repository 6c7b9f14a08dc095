"""CPU oracle for PB-SpGEMM -- test infrastructure, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
never calls the CUDA library; the two share no code.  The arithmetic lives in
``pb_oracle.c`` (plain C, FP64, OpenMP over rows); this file only compiles it
with gcc on first use and marshals numpy arrays.

Functions (each cites the passage it follows in ``pb_oracle.c``):
  flop(A, B)          Alg. 3 total multiplications.
  row_flop(A, B)      Sec. III-B per-row multiplications.
  expand(A, B)        Alg. 2 expand loop: every (row, col, a*b) tuple.
  spgemm(A, B, rows)  C = A*B by definition (Gustavson + dense accumulator),
                      optionally only for the listed rows; also returns
                      sum |a_ik b_kj| per output entry.

All products are computed in FP64; FP32 inputs are widened exactly first.
Parity is pinned by ``tests/test_oracle.py`` against dense matmul, identity and
permutation products, ER and AMG closed forms (see that file).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pb_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pb_oracle.c into oracle/_build/liboracle.so with gcc (-O2 -fopenmp)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.pb_oracle_threads.restype = ctypes.c_int
            lib.pb_oracle_set_threads.restype = None
            lib.pb_oracle_set_threads.argtypes = [ctypes.c_int]
            lib.pb_oracle_flop.restype = i64
            lib.pb_oracle_flop.argtypes = [i32, i32p, i32p]
            lib.pb_oracle_row_flop.restype = None
            lib.pb_oracle_row_flop.argtypes = [i32, i32, i32p, i32p, i32p, i64p]
            lib.pb_oracle_expand.restype = None
            lib.pb_oracle_expand.argtypes = [i32, i32p, i32p, f64p, i32p, i32p, f64p, i32p, i32p, f64p]
            lib.pb_oracle_prepare.restype = ctypes.c_void_p
            lib.pb_oracle_prepare.argtypes = [i32, i32, i32p, i32p, f64p]
            lib.pb_oracle_release.restype = None
            lib.pb_oracle_release.argtypes = [ctypes.c_void_p]
            lib.pb_oracle_spgemm_count.restype = ctypes.c_int
            lib.pb_oracle_spgemm_count.argtypes = [ctypes.c_void_p, i32, i32p, i32p, i64, i64p, i64p]
            lib.pb_oracle_spgemm_fill.restype = ctypes.c_int
            lib.pb_oracle_spgemm_fill.argtypes = [ctypes.c_void_p, i32, i32p, i32p, f64p, i64, i64p, i64p,
                                                  i32p, f64p, f64p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return int(_load().pb_oracle_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of later oracle calls."""
    _load().pb_oracle_set_threads(int(n))


def _check(A, B):
    if A.ncols != B.nrows:
        raise ValueError(f"inner dimensions differ: A is {A.nrows}x{A.ncols}, B is {B.nrows}x{B.ncols}")


def flop(A, B) -> int:
    _check(A, B)
    return int(_load().pb_oracle_flop(A.ncols, _p(_i32(A.colptr), ctypes.c_int32),
                                      _p(_i32(B.rowptr), ctypes.c_int32)))


def row_flop(A, B) -> np.ndarray:
    _check(A, B)
    out = np.zeros(A.nrows, dtype=np.int64)
    _load().pb_oracle_row_flop(A.nrows, A.ncols, _p(_i32(A.colptr), ctypes.c_int32),
                               _p(_i32(A.rowidx), ctypes.c_int32), _p(_i32(B.rowptr), ctypes.c_int32),
                               _p(out, ctypes.c_int64))
    return out


def expand(A, B):
    """All flop tuples (row, col, val) in the outer-product loop order of Alg. 2."""
    _check(A, B)
    f = flop(A, B)
    row = np.empty(f, np.int32)
    col = np.empty(f, np.int32)
    val = np.empty(f, np.float64)
    _load().pb_oracle_expand(A.ncols, _p(_i32(A.colptr), ctypes.c_int32), _p(_i32(A.rowidx), ctypes.c_int32),
                             _p(_f64(A.val), ctypes.c_double), _p(_i32(B.rowptr), ctypes.c_int32),
                             _p(_i32(B.colidx), ctypes.c_int32), _p(_f64(B.val), ctypes.c_double),
                             _p(row, ctypes.c_int32), _p(col, ctypes.c_int32), _p(val, ctypes.c_double))
    return row, col, val


@dataclass
class Product:
    """C = A*B restricted to ``rows`` (all rows when rows is None).

    rowptr[t]..rowptr[t+1] delimit the entries of rows[t]; colidx ascending.
    absval holds sum_k |A(i,k) B(k,j)| for each entry (error-bound scale).
    """
    rows: np.ndarray
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray
    absval: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def spgemm(A, B, rows=None) -> Product:
    _check(A, B)
    lib = _load()
    if rows is None:
        rows = np.arange(A.nrows, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    colptrA, rowidxA, valA = _i32(A.colptr), _i32(A.rowidx), _f64(A.val)
    rowptrB, colidxB, valB = _i32(B.rowptr), _i32(B.colidx), _f64(B.val)
    ctx = lib.pb_oracle_prepare(A.nrows, A.ncols, _p(colptrA, ctypes.c_int32), _p(rowidxA, ctypes.c_int32),
                                _p(valA, ctypes.c_double))
    if not ctx:
        raise MemoryError("oracle: row view of A")
    try:
        cnt = np.zeros(rows.shape[0], dtype=np.int64)
        rc = lib.pb_oracle_spgemm_count(ctx, B.ncols, _p(rowptrB, ctypes.c_int32), _p(colidxB, ctypes.c_int32),
                                        rows.shape[0], _p(rows, ctypes.c_int64), _p(cnt, ctypes.c_int64))
        if rc != 0:
            raise MemoryError("oracle count pass failed")
        ptr = np.zeros(rows.shape[0] + 1, dtype=np.int64)
        np.cumsum(cnt, out=ptr[1:])
        nnz = int(ptr[-1])
        col = np.empty(max(nnz, 1), np.int32)
        val = np.empty(max(nnz, 1), np.float64)
        absval = np.empty(max(nnz, 1), np.float64)
        rc = lib.pb_oracle_spgemm_fill(ctx, B.ncols, _p(rowptrB, ctypes.c_int32), _p(colidxB, ctypes.c_int32),
                                       _p(valB, ctypes.c_double), rows.shape[0], _p(rows, ctypes.c_int64),
                                       _p(ptr, ctypes.c_int64), _p(col, ctypes.c_int32),
                                       _p(val, ctypes.c_double), _p(absval, ctypes.c_double))
        if rc != 0:
            raise MemoryError("oracle fill pass failed")
    finally:
        lib.pb_oracle_release(ctx)
    return Product(rows, ptr, col[:nnz], val[:nnz], absval[:nnz])
