"""Seeded synthetic sparse inputs shared by the oracle, the tests and the bench.

This module holds no SpGEMM arithmetic: it only draws matrices and converts
between storage formats (CSC <-> CSR is a stable reordering of the same
entries).  Every generator is deterministic for a given seed.

Workload shapes follow the paper's inputs:
  * Erdos-Renyi (ER): "d nonzeros uniformly distributed in each column"
    (Sec. II-A).  Read here as exactly d distinct rows per column, drawn
    uniformly without replacement, so flop(A*A) = n*d^2 exactly.
  * R-MAT with quadrant probabilities (a, b, c, d) (Sec. IV-C, Graph500
    setting 0.57/0.19/0.19/0.05); duplicate edges removed, self loops kept,
    no vertex permutation.
  * 3-D 7-point Poisson operator with Dirichlet truncation and the 2x2x2
    piecewise-constant aggregation prolongator (AMG Galerkin product).
  * Column-stochastic R-MAT matrices (Markov clustering squaring).
Values are uniform(-1, 1) unless a generator states otherwise.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSC:
    nrows: int
    ncols: int
    colptr: np.ndarray  # int32 [ncols+1]
    rowidx: np.ndarray  # int32 [nnz]
    val: np.ndarray     # float64 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowidx.shape[0])


@dataclass
class CSR:
    nrows: int
    ncols: int
    rowptr: np.ndarray  # int32 [nrows+1]
    colidx: np.ndarray  # int32 [nnz]
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])


def _ptr_from_counts(counts: np.ndarray) -> np.ndarray:
    ptr = np.zeros(counts.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    if ptr[-1] >= 2**31:
        raise OverflowError("nnz does not fit int32 pointers")
    return ptr.astype(np.int32)


def coo_to_csc(nrows: int, ncols: int, row: np.ndarray, col: np.ndarray, val: np.ndarray) -> CSC:
    """Stable reorder of (row, col, val) entries into CSC (column-major)."""
    order = np.argsort(col, kind="stable")
    counts = np.bincount(col, minlength=ncols)
    return CSC(nrows, ncols, _ptr_from_counts(counts), row[order].astype(np.int32),
               np.ascontiguousarray(val[order]))


def coo_to_csr(nrows: int, ncols: int, row: np.ndarray, col: np.ndarray, val: np.ndarray) -> CSR:
    """Stable reorder of (row, col, val) entries into CSR (row-major)."""
    order = np.argsort(row, kind="stable")
    counts = np.bincount(row, minlength=nrows)
    return CSR(nrows, ncols, _ptr_from_counts(counts), col[order].astype(np.int32),
               np.ascontiguousarray(val[order]))


def csc_entries(A: CSC):
    """(row, col, val) arrays of a CSC matrix in storage order."""
    col = np.repeat(np.arange(A.ncols, dtype=np.int64), np.diff(A.colptr.astype(np.int64)))
    return A.rowidx.astype(np.int64), col, A.val


def csr_entries(B: CSR):
    row = np.repeat(np.arange(B.nrows, dtype=np.int64), np.diff(B.rowptr.astype(np.int64)))
    return row, B.colidx.astype(np.int64), B.val


def csc_to_csr(A: CSC) -> CSR:
    r, c, v = csc_entries(A)
    return coo_to_csr(A.nrows, A.ncols, r, c, v)


def csr_to_csc(B: CSR) -> CSC:
    r, c, v = csr_entries(B)
    return coo_to_csc(B.nrows, B.ncols, r, c, v)


def transpose_csr_as_csc(B: CSR) -> CSC:
    """The CSR arrays of B read as the CSC arrays of B^T (no data movement)."""
    return CSC(B.ncols, B.nrows, B.rowptr, B.colidx, B.val)


def _uniform_vals(rng: np.random.Generator, n: int, dtype) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, n).astype(dtype)


def er_csc(n: int, d: int, seed: int, *, nrows: int | None = None, dtype=np.float64,
           shuffle_within: bool = False) -> CSC:
    """ER matrix: exactly d distinct rows per column, uniform without replacement.

    Shape nrows x n (nrows defaults to n).  Rows inside a column are ascending
    unless ``shuffle_within`` is set (the library must not rely on order).
    """
    m = n if nrows is None else nrows
    if d > m:
        raise ValueError("d must not exceed the number of rows")
    rng = np.random.default_rng(seed)
    draws = rng.integers(0, m, size=(n, d), dtype=np.int64)
    draws.sort(axis=1)
    while True:
        dup = (draws[:, 1:] == draws[:, :-1]).any(axis=1) if d > 1 else np.zeros(n, bool)
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        redo = rng.integers(0, m, size=(bad.size, d), dtype=np.int64)
        redo.sort(axis=1)
        draws[bad] = redo
    val = _uniform_vals(rng, n * d, dtype).reshape(n, d)
    if shuffle_within:
        # same entries, stored in a random order inside each column
        perm = rng.permuted(np.tile(np.arange(d), (n, 1)), axis=1)
        draws = np.take_along_axis(draws, perm, axis=1)
        val = np.take_along_axis(val, perm, axis=1)
    rowidx = draws.reshape(-1).astype(np.int32)
    colptr = (np.arange(n + 1, dtype=np.int64) * d).astype(np.int32)
    return CSC(m, n, colptr, rowidx, np.ascontiguousarray(val.reshape(-1)))


def rmat_coo(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    """R-MAT edges (row, col) of a 2^scale square matrix, duplicates removed.

    Each edge descends ``scale`` levels of the recursive 2x2 quadrant split
    with probabilities (a, b; c, 1-a-b-c).  Output is sorted by (row, col).
    """
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(seed)
    row = np.zeros(m, np.int64)
    col = np.zeros(m, np.int64)
    top = a + b
    for bit in range(scale):
        u = rng.random(m)
        v = rng.random(m)
        lower = u >= top                      # bottom half: quadrants c, d
        right = np.where(lower, v >= c / (1.0 - top), v >= a / top)
        row |= lower.astype(np.int64) << bit
        col |= right.astype(np.int64) << bit
    key = np.unique(row * n + col)
    return n, key // n, key % n, rng


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19, dtype=np.float64):
    """R-MAT matrix as (CSC, CSR) pair of the same entries, values U(-1,1)."""
    n, row, col, rng = rmat_coo(scale, edge_factor, a, b, c, seed)
    val = _uniform_vals(rng, row.shape[0], dtype)
    return coo_to_csc(n, n, row, col, val), coo_to_csr(n, n, row, col, val)


def er(n: int, d: int, seed: int, dtype=np.float64, shuffle_within: bool = False):
    """ER matrix as (CSC, CSR) pair of the same entries."""
    A = er_csc(n, d, seed, dtype=dtype, shuffle_within=shuffle_within)
    return A, csc_to_csr(A)


def random_sparse(m: int, n: int, density: float, seed: int, dtype=np.float64):
    """Bernoulli(density) pattern with U(-1,1) values, as (CSC, CSR)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    r, c = np.nonzero(mask)
    v = _uniform_vals(rng, r.shape[0], dtype)
    return coo_to_csc(m, n, r, c, v), coo_to_csr(m, n, r, c, v)


def poisson7(N: int, dtype=np.float64) -> CSR:
    """3-D 7-point Laplacian on an N^3 grid, Dirichlet truncation.

    Diagonal 6, -1 for each face neighbour inside the grid.  Symmetric, so the
    returned CSR arrays are also its CSC arrays.
    """
    idx = np.arange(N ** 3, dtype=np.int64)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    rows = [idx]
    cols = [idx]
    vals = [np.full(idx.shape, 6.0)]
    for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        xx, yy, zz = x + dx, y + dy, z + dz
        ok = (xx >= 0) & (xx < N) & (yy >= 0) & (yy < N) & (zz >= 0) & (zz < N)
        rows.append(idx[ok])
        cols.append((xx + N * yy + N * N * zz)[ok])
        vals.append(np.full(int(ok.sum()), -1.0))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals).astype(dtype)
    return coo_to_csr(N ** 3, N ** 3, r, c, v)


def aggregation_prolongator(N: int, dtype=np.float64) -> CSR:
    """Piecewise-constant 2x2x2 aggregation P (N^3 x (N/2)^3), one 1.0 per row."""
    if N % 2:
        raise ValueError("N must be even")
    M = N // 2
    idx = np.arange(N ** 3, dtype=np.int64)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    agg = (x // 2) + M * (y // 2) + M * M * (z // 2)
    return coo_to_csr(N ** 3, M ** 3, idx, agg, np.ones(N ** 3, dtype=dtype))


def column_stochastic(A: CSC, dtype=np.float32):
    """Markov matrix from a square pattern, as in Markov clustering.

    A self loop is added to every vertex that lacks one (so no column is
    empty), then |values| are normalised so every column sums to 1.
    Returns (CSC, CSR) of the same entries.
    """
    r, c, v = csc_entries(A)
    has_loop = np.zeros(A.ncols, bool)
    has_loop[c[r == c]] = True
    add = np.nonzero(~has_loop)[0]
    r = np.concatenate([r, add])
    c = np.concatenate([c, add])
    v = np.concatenate([v.astype(np.float64), np.ones(add.shape[0])])
    w = np.abs(v.astype(np.float64)) + 1e-3
    colsum = np.bincount(c, weights=w, minlength=A.ncols)
    w = (w / colsum[c]).astype(dtype)
    return coo_to_csc(A.nrows, A.ncols, r, c, w), coo_to_csr(A.nrows, A.ncols, r, c, w)


def identity(n: int, dtype=np.float64):
    i = np.arange(n, dtype=np.int64)
    v = np.ones(n, dtype=dtype)
    return coo_to_csc(n, n, i, i, v), coo_to_csr(n, n, i, i, v)


def permutation(n: int, seed: int, dtype=np.float64):
    """P with P[i, perm[i]] = 1, as (CSC, CSR, perm)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    i = np.arange(n, dtype=np.int64)
    v = np.ones(n, dtype=dtype)
    return coo_to_csc(n, n, i, perm, v), coo_to_csr(n, n, i, perm, v), perm


def batch_er_shapes(count: int, seed: int, n_lo: int = 512, n_hi: int = 65536,
                    d_lo: int = 2, d_hi: int = 16):
    """(n_i, d_i) for a batch: n log-uniform in [n_lo, n_hi], d uniform in {d_lo..d_hi}."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64)
    n = np.clip(n, n_lo, n_hi)
    d = rng.integers(d_lo, d_hi + 1, count)
    return [(int(a), int(b)) for a, b in zip(n, d)]
