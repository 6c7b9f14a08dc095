"""Roofline byte model of PB-SpGEMM (pure arithmetic on sizes, no data).

Sec. II-C gives the arithmetic intensity bounds; Tab. III gives the bytes each
phase moves.  ``bytes_alg`` restates Tab. III with this build's real element
sizes instead of the paper's flat b = 16 bytes per nonzero:

  symbolic  reads both pointer arrays (Alg. 3) and A's row ids (per-row flop)
  expand    reads A and B once, writes flop tuples            (Tab. III)
  sort      reads flop tuples once (the in-shared-memory passes are not DRAM)
  compress  writes nnz(C) entries and the row pointer         (Tab. III)

The paper counts only multiplications as flops (Sec. II-A); ``gflops_2x``
reports 2 x multiplications (multiply + add), the convention of the metric.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


def ai_upper(cf: float, b: float) -> float:
    """Eq. 1: AI <= cf / b when A, B and C are each touched once."""
    return cf / b


def ai_col_lower(cf: float, b: float) -> float:
    """Column SpGEMM bound with A re-read flop times: cf / ((2 + cf) b)."""
    return cf / ((2.0 + cf) * b)


def ai_outer_lower(cf: float, b: float) -> float:
    """Outer-product ESC bound with 2*flop tuple traffic: cf / ((3 + 2 cf) b)."""
    return cf / ((3.0 + 2.0 * cf) * b)


def peak_flops(beta: float, ai: float) -> float:
    """Roofline ceiling beta * AI (units follow beta)."""
    return beta * ai


def key_bits(n_cols: int, rows_per_bin: int) -> tuple[int, int]:
    """(row bits, col bits) of a packed in-bin key (Sec. III-D key squeezing)."""
    col = max(1, math.ceil(math.log2(max(n_cols, 2))))
    row = 0 if rows_per_bin <= 1 else math.ceil(math.log2(rows_per_bin))
    return row, col


@dataclass
class Bytes:
    symbolic: int
    expand: int
    sort: int
    compress: int

    @property
    def total(self) -> int:
        return self.symbolic + self.expand + self.sort + self.compress

    @property
    def numeric(self) -> int:
        return self.expand + self.sort + self.compress


def bytes_alg(m: int, k: int, nnz_a: int, nnz_b: int, flop: int, nnz_c: int, *,
              val_in: int = 8, tuple_bytes: int = 12, val_out: int = 8, idx: int = 4,
              rowptr_out: int = 8) -> Bytes:
    """Algorithmic DRAM bytes of one product C = A*B (A m x k CSC, B k x n CSR)."""
    ptr_in = 4 * (k + 1)
    symbolic = 2 * ptr_in + idx * nnz_a
    expand = 2 * ptr_in + (idx + val_in) * (nnz_a + nnz_b) + tuple_bytes * flop
    sort = tuple_bytes * flop
    compress = (idx + val_out) * nnz_c + rowptr_out * (m + 1)
    return Bytes(symbolic, expand, sort, compress)


def gflops_2x(flop: int, seconds: float) -> float:
    return 2.0 * flop / seconds / 1e9
