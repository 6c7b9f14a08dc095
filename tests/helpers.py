"""Shared test helpers: device copies and element-wise comparison with the oracle."""
import numpy as np

import oracle
import synth

EPS = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}
# |C_gpu - C_oracle| <= 64 * eps * sum_k |a_ik b_kj| per entry, eps the unit
# roundoff of the type the products are rounded to (FP64, or FP32 in the
# FP32 forms); structure (rowptr, colidx) must match exactly.
TOL_FACTOR = 64.0


def to_host(C):
    return (C.rowptr.cpu().numpy().astype(np.int64), C.colidx.cpu().numpy(),
            C.val.double().cpu().numpy())


def assert_matches(C, ref: oracle.Product, eps: float):
    rowptr, colidx, val = to_host(C)
    nnz = int(rowptr[-1])
    assert np.array_equal(rowptr, ref.rowptr), "row pointers differ"
    assert np.array_equal(colidx[:nnz], ref.colidx), "column indices differ"
    err = np.abs(val[:nnz] - ref.val)
    bound = TOL_FACTOR * eps * ref.absval
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{bad.size} values outside the bound, worst ratio {np.max(err[bad] / np.maximum(bound[bad], 1e-300))}"


def assert_rows_match(C, ref: oracle.Product, eps: float):
    """Compare only the rows the oracle computed (ref.rows)."""
    rowptr, colidx, val = to_host(C)
    for t, i in enumerate(ref.rows):
        a, b = rowptr[i], rowptr[i + 1]
        ra, rb = ref.rowptr[t], ref.rowptr[t + 1]
        assert b - a == rb - ra, f"row {i}: {b - a} entries, oracle {rb - ra}"
        assert np.array_equal(colidx[a:b], ref.colidx[ra:rb]), f"row {i}: columns differ"
        err = np.abs(val[a:b] - ref.val[ra:rb])
        assert np.all(err <= TOL_FACTOR * eps * ref.absval[ra:rb]), f"row {i}: values outside the bound"


def assert_csr_valid(C, ncols: int):
    rowptr, colidx, _ = to_host(C)
    nnz = int(rowptr[-1])
    assert rowptr[0] == 0 and np.all(np.diff(rowptr) >= 0)
    c = colidx[:nnz].astype(np.int64)
    assert np.all((c >= 0) & (c < ncols))
    rows = np.repeat(np.arange(rowptr.shape[0] - 1), np.diff(rowptr))
    same = rows[1:] == rows[:-1]
    assert np.all(c[1:][same] > c[:-1][same]), "columns not strictly ascending inside a row"
