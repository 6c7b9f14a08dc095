"""Pins of the CPU oracle against facts outside itself (no GPU needed).

Each test ties the oracle to the mathematics or to a number printed in the
paper, so that a dropped term, a wrong sign, a wrong index or a transposed
operand in the oracle fails at least one of them:
  * dense brute force on tiny rectangular inputs (values and structure),
  * identity and permutation products (bit-exact),
  * ER closed forms: flop = n*d^2 exactly, nnz(C) <= flop, E[nnz(C)] band,
  * AMG closed form: P^T (A P) = 4 x coarse 7-point operator, bit-exact,
  * Markov matrices: the square of a column-stochastic matrix is column-stochastic,
  * per-row flop and the expand multiset against brute-force enumeration.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

EPS64 = 2.0 ** -53


def dense_of(csr: synth.CSR) -> np.ndarray:
    d = np.zeros((csr.nrows, csr.ncols))
    r, c, v = synth.csr_entries(csr)
    np.add.at(d, (r, c), v.astype(np.float64))
    return d


def pattern_of(csr: synth.CSR) -> np.ndarray:
    p = np.zeros((csr.nrows, csr.ncols), dtype=np.int64)
    r, c, _ = synth.csr_entries(csr)
    p[r, c] = 1
    return p


def to_dense(prod: oracle.Product, m: int, n: int):
    d = np.zeros((m, n))
    pat = np.zeros((m, n), dtype=np.int64)
    rows = np.repeat(prod.rows, np.diff(prod.rowptr))
    d[rows, prod.colidx] = prod.val
    pat[rows, prod.colidx] = 1
    return d, pat


@pytest.mark.parametrize("seed", range(6))
def test_dense_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    m, k, n = (int(x) for x in rng.integers(1, 40, 3))
    dens = float(rng.uniform(0.02, 0.5))
    A, _ = synth.random_sparse(m, k, dens, seed=seed)
    _, B = synth.random_sparse(k, n, dens, seed=1000 + seed)
    C = oracle.spgemm(A, B)
    Ad, Bd = dense_of(synth.csc_to_csr(A)), dense_of(B)
    Cd, Cpat = to_dense(C, m, n)
    # structure: boolean product of the stored patterns
    ref_pat = (pattern_of(synth.csc_to_csr(A)) @ pattern_of(B)) > 0
    assert np.array_equal(Cpat.astype(bool), ref_pat)
    # values within the rounding bound of an n-term sum
    ref = Ad @ Bd
    bound = np.abs(Ad) @ np.abs(Bd)
    assert np.all(np.abs(Cd - ref) <= 64 * EPS64 * bound + 1e-300)
    absd = np.zeros((m, n))
    rows = np.repeat(C.rows, np.diff(C.rowptr))
    absd[rows, C.colidx] = C.absval
    assert np.allclose(absd, bound, rtol=1e-12, atol=0)
    # each row's columns strictly ascending
    for t in range(m):
        seg = C.colidx[C.rowptr[t]:C.rowptr[t + 1]]
        assert np.all(np.diff(seg) > 0)


def test_zero_values_keep_structure():
    """No dropping (Sec. III-E merges equal keys without a value test): with every value
    zero, C's structure is still the boolean product of the stored patterns, and every
    value and magnitude sum is exactly zero."""
    A, B = synth.rmat(7, 8, seed=3)
    Az = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, np.zeros_like(A.val))
    Bz = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, np.zeros_like(B.val))
    C = oracle.spgemm(Az, Bz)
    _, Cpat = to_dense(C, A.nrows, B.ncols)
    ref_pat = (pattern_of(synth.csc_to_csr(Az)) @ pattern_of(Bz)) > 0
    assert ref_pat.any()
    assert np.array_equal(Cpat.astype(bool), ref_pat)
    assert not np.any(C.val) and not np.any(C.absval)


def test_rows_subset_matches_full():
    A, B = synth.er(300, 5, seed=7)
    full = oracle.spgemm(A, B)
    rows = np.array([299, 0, 17, 150, 17], dtype=np.int64)
    sub = oracle.spgemm(A, B, rows)
    for t, i in enumerate(rows):
        a = slice(full.rowptr[i], full.rowptr[i + 1])
        b = slice(sub.rowptr[t], sub.rowptr[t + 1])
        assert np.array_equal(full.colidx[a], sub.colidx[b])
        assert np.array_equal(full.val[a], sub.val[b])


def test_identity_products_bit_exact():
    A, B = synth.er(500, 6, seed=3)
    Ic, Ir = synth.identity(500)
    IB = oracle.spgemm(Ic, B)                    # I * B = B
    ref = synth.coo_to_csr(500, 500, *synth.csr_entries(B))
    # CSR of B sorted by column inside each row
    r, c, v = synth.csr_entries(B)
    order = np.lexsort((c, r))
    assert np.array_equal(IB.rowptr, ref.rowptr.astype(np.int64))
    assert np.array_equal(IB.colidx, c[order].astype(np.int32))
    assert np.array_equal(IB.val, v[order])
    AI = oracle.spgemm(A, Ir)                    # A * I = A
    ra, ca, va = synth.csc_entries(A)
    order = np.lexsort((ca, ra))
    assert np.array_equal(AI.colidx, ca[order].astype(np.int32))
    assert np.array_equal(AI.val, va[order])


def test_permutation_product_bit_exact():
    _, B = synth.er(400, 4, seed=5)
    Pc, _, perm = synth.permutation(400, seed=9)
    PB = oracle.spgemm(Pc, B)                    # row i of P*B is row perm[i] of B
    r, c, v = synth.csr_entries(B)
    for i in range(400):
        src = perm[i]
        seg = slice(B.rowptr[src], B.rowptr[src + 1])
        o = np.argsort(B.colidx[seg], kind="stable")
        got = slice(PB.rowptr[i], PB.rowptr[i + 1])
        assert np.array_equal(PB.colidx[got], B.colidx[seg][o])
        assert np.array_equal(PB.val[got], B.val[seg][o])


@pytest.mark.parametrize("n,d", [(4096, 4), (2048, 8), (1000, 2), (777, 16)])
def test_er_closed_forms(n, d):
    A, B = synth.er(n, d, seed=n + d)
    f = oracle.flop(A, B)
    assert f == n * d * d                        # exactly d per column and per row of B=A
    rf = oracle.row_flop(A, B)
    assert int(rf.sum()) == f
    C = oracle.spgemm(A, B)
    assert C.nnz <= f                            # cf >= 1 (Sec. II-A)
    expected = n * n * (1.0 - (1.0 - d / n) ** d)
    assert abs(C.nnz - expected) <= 6 * np.sqrt(expected) + 0.01 * expected


def test_er_4096_nnz_band():
    A, B = synth.er(4096, 4, seed=0)
    C = oracle.spgemm(A, B)
    # n^2 (1 - (1 - d/n)^d) = 65,408.3 for n = 4096, d = 4
    assert 64_000 < C.nnz <= 65_536


@pytest.mark.parametrize("N", [2, 4, 6])
def test_amg_galerkin_closed_form(N):
    A = synth.poisson7(N)                        # symmetric: CSR arrays are also CSC arrays
    A_csc = synth.CSC(A.nrows, A.ncols, A.rowptr, A.colidx, A.val)
    P = synth.aggregation_prolongator(N)
    AP = oracle.spgemm(A_csc, P)
    AP_csr = synth.CSR(A.nrows, P.ncols, AP.rowptr.astype(np.int32), AP.colidx, AP.val)
    PT = synth.transpose_csr_as_csc(P)           # CSC of P^T is the CSR of P
    G = oracle.spgemm(PT, AP_csr)
    M = N // 2
    Gd, Gpat = to_dense(G, M ** 3, M ** 3)
    ref = np.zeros((M ** 3, M ** 3))
    for I in range(M ** 3):
        x, y, z = I % M, (I // M) % M, I // (M * M)
        ref[I, I] = 24.0
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            xx, yy, zz = x + dx, y + dy, z + dz
            if 0 <= xx < M and 0 <= yy < M and 0 <= zz < M:
                ref[I, xx + M * yy + M * M * zz] = -4.0
    assert np.array_equal(Gd, ref)               # integers: bit-exact in FP64
    assert np.array_equal(Gpat.astype(bool), ref != 0)


def test_markov_square_column_stochastic():
    Ac, _ = synth.rmat(10, 8, seed=4)
    Mc, Mr = synth.column_stochastic(Ac, dtype=np.float64)
    C = oracle.spgemm(Mc, Mr)
    assert np.all(np.diff(Mc.colptr) > 0)         # self loops: no empty column
    colsum = np.bincount(C.colidx, weights=C.val, minlength=Mc.ncols)
    # 1^T (M M) = (1^T M) M = 1^T M = 1^T
    assert np.allclose(colsum, 1.0, rtol=0, atol=1e-12)


def test_row_flop_and_expand_bruteforce():
    rng = np.random.default_rng(11)
    A, _ = synth.random_sparse(23, 17, 0.2, seed=21)
    _, B = synth.random_sparse(17, 29, 0.25, seed=22)
    Apat = pattern_of(synth.csc_to_csr(A))
    nnzB_rows = np.diff(B.rowptr)
    assert np.array_equal(oracle.row_flop(A, B), Apat @ nnzB_rows)
    assert oracle.flop(A, B) == int((Apat @ nnzB_rows).sum())
    row, col, val = oracle.expand(A, B)
    # brute-force enumeration of the same tuples
    Ad, Bd = dense_of(synth.csc_to_csr(A)), dense_of(B)
    ref = sorted((i, j, Ad[i, kk] * Bd[kk, j]) for kk in range(17)
                 for i in range(23) if Apat[i, kk] for j in range(29) if pattern_of(B)[kk, j])
    got = sorted(zip(row.tolist(), col.tolist(), val.tolist()))
    assert got == ref
    # summing the tuples by (row, col) reproduces the dense product
    S = np.zeros((23, 29))
    np.add.at(S, (row, col), val)
    assert np.allclose(S, Ad @ Bd, rtol=0, atol=1e-14)
    del rng


def test_unsorted_columns_same_result():
    A1, B1 = synth.er(700, 7, seed=13)
    A2, _ = synth.er(700, 7, seed=13, shuffle_within=True)
    C1 = oracle.spgemm(A1, B1)
    C2 = oracle.spgemm(A2, B1)
    assert np.array_equal(C1.rowptr, C2.rowptr) and np.array_equal(C1.colidx, C2.colidx)
    assert np.allclose(C1.val, C2.val, rtol=0, atol=1e-15)


def test_empty_and_degenerate():
    # A with an empty column and B with an empty row: no tuples from that k
    A = synth.CSC(3, 3, np.array([0, 2, 2, 3], np.int32), np.array([0, 2, 1], np.int32),
                  np.array([1.0, 2.0, 3.0]))
    B = synth.CSR(3, 2, np.array([0, 1, 2, 2], np.int32), np.array([1, 0], np.int32),
                  np.array([5.0, 7.0]))
    assert oracle.flop(A, B) == 2 * 1 + 0 * 1 + 1 * 0
    C = oracle.spgemm(A, B)
    assert C.rowptr.tolist() == [0, 1, 1, 2]
    assert C.colidx.tolist() == [1, 1]
    assert C.val.tolist() == [5.0, 10.0]
    Z = synth.CSC(4, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    Zb = synth.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.flop(Z, Zb) == 0
    assert oracle.spgemm(Z, Zb).nnz == 0


def test_shape_mismatch_rejected():
    A, _ = synth.er(10, 2, seed=1)
    _, B = synth.er(11, 2, seed=1)
    with pytest.raises(ValueError):
        oracle.spgemm(A, B)


def test_paper_constants_pin_byte_model():
    from paper_2002_11302_gb300 import model
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    assert model.ai_upper(g["ai_upper"]["cf"], g["ai_upper"]["b"]) == g["ai_upper"]["ai"]
    pk = g["peak_skylake"]
    assert abs(model.peak_flops(pk["beta_gbs"], pk["ai"]) - pk["gflops"]) <= 0.005   # printed to 2 decimals
    lo = g["ai_outer_lower"]
    assert model.ai_outer_lower(lo["cf"], lo["b"]) == lo["ai"]
    for beta, mflops in g["pb_lower_bound_mflops"]["cases"]:
        assert model.peak_flops(beta, model.ai_outer_lower(1.0, 16)) * 1000 == pytest.approx(mflops)
    ex = g["in_cache_example"]
    A, B = synth.er(ex["n"] // 64, ex["d"], seed=0)     # closed form scales with n: flop = n d^2
    assert oracle.flop(A, B) * 64 == ex["tuples"]
    assert ex["tuples"] // ex["nbins"] == ex["tuples_per_bin"]
    assert ex["tuples_per_bin"] * (ex["key_bytes"] + ex["val_bytes"]) == ex["bin_bytes"]
    kb = g["key_bits_example"]
    assert model.key_bits(kb["n"], kb["n"] // kb["nbins"]) == (kb["row_bits"], kb["col_bits"])
