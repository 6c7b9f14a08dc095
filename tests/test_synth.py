"""Seeded input generators: the properties the workload readings rely on.

The generators hold none of the method's arithmetic; these checks make sure the
inputs are what the readings say they are: ER with exactly d distinct rows per
column (Sec. II-A), R-MAT with the (a, b, c, d) quadrant split and duplicates
removed (Sec. IV-C), column-stochastic Markov matrices, the 7-point Poisson
matrix and its 2x2x2 aggregation, and the batch shape distribution.
"""
import numpy as np

import synth


def entry_set(r, c, v):
    order = np.lexsort((c, r))
    return r[order], c[order], v[order]


def test_er_exactly_d_distinct_rows_per_column():
    n, d = 5000, 8
    A, B = synth.er(n, d, seed=3)
    assert np.all(np.diff(A.colptr) == d)
    rows = A.rowidx.reshape(n, d).astype(np.int64)
    srt = np.sort(rows, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0) and rows.min() >= 0 and rows.max() < n
    assert np.all(np.abs(A.val) < 1.0)
    # the CSR copy holds the same entries
    ra, ca, va = entry_set(*synth.csc_entries(A))
    rb, cb, vb = entry_set(*synth.csr_entries(B))
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb) and np.array_equal(va, vb)
    # seeded
    A2, _ = synth.er(n, d, seed=3)
    A3, _ = synth.er(n, d, seed=4)
    assert np.array_equal(A.rowidx, A2.rowidx) and not np.array_equal(A.rowidx, A3.rowidx)


def test_er_shuffle_within_keeps_the_entries():
    A, _ = synth.er(3000, 6, seed=5)
    S, _ = synth.er(3000, 6, seed=5, shuffle_within=True)
    assert not np.array_equal(A.rowidx, S.rowidx)
    a = entry_set(*synth.csc_entries(A))
    s = entry_set(*synth.csc_entries(S))
    assert all(np.array_equal(x, y) for x, y in zip(a, s))


def test_rmat_quadrants_and_no_duplicates():
    # sparse enough that deduplication removes few edges: the top bits keep the
    # split of the recursive quadrant choice, P(top row bit 0) = a + b and
    # P(top column bit 0) = a + c
    scale, a, b, c = 16, 0.57, 0.19, 0.19
    n, row, col, _ = synth.rmat_coo(scale, 1, a, b, c, seed=7)
    assert n == 1 << scale
    key = row * n + col
    assert np.unique(key).size == key.size
    assert row.min() >= 0 and row.max() < n and col.min() >= 0 and col.max() < n
    assert key.size > 0.95 * n
    top = 1 << (scale - 1)
    assert abs(np.mean(row < top) - (a + b)) < 0.01
    assert abs(np.mean(col < top) - (a + c)) < 0.01
    assert abs(np.mean((row < top) & (col < top)) - a) < 0.01


def test_rmat_hub_rows_are_skewed():
    A, B = synth.rmat(12, 8, seed=2)
    deg = np.diff(B.rowptr)
    assert deg.max() > 20 * deg.mean()       # power-law hubs
    assert int(np.argmax(deg)) == 0          # no vertex permutation: the hub is row 0


def test_column_stochastic_columns_sum_to_one():
    Ac, _ = synth.rmat(10, 8, seed=2)
    M, Mr = synth.column_stochastic(Ac)
    r, c, v = synth.csc_entries(M)
    assert v.dtype == np.float32 and np.all(v > 0)
    sums = np.bincount(c, weights=v.astype(np.float64), minlength=M.ncols)
    assert np.allclose(sums, 1.0, atol=1e-5)
    assert np.all(np.isin(np.arange(M.ncols), c[r == c]))   # every vertex has a self loop
    rr, cr, vr = synth.csr_entries(Mr)
    assert all(np.array_equal(x, y) for x, y in zip(entry_set(r, c, v), entry_set(rr, cr, vr)))


def test_poisson7_and_aggregation():
    N = 4
    A = synth.poisson7(N)
    r, c, v = synth.csr_entries(A)
    assert np.all(v[r == c] == 6.0) and np.all(v[r != c] == -1.0)
    dense = np.zeros((N ** 3, N ** 3))
    dense[r, c] = v
    assert np.array_equal(dense, dense.T)
    # a corner has 3 neighbours, an interior point 6
    assert dense[0].sum() == 3.0 and dense[1 + N + N * N].sum() == 0.0
    P = synth.aggregation_prolongator(N)
    pr, pc, pv = synth.csr_entries(P)
    assert np.all(np.diff(P.rowptr) == 1) and np.all(pv == 1.0)
    assert np.all(np.bincount(pc, minlength=(N // 2) ** 3) == 8)


def test_batch_shapes_log_uniform():
    shapes = synth.batch_er_shapes(1024, seed=3)
    n = np.array([s[0] for s in shapes])
    d = np.array([s[1] for s in shapes])
    assert len(shapes) == 1024
    assert n.min() >= 512 and n.max() <= 65536 and d.min() >= 2 and d.max() <= 16
    assert set(np.unique(d).tolist()) == set(range(2, 17))
    # log-uniform: log n is uniform between log 512 and log 65536
    u = (np.log(n) - np.log(512)) / (np.log(65536) - np.log(512))
    assert abs(np.mean(u) - 0.5) < 0.03 and abs(np.mean(u < 0.25) - 0.25) < 0.04
