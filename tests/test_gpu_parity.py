"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Structure (row pointers, column indices) must match bit-exactly; values must be
within 64 * eps * sum_k |a_ik b_kj| per entry (eps = 2^-53 for FP64, 2^-24
when products are rounded to FP32).  Inputs are seeded synthetic matrices.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EPS, assert_csr_valid, assert_matches, assert_rows_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import binding
    binding.load_library()
    return binding


def run(pb, A, B, dtype=0, cap=0, rowptr64=True, vdt=None):
    Ad = pb.csc_to_device(A, val_dtype=vdt)
    Bd = pb.csr_to_device(B, val_dtype=vdt)
    cfg = pb.make_config(bin_capacity=cap) if cap else None
    return pb.spgemm(Ad, Bd, dtype=dtype, config=cfg, rowptr64=rowptr64)


@pytest.mark.parametrize("seed", range(8))
def test_tiny_random_rectangular(pb, seed):
    rng = np.random.default_rng(seed)
    m, k, n = (int(x) for x in rng.integers(1, 70, 3))
    dens = float(rng.uniform(0.01, 0.6))
    A, _ = synth.random_sparse(m, k, dens, seed=10 + seed)
    _, B = synth.random_sparse(k, n, dens, seed=20 + seed)
    C = run(pb, A, B)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


@pytest.mark.parametrize("cap", [2048, 4096, 8192])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_bins_with_many_equal_keys(pb, cap, dtype):
    """Rows of 40 x 8 tuples on only 8 columns: every (row, column) key repeats
    about 40 times, above the 32 tuples a bucket takes before a bin falls back to
    the in-bin radix sort.  FP64, FP32 and FP32 tuples (the 4-byte forms read the
    packed {key, value} pairs), at every bin capacity."""
    rng = np.random.default_rng(80 + cap + dtype)
    m, k, n = 300, 200, 8
    rows = np.repeat(np.arange(m), 40)
    cols = np.concatenate([rng.choice(k, 40, replace=False) for _ in range(m)])
    A = synth.coo_to_csc(m, k, rows, cols, rng.uniform(-1, 1, rows.size))
    Bd = rng.uniform(-1, 1, (k, n))
    r, c = np.nonzero(Bd)
    B = synth.coo_to_csr(k, n, r, c, Bd[r, c])
    vdt = None
    if dtype == 1:
        A = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32))
        B = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))
        vdt = torch.float32
    assert int(np.max(oracle.row_flop(A, B))) <= 2048
    C = run(pb, A, B, dtype=dtype, cap=cap, vdt=vdt)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"] if dtype == 0 else EPS["f32"])


def test_er_4096_d4(pb):
    A, B = synth.er(4096, 4, seed=0)
    C = run(pb, A, B)
    ref = oracle.spgemm(A, B)
    assert_matches(C, ref, EPS["f64"])
    assert ref.nnz <= oracle.flop(A, B)


@pytest.mark.parametrize("cap", [2048, 4096, 8192])
@pytest.mark.parametrize("n,d", [(20000, 8), (3000, 16), (50000, 2), (1 << 15, 5)])
def test_er_capacities(pb, n, d, cap):
    A, B = synth.er(n, d, seed=n + d, shuffle_within=True)
    C = run(pb, A, B, cap=cap)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_rmat_small_skewed(pb):
    A, B = synth.rmat(11, 4, seed=2)
    C = run(pb, A, B)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_oversize_rows_dense_tiles(pb):
    """Hub rows above the bin capacity are merged in dense column tiles: structure exact
    (including exact-zero sums: all-zero values keep every structural entry), FP64 and FP32."""
    A, B = synth.rmat(12, 8, seed=41)
    assert int(np.max(oracle.row_flop(A, B))) > 4096
    ref = oracle.spgemm(A, B)
    assert_matches(run(pb, A, B), ref, EPS["f64"])
    A32 = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32))
    B32 = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))
    assert_matches(run(pb, A32, B32, dtype=1, vdt=torch.float32), oracle.spgemm(A32, B32), EPS["f32"])
    Az = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, np.zeros_like(A.val))
    Bz = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, np.zeros_like(B.val))
    C = run(pb, Az, Bz)
    assert np.array_equal(C.rowptr.cpu().numpy(), ref.rowptr)
    assert np.array_equal(C.colidx.cpu().numpy(), ref.colidx)
    assert not np.any(C.val.cpu().numpy())


def test_oversize_rows_counting_run_then_exact_c(pb):
    A, B = synth.rmat(12, 8, seed=42)
    C, plan = pb.spgemm_exact(pb.csc_to_device(A), pb.csr_to_device(B))
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def _revalue(A, B, av, bv):
    return (synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, av),
            synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, bv))


@pytest.mark.parametrize("n", [1, 37, 256, 300, 1000])
@pytest.mark.parametrize("dtype", [0, 2])
def test_oversize_rows_narrow_b(pb, n, dtype):
    """Hub rows when B has few columns: tiles narrower than 4096 columns (one or two
    warp slabs of 256), and many duplicates per column; FP64 and FP32 tuples."""
    A, _ = synth.random_sparse(5, 6000, 0.8, seed=50 + n)
    _, B = synth.random_sparse(6000, n, min(1.0, 3.0 / n), seed=60 + n)
    assert int(np.max(oracle.row_flop(A, B))) > 4096
    assert_matches(run(pb, A, B, dtype=dtype), oracle.spgemm(A, B), EPS["f64"] if dtype == 0 else EPS["f32"])


def test_oversize_rows_integer_values_bit_exact(pb):
    """Small integer values: every partial sum is exact in FP64, so the oracle's
    sequential sums and the dense tiles' atomic sums (any order) agree bit for bit,
    exact cancellations included."""
    A, B = synth.rmat(12, 8, seed=43)
    rng = np.random.default_rng(43)
    A, B = _revalue(A, B, rng.integers(-3, 4, A.nnz).astype(np.float64),
                    rng.integers(-3, 4, B.nnz).astype(np.float64))
    assert int(np.max(oracle.row_flop(A, B))) > 4096
    ref = oracle.spgemm(A, B)
    assert np.any(ref.val == 0) and np.any(ref.absval[ref.val == 0] > 0), "no exact cancellation to check"
    assert_matches(run(pb, A, B), ref, 0.0)


@pytest.mark.parametrize("kind", ["wide", "subnormal", "huge"])
def test_oversize_rows_outside_exact_window(pb, kind):
    """Hub rows whose values span many binades, hold subnormals, or come near the
    overflow range stay within the bound."""
    A, B = synth.rmat(12, 8, seed=44)
    rng = np.random.default_rng(44)
    av, bv = A.val.copy(), B.val.copy()
    if kind == "wide":
        av[rng.random(A.nnz) < 0.1] *= 2.0 ** -80
    elif kind == "subnormal":
        pick = rng.random(B.nnz) < 0.02
        bv[pick] = 5e-324 * rng.integers(1, 1000, int(pick.sum()))
    else:
        av *= 1e150
        bv *= 1e150
    A, B = _revalue(A, B, av, bv)
    assert int(np.max(oracle.row_flop(A, B))) > 4096
    assert_matches(run(pb, A, B), oracle.spgemm(A, B), EPS["f64"])


def test_identity_and_permutation_bit_exact(pb):
    A, B = synth.er(5000, 6, seed=3)
    Ic, Ir = synth.identity(5000)
    C = run(pb, Ic, B)
    ref = oracle.spgemm(Ic, B)
    assert_matches(C, ref, 0.0)             # one product per entry, times 1.0: exact
    Pc, _, perm = synth.permutation(5000, seed=4)
    C = run(pb, Pc, B)
    assert_matches(C, oracle.spgemm(Pc, B), 0.0)
    C = run(pb, A, Ir)
    assert_matches(C, oracle.spgemm(A, Ir), 0.0)


def test_amg_galerkin_chain_bit_exact(pb):
    N = 8
    A = synth.poisson7(N)
    A_csc = synth.CSC(A.nrows, A.ncols, A.rowptr, A.colidx, A.val)
    P = synth.aggregation_prolongator(N)
    AP = run(pb, A_csc, P, rowptr64=False)
    ref_AP = oracle.spgemm(A_csc, P)
    assert_matches(AP, ref_AP, 0.0)          # integer values: exact
    PT = synth.transpose_csr_as_csc(P)
    APh = synth.CSR(A.nrows, P.ncols, AP.rowptr.cpu().numpy(), AP.colidx.cpu().numpy(), AP.val.cpu().numpy())
    G = run(pb, PT, APh)
    Gref = oracle.spgemm(PT, APh)
    assert_matches(G, Gref, 0.0)
    vals = G.val.cpu().numpy()
    assert set(np.unique(vals).tolist()) <= {24.0, -4.0}


def test_fp32_values(pb):
    A, B = synth.er(20000, 6, seed=8, dtype=np.float32)
    C = run(pb, A, B, dtype=pb.PB_F32)
    ref = oracle.spgemm(A, B)               # FP64 oracle on the same (widened) inputs
    assert C.val.dtype == torch.float32
    assert_matches(C, ref, EPS["f32"])


def test_fp32_tuples_fp64_merge(pb):
    A, B = synth.er(30000, 8, seed=9)
    C = run(pb, A, B, dtype=pb.PB_F64_F32TUPLE)
    assert C.val.dtype == torch.float64
    ref = oracle.spgemm(A, B)
    assert_matches(C, ref, EPS["f32"])


@pytest.mark.parametrize("panels", [False, True])
def test_fp32_tuples_oversize_rows_merge_in_fp64(pb, panels):
    """FP32 tuples on hub rows above the bin capacity (dense tiles; the FP64 sums are kept
    in the row's region of the main tuple buffer): structure exact, and every value of the
    heaviest rows is the sum of the FP32-rounded products within the FP64 bound of that
    sum, so the merge itself runs in FP64."""
    import scipy.sparse as sp
    A, B = synth.rmat(12, 8, seed=46)
    rf = oracle.row_flop(A, B)
    assert np.any((rf > 4096) & (rf % 2 == 1)), "want hub rows with an odd tuple count"
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    cfg = pb.make_config(max_tuple_bytes=300000 * 8) if panels else None
    plan = pb.symbolic(Ad, Bd, dtype=pb.PB_F64_F32TUPLE, config=cfg)
    assert (plan.npanels > 1) == panels
    C = pb.alloc_output(plan)
    pb.numeric(plan, Ad, Bd, C, plan.workspace())
    assert plan.status() == 0
    n = int(C.rowptr[-1].item())
    C = pb.CsrMatrix(C.nrows, C.ncols, C.rowptr, C.colidx[:n], C.val[:n])
    assert C.val.dtype == torch.float64
    assert_matches(C, oracle.spgemm(A, B), EPS["f32"])
    rowptr, colidx, val = C.rowptr.cpu().numpy(), C.colidx.cpu().numpy(), C.val.cpu().numpy()
    Ar = sp.csc_matrix((A.val, A.rowidx, A.colptr), shape=(A.nrows, A.ncols)).tocsr()
    for i in np.argsort(rf)[-6:]:
        ks, av = Ar.indices[Ar.indptr[i]:Ar.indptr[i + 1]], Ar.data[Ar.indptr[i]:Ar.indptr[i + 1]]
        cols = np.concatenate([B.colidx[B.rowptr[k]:B.rowptr[k + 1]] for k in ks])
        p32 = np.concatenate([(a * B.val[B.rowptr[k]:B.rowptr[k + 1]]).astype(np.float32) for k, a in zip(ks, av)])
        p32 = p32.astype(np.float64)
        want = np.bincount(cols, weights=p32, minlength=B.ncols)
        mag = np.bincount(cols, weights=np.abs(p32), minlength=B.ncols)
        a, b = rowptr[i], rowptr[i + 1]
        assert np.array_equal(colidx[a:b], np.unique(cols))
        err = np.abs(val[a:b] - want[colidx[a:b]])
        assert np.all(err <= 64 * EPS["f64"] * mag[colidx[a:b]]), f"row {i}: merge not within the FP64 bound"


def test_config_validation(pb):
    """Unsupported tunables are refused by the symbolic phase, not ignored."""
    A, B = synth.er(2000, 4, seed=13)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    for bad in (dict(bin_capacity=3000), dict(bin_capacity=1024), dict(sort_threads=256),
                dict(bin_capacity=8192, sort_threads=512), dict(expand_chunk=100)):
        with pytest.raises(pb.PBError) as e:
            pb.symbolic(Ad, Bd, config=pb.make_config(**bad))
        assert e.value.status == 1, bad  # PB_ERR_INVALID_ARG
    for cap in (2048, 4096, 8192):
        C = pb.spgemm(Ad, Bd, config=pb.make_config(bin_capacity=cap, sort_threads=cap // 8))
        assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_int32_rowptr_output(pb):
    A, B = synth.er(10000, 4, seed=12)
    C = run(pb, A, B, rowptr64=False)
    assert C.rowptr.dtype == torch.int32
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_degenerate_shapes(pb):
    # empty columns of A, empty rows of B, rows with no products, a single row
    A = synth.CSC(4, 3, np.array([0, 2, 2, 3], np.int32), np.array([0, 3, 1], np.int32), np.array([1.0, 2.0, 3.0]))
    B = synth.CSR(3, 5, np.array([0, 2, 3, 3], np.int32), np.array([4, 0, 2], np.int32), np.array([5.0, 7.0, 9.0]))
    C = run(pb, A, B)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])
    # no products at all (flop = 0)
    Z = synth.CSC(6, 3, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = run(pb, Z, B)
    assert C.rowptr.cpu().tolist() == [0] * 7
    # one row, one column
    A1 = synth.CSC(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    B1 = synth.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([-2.0]))
    C = run(pb, A1, B1)
    assert C.rowptr.cpu().tolist() == [0, 1] and C.val.cpu().tolist() == [-6.0]


def test_empty_rows_span_many_bins(pb):
    # a tall A whose rows are mostly empty: bins are cut at the in-bin row limit
    A = synth.er_csc(300, 3, seed=5, nrows=200000)
    _, B = synth.er(300, 7, seed=6)
    C = run(pb, A, B)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_symbolic_arrays_match_oracle(pb):
    A, B = synth.er(40000, 7, seed=21, shuffle_within=True)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd)
    F, R, bin_row, bin_off = (t.cpu().numpy() for t in plan.export())
    assert plan.flop == oracle.flop(A, B) == 40000 * 49
    la, lb = np.diff(A.colptr).astype(np.int64), np.diff(B.rowptr).astype(np.int64)
    assert np.array_equal(F, np.concatenate([[0], np.cumsum(la * lb)]))           # Alg. 3 prefix
    assert np.array_equal(np.diff(R), oracle.row_flop(A, B))                      # per-row flop
    # bins: consecutive row ranges covering all rows, each within the on-chip capacity
    assert bin_row[0] == 0 and bin_row[-1] == A.nrows and np.all(np.diff(bin_row) > 0)
    counts = R[bin_row[1:]] - R[bin_row[:-1]]
    assert counts.max() <= 4096
    assert np.array_equal(np.diff(bin_off), (counts + 3) // 4 * 4)


def test_expand_tuples_match_oracle_expansion(pb):
    A, B = synth.er(6000, 6, seed=31, shuffle_within=True)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd)
    ws = plan.workspace()
    ws, voff = pb.debug_expand(plan, Ad, Bd, ws)
    torch.cuda.synchronize()
    _, R, bin_row, bin_off = (t.cpu().numpy() for t in plan.export())
    wsh = ws.cpu().numpy()
    keys = wsh[: 4 * int(bin_off[-1])].view(np.uint32)
    vals = wsh[voff: voff + 8 * int(bin_off[-1])].view(np.float64)
    colbits = max(1, int(np.ceil(np.log2(max(B.ncols, 2)))))
    rows, cols, vs = [], [], []
    for b in range(plan.nbins):
        cnt = int(R[bin_row[b + 1]] - R[bin_row[b]])
        k = keys[bin_off[b]: bin_off[b] + cnt]
        r = bin_row[b] + (k >> colbits).astype(np.int64)
        assert np.all(r < bin_row[b + 1]), "tuple outside its bin's row range"
        rows.append(r)
        cols.append((k & ((1 << colbits) - 1)).astype(np.int64))
        vs.append(vals[bin_off[b]: bin_off[b] + cnt])
    got = np.lexsort((np.concatenate(vs), np.concatenate(cols), np.concatenate(rows)))
    er, ec, ev = oracle.expand(A, B)
    exp = np.lexsort((ev, ec, er))
    assert np.array_equal(np.concatenate(rows)[got], er[exp].astype(np.int64))
    assert np.array_equal(np.concatenate(cols)[got], ec[exp].astype(np.int64))
    assert np.array_equal(np.concatenate(vs)[got], ev[exp])       # one rounding each: bit-exact


@pytest.mark.parametrize("dtype", ["PB_F32", "PB_F64_F32TUPLE"])
def test_expand_packed_tuples_match_oracle_expansion(pb, dtype):
    """4-byte tuple values are written as packed {key, value bits} pairs; the
    expanded multiset matches the oracle's with each product rounded once to
    FP32 (PB_F32: FP32 inputs; PB_F64_F32TUPLE: the FP64 product rounded)."""
    A, B = synth.er(6000, 6, seed=32, shuffle_within=True)
    f32 = dtype == "PB_F32"
    if f32:
        A = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32))
        B = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))
    vdt = torch.float32 if f32 else torch.float64
    Ad, Bd = pb.csc_to_device(A, val_dtype=vdt), pb.csr_to_device(B, val_dtype=vdt)
    plan = pb.symbolic(Ad, Bd, dtype=getattr(pb, dtype))
    assert pb.debug_tuple_layout(plan) == 1
    ws = plan.workspace()
    ws, _ = pb.debug_expand(plan, Ad, Bd, ws)
    torch.cuda.synchronize()
    _, R, bin_row, bin_off = (t.cpu().numpy() for t in plan.export())
    pairs = ws.cpu().numpy()[: 8 * int(bin_off[-1])].view(np.uint32).reshape(-1, 2)
    colbits = max(1, int(np.ceil(np.log2(max(B.ncols, 2)))))
    rows, cols, vs = [], [], []
    for b in range(plan.nbins):
        cnt = int(R[bin_row[b + 1]] - R[bin_row[b]])
        k = pairs[bin_off[b]: bin_off[b] + cnt, 0]
        r = bin_row[b] + (k >> colbits).astype(np.int64)
        assert np.all(r < bin_row[b + 1]), "tuple outside its bin's row range"
        rows.append(r)
        cols.append((k & ((1 << colbits) - 1)).astype(np.int64))
        vs.append(pairs[bin_off[b]: bin_off[b] + cnt, 1].view(np.float32))
    got = np.lexsort((np.concatenate(vs), np.concatenate(cols), np.concatenate(rows)))
    er, ec, ev = oracle.expand(A, B)
    ev32 = ev.astype(np.float32)
    exp = np.lexsort((ev32, ec, er))
    assert np.array_equal(np.concatenate(rows)[got], er[exp].astype(np.int64))
    assert np.array_equal(np.concatenate(cols)[got], ec[exp].astype(np.int64))
    assert np.array_equal(np.concatenate(vs)[got], ev32[exp])     # one FP32 rounding of the product


def test_capacity_overflow_reported(pb):
    A, B = synth.er(5000, 4, seed=41)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd)
    C = pb.alloc_output(plan, cap=100)
    pb.numeric(plan, Ad, Bd, C, plan.workspace())
    assert plan.status() == 5                # PB_ERR_OVERFLOW, nothing written past cap


def test_workspace_too_small_rejected(pb):
    A, B = synth.er(5000, 4, seed=42)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd)
    C = pb.alloc_output(plan)
    ws = torch.empty(plan.workspace_bytes // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(pb.PBError) as ei:
        pb.numeric(plan, Ad, Bd, C, ws)
    assert ei.value.status == 10


def test_shape_mismatch_rejected(pb):
    A, _ = synth.er(100, 3, seed=1)
    _, B = synth.er(101, 3, seed=1)
    with pytest.raises(pb.PBError) as ei:
        pb.symbolic(pb.csc_to_device(A), pb.csr_to_device(B))
    assert ei.value.status == 2


def test_plan_reuse_with_new_values(pb):
    A, B = synth.er(8000, 5, seed=51)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd)
    ws = plan.workspace()
    for scale in (1.0, -3.5):
        Ad.val.copy_(torch.from_numpy(A.val * scale))
        C = pb.alloc_output(plan)
        pb.numeric(plan, Ad, Bd, C, ws)
        assert plan.status() == 0
        A2 = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val * scale)
        assert_matches(C, oracle.spgemm(A2, B), EPS["f64"])


@pytest.mark.slow
def test_er_full_size_all_rows(pb):
    """The bench workload (ER n=2^21, d=8, FP64) in the bench's launch
    configuration, every entry of C against the full oracle product."""
    n, d = 1 << 21, 8
    A, B = synth.er(n, d, seed=1)
    C = run(pb, A, B)
    assert_csr_valid(C, n)
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])
    assert int(C.rowptr[-1].item()) <= n * d * d


def test_er22_fp32_tuples_full_size(pb):
    """The mixed-precision configuration (ER n=2^22, d=8): FP64 inputs, products
    rounded to FP32 in the tuples, merged in FP64; every entry of C against the
    full FP64 oracle product with the FP32 rounding bound, structure exact."""
    n, d = 1 << 22, 8
    A, B = synth.er(n, d, seed=4)
    C = run(pb, A, B, dtype=pb.PB_F64_F32TUPLE)
    assert C.val.dtype == torch.float64
    assert_matches(C, oracle.spgemm(A, B), EPS["f32"])


@pytest.mark.parametrize("budget_tuples", [20000, 60000])
def test_row_panels_match_oracle(pb, budget_tuples):
    """Products whose tuples exceed the workspace budget run in several row panels."""
    A, B = synth.er(30000, 6, seed=81, shuffle_within=True)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    cfg = pb.make_config(max_tuple_bytes=budget_tuples * 12)
    plan = pb.symbolic(Ad, Bd, config=cfg)
    assert plan.npanels > 1
    C = pb.alloc_output(plan)
    pb.numeric(plan, Ad, Bd, C, plan.workspace())
    assert plan.status() == 0
    n = int(C.rowptr[-1].item())
    C = pb.CsrMatrix(C.nrows, C.ncols, C.rowptr, C.colidx[:n], C.val[:n])
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_row_panels_with_oversize_rows(pb):
    A, B = synth.rmat(12, 8, seed=82)
    cfg = pb.make_config(max_tuple_bytes=400000 * 12)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd, config=cfg)
    assert plan.npanels > 1
    C = pb.alloc_output(plan)
    pb.numeric(plan, Ad, Bd, C, plan.workspace())
    assert plan.status() == 0
    n = int(C.rowptr[-1].item())
    C = pb.CsrMatrix(C.nrows, C.ncols, C.rowptr, C.colidx[:n], C.val[:n])
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_counting_run_gives_exact_nnz(pb):
    A, B = synth.rmat(11, 8, seed=83)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd)
    nnz = torch.zeros(1, dtype=torch.int64, device="cuda")
    empty = pb.CsrMatrix(plan.m, plan.n, torch.empty(0, dtype=torch.int64, device="cuda"),
                         torch.empty(0, dtype=torch.int32, device="cuda"),
                         torch.empty(0, dtype=torch.float64, device="cuda"))
    pb.numeric_count(plan, Ad, Bd, plan.workspace(), nnz)
    assert plan.status() == 0
    assert int(nnz.item()) == oracle.spgemm(A, B).nnz
    del empty


def _rows_from_device(C, rows):
    """Row segments of a device CSR for the listed rows (copies only those)."""
    rp = C.rowptr.cpu().numpy().astype(np.int64)
    out = []
    for i in rows:
        a, b = int(rp[i]), int(rp[i + 1])
        out.append((C.colidx[a:b].cpu().numpy(), C.val[a:b].double().cpu().numpy()))
    return rp, out


@pytest.mark.slow
def test_rmat_scale20_full_size_sampled_rows(pb):
    """R-MAT scale 20, edge factor 16, (0.57, 0.19, 0.19, 0.05), C = A*A: 2.1e10 tuples,
    nnz(C) above 2^31, hub rows far above a bin's capacity.  Runs in row panels with
    C sized by a counting run; sampled rows (the heaviest included) match the oracle."""
    A, B = synth.rmat(20, 16, seed=2)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    cfg = pb.make_config(max_tuple_bytes=64 << 30)
    C, plan = pb.spgemm_exact(Ad, Bd, config=cfg)
    assert plan.npanels > 1
    assert plan.flop == oracle.flop(A, B)
    rf = oracle.row_flop(A, B)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([np.argsort(rf)[-20:], rng.choice(A.nrows, 200, replace=False), [0, A.nrows - 1]]))
    ref = oracle.spgemm(A, B, rows)
    rp, segs = _rows_from_device(C, rows)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == C.nnz
    for t, (cols, vals) in enumerate(segs):
        ra, rb = ref.rowptr[t], ref.rowptr[t + 1]
        assert np.array_equal(cols, ref.colidx[ra:rb]), f"row {rows[t]}: columns differ"
        assert np.all(np.abs(vals - ref.val[ra:rb]) <= 64 * EPS["f64"] * ref.absval[ra:rb])
