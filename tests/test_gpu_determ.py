"""Deterministic mode (pb_config.deterministic) through the C ABI.

Runs are placed at positions fixed in the plan (CSC order of A inside every
bin) and equal keys merge in position order, so every C(i,j) is summed over
ascending k.  The CPU oracle also accumulates each row over ascending k
(starting from zero), and both round every FP64 product once, so in FP64 the
two results are equal element for element -- a stronger check than the
tolerance used for the atomic-cursor path.  Repeated runs must be bitwise
identical in every dtype.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EPS, assert_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import binding
    binding.load_library()
    return binding


def run_det(pb, A, B, dtype=0, vdt=None, **cfg):
    Ad, Bd = pb.csc_to_device(A, val_dtype=vdt), pb.csr_to_device(B, val_dtype=vdt)
    C = pb.spgemm(Ad, Bd, dtype=dtype, config=pb.make_config(deterministic=True, **cfg))
    return C.rowptr.cpu().numpy(), C.colidx.cpu().numpy(), C.val.cpu().numpy()


def assert_oracle_exact(got, ref):
    rowptr, colidx, val = got
    assert np.array_equal(rowptr, ref.rowptr), "row pointers differ"
    assert np.array_equal(colidx, ref.colidx), "column indices differ"
    bad = np.nonzero(val != ref.val)[0]
    assert bad.size == 0, f"{bad.size} values differ from the oracle's ascending-k sums"


@pytest.mark.parametrize("n,d,cap", [(20000, 8, 4096), (3000, 16, 2048), (50000, 3, 8192), (1 << 15, 6, 4096)])
def test_er_fp64_equals_oracle_exactly(pb, n, d, cap):
    A, B = synth.er(n, d, seed=n + d, shuffle_within=True)
    assert_oracle_exact(run_det(pb, A, B, bin_capacity=cap), oracle.spgemm(A, B))


@pytest.mark.parametrize("seed", range(4))
def test_rectangular_fp64_equals_oracle_exactly(pb, seed):
    rng = np.random.default_rng(seed)
    m, k, n = (int(x) for x in rng.integers(1, 400, 3))
    A, _ = synth.random_sparse(m, k, 0.08, seed=30 + seed)
    _, B = synth.random_sparse(k, n, 0.08, seed=40 + seed)
    assert_oracle_exact(run_det(pb, A, B), oracle.spgemm(A, B))


def test_rmat_oversize_rows_fp64_equals_oracle_exactly(pb):
    A, B = synth.rmat(12, 8, seed=9)          # hub rows above the bin capacity: global-memory sort
    assert int(np.max(oracle.row_flop(A, B))) > 4096
    assert_oracle_exact(run_det(pb, A, B), oracle.spgemm(A, B))


def test_row_panels_fp64_equals_oracle_exactly(pb):
    A, B = synth.rmat(12, 8, seed=10)
    assert_oracle_exact(run_det(pb, A, B, max_tuple_bytes=60000 * 12), oracle.spgemm(A, B))


def test_repeated_runs_bitwise_identical(pb):
    A, B = synth.rmat(11, 8, seed=11)
    for dtype, vdt, eps in ((0, None, EPS["f64"]), (1, torch.float32, EPS["f32"]), (2, None, EPS["f32"])):
        if dtype == 1:
            A1 = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32))
            B1 = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))
        else:
            A1, B1 = A, B
        first = run_det(pb, A1, B1, dtype=dtype, vdt=vdt)
        for _ in range(3):
            again = run_det(pb, A1, B1, dtype=dtype, vdt=vdt)
            assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])
            assert first[2].tobytes() == again[2].tobytes(), f"dtype {dtype}: values differ between runs"
        ref = oracle.spgemm(A1, B1)
        C = pb.CsrMatrix(A.nrows, B.ncols, torch.from_numpy(first[0]), torch.from_numpy(first[1]),
                         torch.from_numpy(first[2]))
        assert_matches(C, ref, eps)


def test_plan_reuse_with_new_values_stays_exact(pb):
    """A deterministic plan reused for new values (same structure) still reproduces the oracle."""
    A, B = synth.er(8000, 7, seed=12)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    plan = pb.symbolic(Ad, Bd, config=pb.make_config(deterministic=True))
    C = pb.alloc_output(plan)
    ws = plan.workspace()
    rng = np.random.default_rng(5)
    for _ in range(2):
        av, bv = rng.uniform(-1, 1, A.nnz), rng.uniform(-1, 1, B.nnz)
        Ad.val.copy_(torch.from_numpy(av))
        Bd.val.copy_(torch.from_numpy(bv))
        pb.numeric(plan, Ad, Bd, C, ws)
        assert plan.status() == 0
        nnz = int(C.rowptr[-1].item())
        got = (C.rowptr.cpu().numpy(), C.colidx[:nnz].cpu().numpy(), C.val[:nnz].cpu().numpy())
        ref = oracle.spgemm(synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, av),
                            synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, bv))
        assert_oracle_exact(got, ref)
