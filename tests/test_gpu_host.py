"""pb_spgemm_host: the product from and to host memory, copies overlapped with the kernels.

Results must match the oracle exactly as the device entry points do (structure
bit-exact, values within 64 * eps * sum |a b|), with and without row panels
(each panel's rows of C are copied back while the next panel computes).
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


def host_out(pb, m, cap, vdt=torch.float64):
    return pb.CsrMatrix(m, 0, torch.empty(m + 1, dtype=torch.int64).pin_memory(),
                        torch.empty(max(cap, 1), dtype=torch.int32).pin_memory(),
                        torch.empty(max(cap, 1), dtype=vdt).pin_memory())


def run_host(pb, A, B, dtype=0, vdt=None, cap=None, **cfg):
    hA, hB = pb.host_tensors(A, vdt), pb.host_tensors(B, vdt)
    cap = oracle.flop(A, B) if cap is None else cap
    C = host_out(pb, A.nrows, cap, vdt or torch.float64)
    nnz, st = pb.spgemm_host(hA, hB, C, dtype=dtype, config=pb.make_config(**cfg) if cfg else None)
    return C, nnz, st


def trimmed(C, nnz, ncols):
    return type(C)(C.nrows, ncols, C.rowptr, C.colidx[:nnz], C.val[:nnz])


@pytest.mark.parametrize("n,d,panels", [(4096, 4, 0), (1 << 17, 8, 0), (1 << 17, 8, 4), (1 << 17, 8, 1)])
def test_host_product_matches_oracle(pb, n, d, panels):
    A, B = synth.er(n, d, seed=n + d)
    C, nnz, st = run_host(pb, A, B, min_panels=panels) if panels else run_host(pb, A, B)
    assert st == 0
    ref = oracle.spgemm(A, B)
    assert nnz == ref.nnz
    assert_matches(trimmed(C, nnz, B.ncols), ref, EPS["f64"])


def test_host_product_rmat_oversize_rows_in_panels(pb):
    A, B = synth.rmat(13, 8, seed=31)
    C, nnz, st = run_host(pb, A, B, min_panels=3)
    assert st == 0
    assert_matches(trimmed(C, nnz, B.ncols), oracle.spgemm(A, B), EPS["f64"])


def test_host_product_rmat_fp32_tuples_in_panels(pb):
    """FP32 tuples with hub rows (dense tiles keep their FP64 sums in the main tuple
    buffer) and row panels copied back one by one."""
    A, B = synth.rmat(13, 8, seed=32)
    assert int(np.max(oracle.row_flop(A, B))) > 4096
    C, nnz, st = run_host(pb, A, B, dtype=2, min_panels=3)
    assert st == 0 and C.val.dtype == torch.float64
    assert_matches(trimmed(C, nnz, B.ncols), oracle.spgemm(A, B), EPS["f32"])


def test_host_product_fp32(pb):
    A, B = synth.er(20000, 6, seed=5)
    A32 = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32))
    B32 = synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))
    C, nnz, st = run_host(pb, A32, B32, dtype=1, vdt=torch.float32)
    assert st == 0
    assert_matches(trimmed(C, nnz, B.ncols), oracle.spgemm(A32, B32), EPS["f32"])


def test_host_product_too_small_c_reports_overflow(pb):
    A, B = synth.er(30000, 6, seed=6)
    ref = oracle.spgemm(A, B)
    C, nnz, st = run_host(pb, A, B, cap=ref.nnz - 10)
    assert st == 5 and nnz == ref.nnz      # PB_ERR_OVERFLOW; the true size is reported


def test_host_product_empty(pb):
    A = synth.CSC(0, 5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.CSR(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C, nnz, st = run_host(pb, A, B, cap=1)
    assert st == 0 and nnz == 0 and int(C.rowptr[0]) == 0
