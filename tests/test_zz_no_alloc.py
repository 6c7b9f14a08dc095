"""pb_spgemm_noalloc: the product without any device allocation by the library.

Callers whose device memory is owned by their own memory manager, or that run
in loops or callbacks where entering an allocator is not allowed, cannot let
the library call cudaMalloc.  pb_spgemm_noalloc serves them from a fixed
scratch array inside the library.  These tests call it through the C ABI and
compare its result with the CPU oracle (structure exactly, values within
64 * eps * sum |a b| for the dtype's rounding) on two calls in a row: the array
keeps the previous call's contents, so the second call also checks that
nothing stale leaks into a result.  They cover FP64, FP32 and FP32 tuples,
inputs with rows above the on-chip bin capacity (R-MAT hub rows, merged by the
global radix sort), and int32 row pointers.

This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EPS, TOL_FACTOR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import binding
    binding.load_library()
    return binding


def _flop(A, B) -> int:
    return int((np.diff(A.colptr).astype(np.int64) * np.diff(B.rowptr).astype(np.int64)).sum())


def _run_noalloc(pb, A, B, dtype, rowptr64=True):
    vdt = torch.float32 if dtype == pb.PB_F32 else torch.float64
    Ad, Bd = pb.csc_to_device(A, val_dtype=vdt), pb.csr_to_device(B, val_dtype=vdt)
    cap = max(_flop(A, B), 1)
    C = pb.CsrMatrix(A.nrows, B.ncols,
                     torch.empty(A.nrows + 1, dtype=torch.int64 if rowptr64 else torch.int32, device="cuda"),
                     torch.empty(cap, dtype=torch.int32, device="cuda"), torch.empty(cap, dtype=vdt, device="cuda"))
    nnz = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = pb.spgemm_noalloc(Ad, Bd, C, dtype=dtype, nnz_out=nnz)
    assert status == 0, f"device status {status}"
    k = int(nnz.item())
    rowptr = C.rowptr.cpu().numpy().astype(np.int64)
    assert k == int(rowptr[-1])
    return rowptr, C.colidx[:k].cpu().numpy(), C.val[:k].double().cpu().numpy()


def _matches_oracle(got, ref, eps):
    assert np.array_equal(got[0], ref.rowptr), "row pointers differ from the oracle"
    assert np.array_equal(got[1], ref.colidx), "column indices differ from the oracle"
    err = np.abs(got[2] - ref.val)
    assert np.all(err <= TOL_FACTOR * eps * ref.absval), f"values outside the bound (max {err.max():.3e})"


CASES = [  # (name, inputs, dtype name, eps key)
    ("er_f64", lambda: synth.er(6000, 6, seed=71), "PB_F64", "f64"),
    ("rmat_hubs_f64", lambda: synth.rmat(11, 4, seed=72), "PB_F64", "f64"),
    ("rmat_hubs_f32", lambda: synth.rmat(11, 4, seed=73, dtype=np.float32), "PB_F32", "f32"),
    ("rmat_hubs_f32tuple", lambda: synth.rmat(11, 4, seed=74), "PB_F64_F32TUPLE", "f32"),
]


@pytest.mark.parametrize("name,make,dtype,eps", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_on_two_calls(pb, name, make, dtype, eps):
    A, B = make()
    ref = oracle.spgemm(A, B)
    if name.startswith("rmat"):  # the case must exercise rows above the on-chip capacity
        assert int(oracle.row_flop(A, B).max()) > 4096
    for _ in range(2):
        _matches_oracle(_run_noalloc(pb, A, B, getattr(pb, dtype)), ref, EPS[eps])


def test_noalloc_int32_row_pointers(pb):
    A, B = synth.er(5000, 5, seed=75)
    ref = oracle.spgemm(A, B)
    for _ in range(2):
        _matches_oracle(_run_noalloc(pb, A, B, pb.PB_F64, rowptr64=False), ref, EPS["f64"])


def test_noalloc_rejects_products_above_its_scratch(pb):
    from paper_2002_11302_gb300 import binding
    A, B = synth.er(1 << 17, 8, seed=73)   # about 8.4M tuples: more than the fixed scratch holds
    with pytest.raises(binding.PBError) as ei:
        _run_noalloc(pb, A, B, pb.PB_F64)
    assert ei.value.status == 10           # PB_ERR_WORKSPACE
