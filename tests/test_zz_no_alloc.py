"""pb_spgemm_noalloc: the product without any device allocation by the library.

Callers whose device memory is owned by their own memory manager, or that run
in loops or callbacks where entering an allocator is not allowed, cannot let
the library call cudaMalloc.  pb_spgemm_noalloc serves them from a fixed
scratch array inside the library.  These tests call it through the C ABI and
compare its result with the regular entry points (pb_spgemm_symbolic +
pb_spgemm_numeric) on two calls in a row, with the same tolerance as the other
parity tests; the array keeps the previous call's contents, so the second call
also checks that nothing stale leaks into a result.

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


def _run_noalloc(pb, A, B):
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    cap = max(_flop(A, B), 1)
    C = pb.CsrMatrix(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda"),
                     torch.empty(cap, dtype=torch.int32, device="cuda"),
                     torch.empty(cap, dtype=torch.float64, device="cuda"))
    nnz = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = pb.spgemm_noalloc(Ad, Bd, C, nnz_out=nnz)
    assert status == 0, f"device status {status}"
    k = int(nnz.item())
    assert k == int(C.rowptr[-1].item())
    return C.rowptr.cpu().numpy(), C.colidx[:k].cpu().numpy(), C.val[:k].cpu().numpy()


def _run_regular(pb, A, B):
    C = pb.spgemm(pb.csc_to_device(A), pb.csr_to_device(B))
    return C.rowptr.cpu().numpy(), C.colidx.cpu().numpy(), C.val.cpu().numpy()


def _same(got, ref, scale):
    assert np.array_equal(got[0], ref[0]), "row pointers differ"
    assert np.array_equal(got[1], ref[1]), "column indices differ"
    # both results lie within 64 eps sum|a b| of the exact product, hence of each other within twice that
    assert np.all(np.abs(got[2] - ref[2]) <= 2 * TOL_FACTOR * EPS["f64"] * scale)


def test_noalloc_matches_regular_entry_points_on_two_calls(pb):
    problems = [synth.er(6000, 6, seed=71), synth.rmat(11, 4, seed=72)]  # the second has oversize rows
    for A, B in problems:
        ref = _run_regular(pb, A, B)
        scale = oracle.spgemm(A, B).absval
        got = _run_noalloc(pb, A, B)
        _same(got, ref, scale)


def test_noalloc_repeated_call_same_result(pb):
    A, B = synth.er(4096, 4, seed=0)
    first = _run_noalloc(pb, A, B)
    second = _run_noalloc(pb, A, B)
    assert np.array_equal(first[0], second[0]) and np.array_equal(first[1], second[1])
    scale = oracle.spgemm(A, B).absval
    assert np.all(np.abs(first[2] - second[2]) <= 2 * TOL_FACTOR * EPS["f64"] * scale)


def test_noalloc_rejects_products_above_its_scratch(pb):
    from paper_2002_11302_gb300 import binding
    A, B = synth.er(1 << 17, 8, seed=73)   # about 8.4M tuples: more than the fixed scratch holds
    with pytest.raises(binding.PBError) as ei:
        _run_noalloc(pb, A, B)
    assert ei.value.status == 10           # PB_ERR_WORKSPACE
