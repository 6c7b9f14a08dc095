"""pb_validate_operands: device checks of the preconditions the compute calls trust.

Each invalid operand is built on the host (arrays of the declared sizes, so the
checks read nothing outside them) and must be reported with the array named.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import binding
    binding.load_library()
    return binding


def dev(pb, A, B):
    return pb.csc_to_device(A), pb.csr_to_device(B)


def test_valid_operands_pass(pb):
    for A, B in (synth.er(5000, 6, seed=1), synth.rmat(10, 4, seed=2), synth.identity(100)):
        st, msg = pb.validate(*dev(pb, A, B))
        assert st == 0 and msg == ""


def broken(A, B, what):
    A = synth.CSC(A.nrows, A.ncols, A.colptr.copy(), A.rowidx.copy(), A.val)
    B = synth.CSR(B.nrows, B.ncols, B.rowptr.copy(), B.colidx.copy(), B.val)
    if what == "colptr_start":
        A.colptr[0] = 1
    elif what == "colptr_decreasing":
        A.colptr[6] = A.colptr[5] - 1       # column 5 holds d > 0 entries, so this goes backwards
    elif what == "colptr_end":
        A.colptr[-1] -= 1
    elif what == "rowidx_negative":
        A.rowidx[7] = -3
    elif what == "rowidx_high":
        A.rowidx[-1] = A.nrows
    elif what == "rowptr_end":
        B.rowptr[-1] = B.rowptr[-1] + 5
    elif what == "colidx_high":
        B.colidx[3] = B.ncols + 100
    return A, B


@pytest.mark.parametrize("what,needle", [("colptr_start", "A.colptr"), ("colptr_decreasing", "A.colptr"),
                                         ("colptr_end", "A.colptr"), ("rowidx_negative", "A.rowidx"),
                                         ("rowidx_high", "A.rowidx"), ("rowptr_end", "B.rowptr"),
                                         ("colidx_high", "B.colidx")])
def test_invalid_operands_reported(pb, what, needle):
    A, B = broken(*synth.er(3000, 5, seed=3), what)
    st, msg = pb.validate(*dev(pb, A, B))
    assert st == 1, what          # PB_ERR_INVALID_ARG
    assert needle in msg, msg
