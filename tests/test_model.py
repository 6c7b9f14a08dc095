"""The roofline byte model (Tab. III with this build's element sizes), on CPU.

bytes_alg is the numerator of every beta*AI figure the bench reports, so its
phase split and its response to element sizes are pinned here.
"""
import pytest

from paper_2002_11302_gb300 import model


def test_er_2_21_numeric_bytes():
    # ER n = 2^21, d = 8: flop = n d^2 exactly, nnz(C) as measured on the oracle
    n, d = 1 << 21, 8
    nnz = n * d
    flop = n * d * d
    nnz_c = 134_215_938
    b = model.bytes_alg(n, n, nnz, nnz, flop, nnz_c)
    # expand: both operands once (4 B index + 8 B value) plus both pointer arrays,
    # flop tuples of 12 B out; sort: the tuples once; compress: C once
    assert b.expand == 2 * 4 * (n + 1) + 12 * 2 * nnz + 12 * flop
    assert b.sort == 12 * flop
    assert b.compress == 12 * nnz_c + 8 * (n + 1)
    assert b.total == pytest.approx(5.35e9, rel=0.005)
    assert b.numeric == b.total - b.symbolic


def test_fp32_tuples_save_eight_bytes_per_tuple():
    # 12-byte tuples (u32 key + f64) against 8-byte tuples (u32 key + f32): each tuple
    # is written once in expand and read once in sort
    args = (5000, 4000, 30000, 28000, 250000, 200000)
    b12 = model.bytes_alg(*args)
    b8 = model.bytes_alg(*args, tuple_bytes=8)
    assert b12.numeric - b8.numeric == 2 * 4 * 250000
    assert b12.symbolic == b8.symbolic and b12.compress == b8.compress


def test_phase_bytes_scale_with_their_own_sizes():
    base = dict(m=100, k=80, nnz_a=500, nnz_b=400, flop=4000, nnz_c=3000)
    b0 = model.bytes_alg(**base)
    b1 = model.bytes_alg(**dict(base, flop=8000))
    assert b1.expand - b0.expand == 12 * 4000 and b1.sort - b0.sort == 12 * 4000
    assert b1.compress == b0.compress and b1.symbolic == b0.symbolic
    b2 = model.bytes_alg(**dict(base, nnz_c=6000))
    assert b2.compress - b0.compress == 12 * 3000 and b2.expand == b0.expand


def test_gflops_counts_multiply_and_add():
    assert model.gflops_2x(134_217_728, 3.63e-3) == pytest.approx(73.95, abs=0.01)
