"""Batched products (pb_spgemm_batch) against the CPU oracle, through the C ABI.

Every product of a batch must match the oracle as if it were computed alone:
structure bit-exact, values within 64 * eps * sum_k |a_ik b_kj|.  Batches mix
sizes, densities, rectangular shapes, empty products and all three sort
capacity levels, and rows above every capacity (R-MAT hub rows, dense rows);
two tests capture a batch into a CUDA graph and replay it after the operand
values change.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EPS, assert_csr_valid, assert_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import binding
    binding.load_library()
    return binding


def empty_csc(m, k):
    return synth.CSC(m, k, np.zeros(k + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))


def empty_csr(k, n):
    return synth.CSR(k, n, np.zeros(k + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))


def mixed_problems(seed=0):
    """Host (A, B) pairs of many shapes, including degenerate ones."""
    rng = np.random.default_rng(seed)
    probs = []
    for (n, d) in synth.batch_er_shapes(24, seed=seed, n_lo=64, n_hi=6000, d_lo=1, d_hi=16):
        probs.append(synth.er(n, d, seed=int(rng.integers(1 << 30)), shuffle_within=True))
    for _ in range(6):  # rectangular
        m, k, n = (int(x) for x in rng.integers(1, 300, 3))
        A, _ = synth.random_sparse(m, k, float(rng.uniform(0.01, 0.2)), seed=int(rng.integers(1 << 30)))
        _, B = synth.random_sparse(k, n, float(rng.uniform(0.01, 0.2)), seed=int(rng.integers(1 << 30)))
        probs.append((A, B))
    probs.append((empty_csc(0, 5), empty_csr(5, 7)))        # no rows
    probs.append((empty_csc(9, 0), empty_csr(0, 4)))        # inner dimension 0
    probs.append((empty_csc(6, 6), empty_csr(6, 6)))        # no entries
    probs.append(synth.identity(777))
    P = synth.permutation(500, seed=3)
    probs.append((P[0], P[1]))
    probs.append(synth.rmat(10, 4, seed=5))                 # skewed rows
    return probs


def run_batch(pb, probs, dtype=0, rowptr64=True, vdt=None, tuning=None, handle=None):
    handle = handle or pb.Handle()
    if tuning is not None:
        pb.set_tuning(tuning, handle)
    As = [pb.csc_to_device(A, val_dtype=vdt) for A, _ in probs]
    Bs = [pb.csr_to_device(B, val_dtype=vdt) for _, B in probs]
    bt = pb.Batch(As, Bs, dtype=dtype, handle=handle, rowptr64=rowptr64)
    bt.run()
    return bt


def check_all(bt, probs, eps):
    assert bt.status() == 0, f"device status {bt.status()}"
    for i, (A, B) in enumerate(probs):
        C = bt.result(i)
        ref = oracle.spgemm(A, B)
        assert C.nrows == A.nrows and C.ncols == B.ncols
        assert_matches(C, ref, eps)
        assert_csr_valid(C, B.ncols)


def test_batch_mixed_fp64(pb):
    probs = mixed_problems(0)
    bt = run_batch(pb, probs)
    for i, (A, B) in enumerate(probs):
        assert int(bt.flop[i]) == oracle.flop(A, B)
    check_all(bt, probs, EPS["f64"])


def test_batch_int32_rowptr(pb):
    probs = mixed_problems(1)[:12]
    check_all(run_batch(pb, probs, rowptr64=False), probs, EPS["f64"])


def test_batch_fp32_and_fp32_tuples(pb):
    probs = mixed_problems(2)[:16]
    probs32 = [(synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32)),
                synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))) for A, B in probs]
    check_all(run_batch(pb, probs32, dtype=1, vdt=torch.float32), probs32, EPS["f32"])
    check_all(run_batch(pb, probs, dtype=2), probs, EPS["f32"])


def all_classes(probs, cap, rmax=11, chunk=4096):
    """A tuning table that puts every class of these problems at one capacity."""
    out = {}
    for A, _ in probs:
        log2n = int(np.ceil(np.log2(max(A.nrows, 2))))
        d = int(np.floor(A.nnz / A.ncols + 0.5)) if A.ncols else 0   # round half up, as the library
        out[(log2n, d.bit_length())] = dict(log2n=log2n, dclass=d.bit_length(), bin_capacity=cap,
                                           rmax_log2=rmax, expand_chunk=chunk)
    return list(out.values())


@pytest.mark.parametrize("cap,rmax,chunk", [(2048, 11, 256), (8192, 4, 16384), (4096, 1, 1024)])
def test_batch_one_level(pb, cap, rmax, chunk):
    probs = mixed_problems(3)
    check_all(run_batch(pb, probs, tuning=all_classes(probs, cap, rmax, chunk)), probs, EPS["f64"])


def test_batch_three_levels_interleaved(pb):
    """Products of one batch spread over the 2048/4096/8192 sort launches."""
    probs = mixed_problems(4)
    table = all_classes(probs, 4096)
    caps = [2048, 4096, 8192]
    for j, e in enumerate(table):
        e["bin_capacity"] = caps[j % 3]
        e["expand_chunk"] = [512, 2048, 8192][(j // 3) % 3]
    check_all(run_batch(pb, probs, tuning=table), probs, EPS["f64"])


def test_batch_matches_single_product_path(pb):
    probs = mixed_problems(5)[:20]
    bt = run_batch(pb, probs)
    assert bt.status() == 0
    for i, (A, B) in enumerate(probs):
        if A.nrows == 0:
            continue
        single = pb.spgemm(pb.csc_to_device(A), pb.csr_to_device(B))
        got = bt.result(i)
        assert torch.equal(got.rowptr.cpu(), single.rowptr.cpu())
        assert torch.equal(got.colidx.cpu(), single.colidx.cpu())


def test_batch_many_er_products(pb):
    """A few hundred ER products with the size and degree mix of the batched workload, scaled down."""
    shapes = synth.batch_er_shapes(300, seed=11, n_lo=512, n_hi=8192)
    probs = [synth.er(n, d, seed=1000 + i) for i, (n, d) in enumerate(shapes)]
    bt = run_batch(pb, probs)
    assert bt.status() == 0
    for i in range(0, 300, 7):
        assert_matches(bt.result(i), oracle.spgemm(*probs[i]), EPS["f64"])


def test_batch_cuda_graph_replay(pb):
    """Capture one batch launch, replay it after the operand values change."""
    probs = mixed_problems(6)[:18]
    handle = pb.Handle()
    As = [pb.csc_to_device(A) for A, _ in probs]
    Bs = [pb.csr_to_device(B) for _, B in probs]
    bt = pb.Batch(As, Bs, handle=handle)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.run(stream=s)  # warm-up outside capture (kernel attributes, lazy module loading)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    launches0 = pb.kernel_launches()
    with torch.cuda.graph(g, stream=s):
        bt.run(stream=s)
    assert pb.kernel_launches() > launches0
    for rep in range(2):
        rng = np.random.default_rng(100 + rep)
        new = []
        for (A, B), Ad, Bd in zip(probs, As, Bs):
            av = rng.uniform(-1, 1, A.nnz)
            bv = rng.uniform(-1, 1, B.nnz)
            Ad.val.copy_(torch.from_numpy(av))
            Bd.val.copy_(torch.from_numpy(bv))
            new.append((synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, av),
                        synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, bv)))
        bt.device_status.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        check_all(bt, new, EPS["f64"])


def test_batch_autotune(pb):
    shapes = [(600, 2), (700, 3), (3000, 8), (2500, 9), (9000, 4), (12000, 16)]
    probs = [synth.er(n, d, seed=40 + i) for i, (n, d) in enumerate(shapes)]
    handle = pb.Handle()
    As = [pb.csc_to_device(A) for A, _ in probs]
    Bs = [pb.csr_to_device(B) for _, B in probs]
    bt = pb.Batch(As, Bs, handle=handle)
    bt.autotune(reps=1)
    table = pb.get_tuning(handle)
    assert len(table) == len({(int(np.ceil(np.log2(n))), d.bit_length()) for n, d in shapes})
    for e in table:
        assert e["bin_capacity"] in (2048, 4096, 8192) and 1 <= e["rmax_log2"] <= 11
    check_all(bt, probs, EPS["f64"])   # the autotuner leaves C holding the products
    bt.run()
    check_all(bt, probs, EPS["f64"])


def test_batch_c_overflow_status(pb):
    probs = [synth.er(2000, 6, seed=1), synth.er(1500, 4, seed=2)]
    handle = pb.Handle()
    As = [pb.csc_to_device(A) for A, _ in probs]
    Bs = [pb.csr_to_device(B) for _, B in probs]
    caps = [oracle.spgemm(*probs[0]).nnz, oracle.spgemm(*probs[1]).nnz - 1]  # the second C is one entry short
    bt = pb.Batch(As, Bs, handle=handle, caps=caps)
    bt.run()
    assert bt.status() == 5  # PB_ERR_OVERFLOW
    assert_matches(bt.result(0), oracle.spgemm(*probs[0]), EPS["f64"])


def hub_problems(seed=0):
    """R-MAT products of scale 10..12, whose hub rows exceed every bin capacity,
    mixed with ER products and with single dense rows at a product's first and
    last row (one row of 100 x 100 = 10,000 tuples merging into 100 entries)."""
    rng = np.random.default_rng(seed)
    probs = [synth.rmat(sc, ef, seed=seed * 100 + i)
             for i, (sc, ef) in enumerate([(10, 8), (11, 8), (12, 8), (12, 16), (10, 16), (11, 4)])]
    probs += [synth.er(3000, 8, seed=seed + 7), synth.er(500, 3, seed=seed + 8)]
    k = 100
    Bd = rng.uniform(-1, 1, (k, 100))
    r, c = np.nonzero(Bd)
    B = synth.coo_to_csr(k, 100, r, c, Bd[r, c])
    for row in (0, 2):
        A = synth.coo_to_csc(3, k, np.full(k, row, np.int64), np.arange(k), rng.uniform(-1, 1, k))
        probs.append((A, B))
    return probs


def test_batch_hub_rows(pb):
    """Rows above the bin capacity are merged inside the batch (Sec. III-D)."""
    probs = hub_problems(0)
    heavy = [int(oracle.row_flop(A, B).max()) for A, B in probs]
    assert max(heavy) > 8192 and sum(h > 4096 for h in heavy) >= 6
    bt = run_batch(pb, probs)
    for i, (A, B) in enumerate(probs):
        assert int(bt.max_row[i]) == heavy[i]
    check_all(bt, probs, EPS["f64"])


@pytest.mark.parametrize("cap", [2048, 4096, 8192])
def test_batch_hub_rows_each_level(pb, cap):
    probs = hub_problems(1)
    check_all(run_batch(pb, probs, tuning=all_classes(probs, cap)), probs, EPS["f64"])


def test_batch_hub_rows_fp32_tuples_and_int32_rowptr(pb):
    probs = hub_problems(2)
    probs32 = [(synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.val.astype(np.float32)),
                synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, B.val.astype(np.float32))) for A, B in probs]
    check_all(run_batch(pb, probs32, dtype=1, vdt=torch.float32), probs32, EPS["f32"])
    check_all(run_batch(pb, probs, dtype=2), probs, EPS["f32"])
    check_all(run_batch(pb, probs, rowptr64=False), probs, EPS["f64"])


def test_batch_hub_rows_cuda_graph_replay(pb):
    """A batch with hub rows captured once and replayed after the values change."""
    probs = hub_problems(3)
    handle = pb.Handle()
    As = [pb.csc_to_device(A) for A, _ in probs]
    Bs = [pb.csr_to_device(B) for _, B in probs]
    bt = pb.Batch(As, Bs, handle=handle)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    check_all(bt, probs, EPS["f64"])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bt.run(stream=s)
    for rep in range(2):
        rng = np.random.default_rng(200 + rep)
        new = []
        for (A, B), Ad, Bd in zip(probs, As, Bs):
            av = rng.uniform(-1, 1, A.nnz)
            bv = rng.uniform(-1, 1, B.nnz)
            Ad.val.copy_(torch.from_numpy(av))
            Bd.val.copy_(torch.from_numpy(bv))
            new.append((synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, av),
                        synth.CSR(B.nrows, B.ncols, B.rowptr, B.colidx, bv)))
        bt.device_status.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        check_all(bt, new, EPS["f64"])


def test_batch_hub_row_in_too_wide_product_rejected(pb):
    """A hub row of a product with more than 2^22 columns is beyond the dense tiles:
    the batch reports PB_ERR_UNSUPPORTED and the single-product path computes it."""
    rng = np.random.default_rng(0)
    k, n = 100, (1 << 22) + 1
    A = synth.coo_to_csc(3, k, np.zeros(k, np.int64), np.arange(k), rng.uniform(-1, 1, k))   # row 0 full
    rows = np.repeat(np.arange(k), 50)
    cols = np.concatenate([np.sort(rng.choice(n, 50, replace=False)) for _ in range(k)])
    B = synth.coo_to_csr(k, n, rows, cols, rng.uniform(-1, 1, k * 50))                      # row flop 5000
    probs = [synth.er(500, 3, seed=9), (A, B)]
    bt = run_batch(pb, probs)
    assert int(bt.max_row[1]) == 5000
    assert bt.status() == 9  # PB_ERR_UNSUPPORTED
    C = pb.spgemm(pb.csc_to_device(A), pb.csr_to_device(B))
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])


def test_batch_exact_queried_workspace_every_row_its_own_bin(pb):
    """A workspace of exactly the queried size suffices when every row is a bin of
    its own.  At capacity 2048, rows of 1250..1800 tuples (above half the capacity)
    each make a bin and leave the query 8 tuples of slack; one product's rows of
    3000 tuples are hub rows."""
    rng = np.random.default_rng(7)
    probs = []
    for rows, k, n in ((4, 100, 15), (3, 60, 30), (6, 50, 25), (2, 100, 30)):   # row flop 1500, 1800, 1250, 3000
        A = synth.coo_to_csc(rows, k, np.repeat(np.arange(rows), k), np.tile(np.arange(k), rows),
                             rng.uniform(-1, 1, rows * k))
        Bd = rng.uniform(-1, 1, (k, n))
        r, c = np.nonzero(Bd)
        probs.append((A, synth.coo_to_csr(k, n, r, c, Bd[r, c])))
    handle = pb.Handle()
    pb.set_tuning(all_classes(probs, 2048), handle)
    As = [pb.csc_to_device(A) for A, _ in probs]
    Bs = [pb.csr_to_device(B) for _, B in probs]
    bt = pb.Batch(As, Bs, handle=handle)
    bt.workspace_bytes -= 256   # the binding's margin off: exactly what the query reported
    bt.run()
    check_all(bt, probs, EPS["f64"])


def test_batch_workspace_too_small(pb):
    probs = [synth.er(3000, 8, seed=12), synth.er(2000, 5, seed=13)]
    handle = pb.Handle()
    As = [pb.csc_to_device(A) for A, _ in probs]
    Bs = [pb.csr_to_device(B) for _, B in probs]
    bt = pb.Batch(As, Bs, handle=handle)
    full = bt.workspace_bytes
    total_flop = int(sum(bt.flop))
    bt.workspace_bytes = full - 12 * total_flop // 2   # room for about half of the tuples
    bt.run()
    assert bt.status() == 10  # PB_ERR_WORKSPACE
    bt.workspace_bytes = full
    bt.run()
    check_all(bt, probs, EPS["f64"])


def test_batch_empty(pb):
    bt = pb.Batch([], [], handle=pb.Handle())
    bt.run()
    assert bt.status() == 0


def test_batch_tuning_table_validation(pb):
    handle = pb.Handle()
    good = [dict(log2n=12, dclass=3, bin_capacity=2048, rmax_log2=9, expand_chunk=1024)]
    pb.set_tuning(good, handle)
    assert pb.get_tuning(handle) == good
    for bad in (dict(good[0], bin_capacity=3000), dict(good[0], rmax_log2=12), dict(good[0], expand_chunk=100)):
        with pytest.raises(pb.PBError) as ei:
            pb.set_tuning([bad], handle)
        assert ei.value.status == 1
    assert pb.get_tuning(handle) == good
