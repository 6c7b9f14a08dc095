"""Serving (pb_server_*): continuous batching of AMG Galerkin and Markov-clustering requests.

Each result must match the CPU oracle (structure bit-exact, values within
64 * eps * sum |a b|), the AMG coarse operator must equal its closed form
(24 on the diagonal, -4 for face neighbours, exact in FP64), and every result
computed in a mix of concurrent requests must equal the same request computed
alone.  Budgets are checked: the server never holds more than its budget.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EPS, TOL_FACTOR, assert_csr_valid, assert_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import binding
    binding.load_library()
    return binding


def amg_host(N):
    A = synth.poisson7(N)
    A_csc = synth.CSC(A.nrows, A.ncols, A.rowptr, A.colidx, A.val)  # symmetric: CSR arrays are CSC arrays
    return A_csc, synth.aggregation_prolongator(N)


def galerkin_oracle(A_csc, P):
    AP = oracle.spgemm(A_csc, P)
    AP_csr = synth.CSR(A_csc.nrows, P.ncols, AP.rowptr.astype(np.int32), AP.colidx, AP.val)
    return oracle.spgemm(synth.transpose_csr_as_csc(P), AP_csr)


def mcl_host(scale, seed):
    Ac, _ = synth.rmat(scale, 8, seed=seed)
    return synth.column_stochastic(Ac, dtype=np.float32)


def coarse_closed_form(N):
    """P^T A P for the 7-point stencil and 2x2x2 aggregation, as a dense matrix."""
    M = N // 2
    ref = np.zeros((M ** 3, M ** 3))
    for I in range(M ** 3):
        x, y, z = I % M, (I // M) % M, I // (M * M)
        ref[I, I] = 24.0
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            xx, yy, zz = x + dx, y + dy, z + dz
            if 0 <= xx < M and 0 <= yy < M and 0 <= zz < M:
                ref[I, xx + M * yy + M * M * zz] = -4.0
    return ref


def dense(C):
    rp, ci, va = C.rowptr.cpu().numpy(), C.colidx.cpu().numpy(), C.val.double().cpu().numpy()
    D = np.zeros((C.nrows, C.ncols))
    for i in range(C.nrows):
        D[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    return D


def test_galerkin_request_closed_form(pb):
    srv = pb.Server(1 << 30, max_slots=2)
    N = 8
    A, P = amg_host(N)
    rid = srv.submit_galerkin(pb.csc_to_device(A), pb.csr_to_device(P))
    assert srv.wait(rid) == 0
    C = srv.result(rid)
    assert C.nrows == C.ncols == (N // 2) ** 3
    assert np.array_equal(dense(C), coarse_closed_form(N))
    assert_matches(C, galerkin_oracle(A, P), EPS["f64"])
    srv.release(rid)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_mcl_request_fp32(pb):
    srv = pb.Server(1 << 30, max_slots=2)
    Mc, Mr = mcl_host(10, seed=3)
    rid = srv.submit_product(pb.csc_to_device(Mc, val_dtype=torch.float32),
                             pb.csr_to_device(Mr, val_dtype=torch.float32), dtype=pb.PB_F32)
    assert srv.wait(rid) == 0
    C = srv.result(rid)
    assert_matches(C, oracle.spgemm(Mc, Mr), EPS["f32"])
    colsum = np.bincount(C.colidx.cpu().numpy(), weights=C.val.double().cpu().numpy(), minlength=Mc.ncols)
    assert np.allclose(colsum, 1.0, atol=1e-5)
    srv.release(rid)
    srv.close()


def mixed_requests(pb, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for j in range(24):
        if j % 2 == 0:
            N = int(rng.choice([4, 8, 12, 16]))
            A, P = amg_host(N)
            reqs.append(("galerkin", A, P, pb.PB_F64, pb.csc_to_device(A), pb.csr_to_device(P)))
        else:
            Mc, Mr = mcl_host(int(rng.integers(7, 12)), seed=int(rng.integers(1 << 20)))
            reqs.append(("product", Mc, Mr, pb.PB_F32, pb.csc_to_device(Mc, val_dtype=torch.float32),
                         pb.csr_to_device(Mr, val_dtype=torch.float32)))
    return reqs


def submit(srv, r):
    kind, _, _, dt, Ad, Bd = r
    return srv.submit_galerkin(Ad, Bd, dt) if kind == "galerkin" else srv.submit_product(Ad, Bd, dt)


def host_result(C):
    return C.rowptr.cpu().numpy(), C.colidx.cpu().numpy(), C.val.double().cpu().numpy()


def test_mixed_stream_same_as_alone(pb):
    """Results of 24 concurrent requests equal the oracle and the same requests run alone."""
    reqs = mixed_requests(pb, 1)
    srv = pb.Server(4 << 30, max_slots=4)
    ids = [submit(srv, r) for r in reqs]
    mixed = []
    for rid in ids:
        assert srv.wait(rid) == 0
        mixed.append(host_result(srv.result(rid)))
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["bytes_in_use"] == 0 and st["peak_bytes"] <= 4 << 30
    srv.close()
    alone_srv = pb.Server(4 << 30, max_slots=1)
    for r, got in zip(reqs, mixed):
        kind, A, B, dt, _, _ = r
        rid = submit(alone_srv, r)
        assert alone_srv.wait(rid) == 0
        alone = host_result(alone_srv.result(rid))
        alone_srv.release(rid)
        eps = EPS["f64"] if dt == pb.PB_F64 else EPS["f32"]
        ref = galerkin_oracle(A, B) if kind == "galerkin" else oracle.spgemm(A, B)
        assert np.array_equal(got[0], alone[0]) and np.array_equal(got[1], alone[1])
        assert np.array_equal(got[0], ref.rowptr) and np.array_equal(got[1], ref.colidx)
        # both lie within 64 eps sum|ab| of the exact result (per product of the chain)
        bound = TOL_FACTOR * eps * ref.absval
        assert np.all(np.abs(got[2] - ref.val) <= bound) or kind == "galerkin"
        assert np.all(np.abs(got[2] - alone[2]) <= 2 * bound) or kind == "galerkin"
        if kind == "galerkin":  # integer data: exact in any order
            assert np.array_equal(got[2], ref.val) and np.array_equal(alone[2], ref.val)
    alone_srv.close()


def drain(srv, ids, check):
    """Poll every pending request; check and release each as it finishes (as a client would)."""
    import time
    pending = dict(enumerate(ids))
    t0 = time.time()
    while pending:
        for j, rid in list(pending.items()):
            done, st = srv.poll(rid)
            if done:
                assert st == 0, f"request {j}: status {st}"
                check(j, srv.result(rid))
                srv.release(rid)
                del pending[j]
        assert time.time() - t0 < 120, "requests did not finish"
        time.sleep(0.001)


def step_needs(pb, r):
    """Per product step of a request: (bytes with an exact C, bytes with a flop-sized C), as the server counts."""
    kind, A, B, dt, Ad, Bd = r
    vb = 8 if dt == pb.PB_F64 else 4
    steps = [(A, B, Ad, Bd, 4 if kind == "galerkin" else 8)]
    if kind == "galerkin":
        AP = oracle.spgemm(A, B)
        APc = synth.CSR(A.nrows, B.ncols, AP.rowptr.astype(np.int32), AP.colidx, AP.val)
        steps.append((synth.transpose_csr_as_csc(B), APc, pb.CscMatrix(B.ncols, B.nrows, Bd.rowptr, Bd.colidx, Bd.val),
                      pb.csr_to_device(APc), 8))
    out = []
    held = 0
    for A1, B1, A1d, B1d, rp in steps:
        plan = pb.symbolic(A1d, B1d, dtype=dt)
        nnz = oracle.spgemm(A1, B1).nnz
        base = held + 16 * (A1.ncols + 2) + 96 * (A1.nrows + 2) + 12 * A1.nnz + (1 << 20) + plan.workspace_bytes
        base += rp * (A1.nrows + 1) + 4096
        out.append((base + (4 + vb) * nnz, base + (4 + vb) * plan.flop))
        held = rp * (A1.nrows + 1) + (4 + vb) * nnz + 1024
    return out


def test_tight_budget_counting_runs_and_preemption(pb):
    """A budget that holds the largest request only with an exactly sized C: the largest requests are
    sized by counting runs, the others wait or are preempted, and the budget is never exceeded."""
    reqs = mixed_requests(pb, 2)
    needs = [n for r in reqs for n in step_needs(pb, r)]
    budget = max(exact for exact, _ in needs) + (1 << 20)
    assert any(flop_sized > budget for _, flop_sized in needs)   # some steps must count first
    srv = pb.Server(budget, max_slots=4)
    ids = [submit(srv, r) for r in reqs]

    def check(j, C):
        kind, A, B, dt, _, _ = reqs[j]
        ref = galerkin_oracle(A, B) if kind == "galerkin" else oracle.spgemm(A, B)
        if kind == "galerkin":
            assert np.array_equal(host_result(C)[2], ref.val)
        assert_matches(C, ref, EPS["f64"] if dt == pb.PB_F64 else EPS["f32"])
        assert_csr_valid(C, C.ncols)

    drain(srv, ids, check)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["peak_bytes"] <= budget, st
    assert st["bytes_in_use"] == 0
    srv.close()


def test_request_larger_than_budget_is_busy(pb):
    srv = pb.Server(1 << 20, max_slots=2)   # 1 MiB
    A, B = synth.er(20000, 8, seed=5)
    Ad, Bd = pb.csc_to_device(A), pb.csr_to_device(B)
    with pytest.raises(pb.PBError) as ei:   # the operands' index arrays alone exceed the budget
        srv.submit_product(Ad, Bd)
    assert ei.value.status == 8
    A2, B2 = synth.er(3000, 8, seed=6)      # small operands, but C and the tuples exceed 1 MiB
    rid = srv.submit_product(pb.csc_to_device(A2), pb.csr_to_device(B2))
    assert srv.wait(rid) == 8               # PB_ERR_BUSY
    srv.release(rid)
    srv.close()


def test_results_resident_until_release(pb):
    srv = pb.Server(1 << 30, max_slots=2)
    A, B = synth.er(5000, 6, seed=7)
    rid = srv.submit_product(pb.csc_to_device(A), pb.csr_to_device(B))
    assert srv.wait(rid) == 0
    held = srv.stats()["bytes_in_use"]
    assert held > 0
    C = srv.result(rid, copy=False)          # a view of the server's memory
    assert_matches(C, oracle.spgemm(A, B), EPS["f64"])
    q, t = srv.timing(rid)
    assert 0 <= q <= t
    srv.release(rid)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_small_requests_coalesced(pb):
    """Small requests that queue together run as batched launches (Galerkin members:
    one launch for all A P, one for all P^T (A P)).  Each result matches the oracle
    (Galerkin: the closed form, exactly); FP64 and FP32 requests never share a
    launch.  With coalescing off the same requests run one by one."""
    reqs = mixed_requests(pb, 3)
    Abig, Bbig = synth.er(1 << 20, 8, seed=9)   # above the small-request bound: runs alone
    big = (pb.csc_to_device(Abig), pb.csr_to_device(Bbig))
    for batching in (True, False):
        srv = pb.Server(8 << 30, max_slots=1)
        if not batching:
            srv.set_batching(1, 0.0)
        # two long requests hold the only slot while the small ones queue up behind them
        first = [srv.submit_product(*big), srv.submit_product(*big)]
        ids = [submit(srv, r) for r in reqs]
        for rid in first:
            assert srv.wait(rid) == 0
            srv.release(rid)

        def check(j, C):
            kind, A, B, dt, _, _ = reqs[j]
            if kind == "galerkin":
                N = round(A.nrows ** (1 / 3))
                assert np.array_equal(dense(C), coarse_closed_form(N))
            else:
                assert_matches(C, oracle.spgemm(A, B), EPS["f32"])
            assert_csr_valid(C, C.ncols)

        drain(srv, ids, check)
        st = srv.stats()
        assert st["completed"] == len(reqs) + 2 and st["bytes_in_use"] == 0
        if batching:
            # at least the FP64 Galerkin group (two launches) and the FP32 group ran batched
            assert st["batched_requests"] >= 4 and st["batch_launches"] >= 3, st
        else:
            assert st["batched_requests"] == 0 and st["batch_launches"] == 0, st
        srv.close()
