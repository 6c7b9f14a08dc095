// Serving loop with continuous batching over the PB-SpGEMM entry points.
//
// A server has `max_slots` slots; each slot is a host thread with its own CUDA
// stream and library handle.  A free slot takes the oldest queued request and
// runs it to completion: a short chain of products (one for C = A*B, two for
// the Galerkin product P^T (A P)), each as the symbolic phase (Alg. 3; its one
// host synchronisation blocks only this slot), optionally a counting run (when
// a flop-sized C could never fit the budget), then the numeric phase (Alg. 2).
// Slots run concurrently, so a request that arrives while others are on the
// GPU starts as soon as a slot and memory are free and its kernels overlap
// with theirs.  Among queued requests the one with the least estimated work
// goes first (nnz(A) times the mean row length of B), unless the oldest has
// been passed over MAX_BYPASS times already.
//
// Small requests are coalesced: a slot that admits a request of at most
// `batch_work` estimated work also takes the other queued small requests of
// the same value type (up to `batch_max` in all) and runs them as one batched
// launch (pb_spgemm_batch; a Galerkin group as two: A P for all members, then
// P^T (A P)).  If the group cannot run as a batch (its need exceeds the
// budget, a device error), its members run one by one.
//
// Every device byte the server holds (plans, workspaces, intermediates and
// results) comes from the server's own memory pool and is counted against the
// budget before it is allocated.  A slot that lacks memory waits; no new
// request is admitted while any slot waits.  When every busy slot waits, the
// most recently admitted request is preempted: its memory is released and it
// is queued again at the front.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pb_common.cuh"
#include "pb_host.h"

using namespace pb;

namespace {

using Clock = std::chrono::steady_clock;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Req {
    uint64_t id = 0;
    pb_request r{};
    int nsteps = 1;
    bool done = false;
    bool preempt = false;  // set by another slot: release everything and queue again
    bool waiting = false;  // waiting for memory
    pb_status result = PB_OK;
    int restarts = 0;
    bool admitted_once = false;
    int bypassed = 0;      // later requests admitted before this one
    double est = 0;        // estimated work (flop)
    Clock::time_point t_submit, t_first_admit, t_admit, t_done;
    int64_t nnz = 0;
    Buf out_rowptr, out_colidx, out_val;  // the final C
};

size_t val_bytes(int32_t dtype) { return dtype == PB_F32 ? 4 : 8; }

}  // namespace

struct pb_server {
    pb_handle *user = nullptr;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    size_t budget = 0, in_use = 0, peak = 0;
    int max_slots = 0;
    std::vector<cudaStream_t> streams;
    std::vector<pb_handle *> hs;  // one library handle per slot (plans come from the server pool)
    std::vector<Req *> active;    // request running in each slot
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> threads;
    bool stop = false;
    int waiting = 0;  // slots waiting for memory
    uint64_t next_id = 1;
    int64_t completed = 0, preempted = 0;
    int batch_max = 16;                   // requests per coalesced launch (1: no coalescing)
    double batch_work = (double)(1 << 24);  // largest estimated work of a coalesced request
    int64_t batched_requests = 0, batch_launches = 0;
};

namespace {

constexpr int MAX_BYPASS = 16;

struct SlotCtx {
    pb_server *S;
    int slot;
};

// ---- budget -----------------------------------------------------------------
// Reserve `b` bytes, waiting while they do not fit.  Returns false when this
// request has been chosen for preemption.
bool wait_reserve(pb_server *S, Req *q, size_t b) {
    std::unique_lock<std::mutex> lk(S->mu);
    bool counted = false;
    while (S->in_use + b > S->budget) {
        if (q->preempt) break;
        if (!counted) {
            counted = true;
            q->waiting = true;
            ++S->waiting;
        }
        int busy = 0;
        Req *youngest = nullptr;
        for (Req *x : S->active) {
            if (!x) continue;
            ++busy;
            if (x->waiting && (!youngest || x->t_admit > youngest->t_admit)) youngest = x;
        }
        if (busy >= 2 && S->waiting == busy && youngest) {
            youngest->preempt = true;
            S->cv_work.notify_all();
            if (youngest == q) break;
        }
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
    if (counted) {
        q->waiting = false;
        --S->waiting;
        S->cv_work.notify_all();
    }
    if (q->preempt) return false;
    S->in_use += b;
    S->peak = std::max(S->peak, S->in_use);
    return true;
}

// Replace a reservation of `was` bytes by one of `now` bytes in one step, so no
// other slot can take the difference in between.
void swap_reserve(pb_server *S, size_t was, size_t now) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use = S->in_use - std::min(was, S->in_use) + now;
    S->peak = std::max(S->peak, S->in_use);
    if (now < was) S->cv_work.notify_all();
}

void unreserve(pb_server *S, size_t b) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= std::min(b, S->in_use);
    S->cv_work.notify_all();
}

// Allocate bytes already reserved; on success they move from *left to b.
pb_status alloc(pb_server *S, cudaStream_t s, Buf &b, size_t bytes, size_t *left) {
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, S->pool, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return PB_ERR_OOM;
    }
    b.p = p;
    b.bytes = bytes;
    *left -= bytes;
    return PB_OK;
}

// nnz(C) written by the step's kernels, read on the slot's stream.
pb_status read_nnz(cudaStream_t s, const Buf &nnz, int64_t *out) {
    if (cudaMemcpyAsync(out, nnz.p, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PB_ERR_CUDA;
    return PB_OK;
}

void put(pb_server *S, cudaStream_t s, Buf &b) {
    if (!b.p) return;
    (void)cudaFreeAsync(b.p, s);
    unreserve(S, b.bytes);
    b = Buf{};
}

size_t r256(size_t b) { return std::max<size_t>((b + 255) & ~size_t(255), 256); }

// Allocator of the slots' handles: plan arrays from the server pool (counted
// by the caller through plan_device_bytes).
void *pool_alloc(size_t bytes, pb_stream_t stream, void *ctx) {
    pb_server *S = static_cast<pb_server *>(ctx);
    void *p = nullptr;
    cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : S->streams[0];
    if (cudaMallocFromPoolAsync(&p, bytes ? bytes : 256, S->pool, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Plans are destroyed only after their stream has finished with them.
void pool_free(void *p, size_t, pb_stream_t stream, void *ctx) {
    pb_server *S = static_cast<pb_server *>(ctx);
    if (p) (void)cudaFreeAsync(p, stream ? reinterpret_cast<cudaStream_t>(stream) : S->streams[0]);
}

// Upper estimate of a plan's device bytes, reserved while the plan is built.
size_t plan_estimate(const pb_csc &A) {
    const size_t m = (size_t)A.nrows, k = (size_t)A.ncols, e = (size_t)A.nnz;
    return 16 * (k + 2) + 96 * (m + 2) + 12 * e + (1u << 20);
}

void finish(pb_server *S, Req *q, pb_status st) {
    std::lock_guard<std::mutex> lk(S->mu);
    q->result = st;
    q->t_done = Clock::now();
    q->done = true;
    ++S->completed;
    S->cv_done.notify_all();
}

// Everything one request holds while it runs in a slot.
struct Held {
    pb_plan *plan = nullptr;
    size_t plan_bytes = 0;
    Buf ws, nnz, prev_rowptr, prev_colidx, prev_val, out_rowptr, out_colidx, out_val;
    int64_t prev_nnz = 0;
};

void drop_step(pb_server *S, cudaStream_t s, Held &h) {
    put(S, s, h.ws);
    put(S, s, h.nnz);
    if (h.plan) pb_plan_destroy(h.plan);
    h.plan = nullptr;
    unreserve(S, h.plan_bytes);
    h.plan_bytes = 0;
}

void drop_all(pb_server *S, cudaStream_t s, Held &h) {
    drop_step(S, s, h);
    for (Buf *b : {&h.prev_rowptr, &h.prev_colidx, &h.prev_val, &h.out_rowptr, &h.out_colidx, &h.out_val})
        put(S, s, *b);
}

enum Outcome { OK_DONE, FAILED, PREEMPTED };

// Run request q in a slot.  On success the final C stays reserved and owned by q.
Outcome run(pb_server *S, int slot, Req *q, pb_status *status) {
    pb_handle *hd = S->hs[slot];
    cudaStream_t s = S->streams[slot];
    pb_stream_t ps = reinterpret_cast<pb_stream_t>(s);
    const pb_request &r = q->r;
    const int32_t dtype = r.dtype;
    const size_t vb = val_bytes(dtype);
    Held h;
    size_t left = 0;  // reserved but not yet allocated
    auto fail = [&](pb_status st) {
        (void)cudaStreamSynchronize(s);  // nothing launched may still use what is freed
        unreserve(S, left);
        left = 0;
        drop_all(S, s, h);
        *status = st;
        return FAILED;
    };
    auto preempted = [&]() {
        drop_all(S, s, h);
        return PREEMPTED;
    };
    for (int step = 0; step < q->nsteps; ++step) {
        // the operands of this step
        pb_csc A = r.A;
        pb_csr B = r.B;
        bool intermediate = false;
        if (r.kind == PB_REQ_GALERKIN && step == 0) {
            intermediate = true;  // AP = A * P, the next step's B
        } else if (r.kind == PB_REQ_GALERKIN) {
            // P^T as CSC is P's CSR arrays read column-wise; AP is the previous step's C
            A = pb_csc{r.B.ncols, r.B.nrows, r.B.nnz, r.B.rowptr, r.B.colidx, r.B.val};
            B = pb_csr{r.A.nrows, r.B.ncols, h.prev_nnz, static_cast<const int32_t *>(h.prev_rowptr.p),
                       static_cast<const int32_t *>(h.prev_colidx.p), h.prev_val.p};
        }
        const size_t held_prev = h.prev_rowptr.bytes + h.prev_colidx.bytes + h.prev_val.bytes;
        // symbolic phase
        const size_t est = plan_estimate(A);
        if (est + held_prev > S->budget) return fail(PB_ERR_BUSY);
        if (!wait_reserve(S, q, est)) return preempted();
        pb_config cfg{};
        cfg.max_tuple_bytes = (int64_t)(S->budget / 2);  // larger products run in row panels
        pb_status st = pb_spgemm_symbolic(hd, &A, &B, (pb_dtype)dtype, &cfg, ps, &h.plan);
        if (st != PB_OK) {
            unreserve(S, est);
            h.plan = nullptr;
            return fail(st);
        }
        h.plan_bytes = plan_device_bytes(h.plan);
        swap_reserve(S, est, h.plan_bytes);  // the estimate bounds the plan's actual size
        int64_t flop = 0;
        size_t ws_bytes = 0;
        pb_plan_query(h.plan, &flop, nullptr, &ws_bytes, nullptr, nullptr);
        const size_t m = (size_t)A.nrows;
        const size_t rp = intermediate ? 4 : 8;
        auto out_bytes = [&](int64_t cap) {
            const size_t c = (size_t)std::max<int64_t>(cap, 1);
            return r256(rp * (m + 1)) + r256(4 * c) + r256(vb * c);
        };
        const size_t fixed = h.plan_bytes + held_prev + r256(ws_bytes) + 256;
        if (fixed > S->budget) return fail(PB_ERR_BUSY);
        int64_t cap = flop;
        if (fixed + out_bytes(flop) > S->budget) {
            // size C exactly first: the counting run needs only the workspace
            if (!wait_reserve(S, q, r256(ws_bytes) + 256)) return preempted();
            left = r256(ws_bytes) + 256;
            if ((st = alloc(S, s, h.ws, r256(ws_bytes), &left)) != PB_OK) return fail(st);
            if ((st = alloc(S, s, h.nnz, 256, &left)) != PB_OK) return fail(st);
            pb_csr_out Cc{A.nrows, B.ncols, 0, nullptr, nullptr, nullptr, nullptr, static_cast<int64_t *>(h.nnz.p)};
            pb_status dev = PB_OK;
            st = pb_spgemm_numeric(hd, h.plan, &A, &B, &Cc, h.ws.p, h.ws.bytes, ps);
            if (st == PB_OK) st = pb_plan_status(h.plan, ps, &dev);
            if (st == PB_OK) st = dev;
            int64_t nnz = 0;
            if (st == PB_OK) st = read_nnz(s, h.nnz, &nnz);
            if (st != PB_OK) return fail(st);
            cap = nnz;
        }
        if (fixed + out_bytes(cap) > S->budget) return fail(PB_ERR_BUSY);
        // what the step still lacks, reserved together
        const size_t lack = (h.ws.p ? 0 : r256(ws_bytes)) + (h.nnz.p ? 0 : 256) + out_bytes(cap);
        if (!wait_reserve(S, q, lack)) return preempted();
        left = lack;
        if (!h.ws.p && (st = alloc(S, s, h.ws, r256(ws_bytes), &left)) != PB_OK) return fail(st);
        if (!h.nnz.p && (st = alloc(S, s, h.nnz, 256, &left)) != PB_OK) return fail(st);
        const size_t c = (size_t)std::max<int64_t>(cap, 1);
        if ((st = alloc(S, s, h.out_rowptr, r256(rp * (m + 1)), &left)) != PB_OK) return fail(st);
        if ((st = alloc(S, s, h.out_colidx, r256(4 * c), &left)) != PB_OK) return fail(st);
        if ((st = alloc(S, s, h.out_val, r256(vb * c), &left)) != PB_OK) return fail(st);
        pb_csr_out C{A.nrows, B.ncols, cap, intermediate ? nullptr : static_cast<int64_t *>(h.out_rowptr.p),
                     intermediate ? static_cast<int32_t *>(h.out_rowptr.p) : nullptr,
                     static_cast<int32_t *>(h.out_colidx.p), h.out_val.p, static_cast<int64_t *>(h.nnz.p)};
        pb_status dev = PB_OK;
        st = pb_spgemm_numeric(hd, h.plan, &A, &B, &C, h.ws.p, h.ws.bytes, ps);
        if (st == PB_OK) st = pb_plan_status(h.plan, ps, &dev);  // synchronises this slot's stream only
        if (st == PB_OK) st = dev;
        int64_t nnz = 0;
        if (st == PB_OK) st = read_nnz(s, h.nnz, &nnz);
        if (st != PB_OK) return fail(st);
        drop_step(S, s, h);
        if (intermediate) {
            for (Buf *b : {&h.prev_rowptr, &h.prev_colidx, &h.prev_val}) put(S, s, *b);
            h.prev_rowptr = h.out_rowptr;
            h.prev_colidx = h.out_colidx;
            h.prev_val = h.out_val;
            h.prev_nnz = nnz;
            h.out_rowptr = h.out_colidx = h.out_val = Buf{};
        } else {
            q->nnz = nnz;
        }
    }
    for (Buf *b : {&h.prev_rowptr, &h.prev_colidx, &h.prev_val}) put(S, s, *b);
    q->out_rowptr = h.out_rowptr;
    q->out_colidx = h.out_colidx;
    q->out_val = h.out_val;
    *status = PB_OK;
    return OK_DONE;
}

// ---- coalesced small requests -----------------------------------------------
// One batched launch: the products of a group's members and their results.
struct BatchStep {
    std::vector<Req *> owner;
    std::vector<pb_csc> A;
    std::vector<pb_csr> B;
    std::vector<bool> rp32;  // int32 row pointers (an intermediate AP)
    std::vector<Buf> rowptr, colidx, val;
    std::vector<int64_t> nnz;
    void add(Req *q, const pb_csc &a, const pb_csr &b, bool r32) {
        owner.push_back(q);
        A.push_back(a);
        B.push_back(b);
        rp32.push_back(r32);
    }
};

void drop_step(pb_server *S, cudaStream_t s, BatchStep &st) {
    for (auto *v : {&st.rowptr, &st.colidx, &st.val})
        for (Buf &b : *v) put(S, s, b);
}

// Run a batch step: reserve, allocate, launch, read the statuses and nnz.
Outcome run_batch_step(pb_server *S, int slot, Req *primary, int32_t dtype, BatchStep &st, pb_status *status) {
    pb_handle *hd = S->hs[slot];
    cudaStream_t s = S->streams[slot];
    pb_stream_t ps = reinterpret_cast<pb_stream_t>(s);
    const int32_t n = (int32_t)st.A.size();
    const size_t vb = val_bytes(dtype);
    // the query's temporary index arrays, counted by the plans' estimate
    size_t est = 0;
    for (const pb_csc &a : st.A) est += plan_estimate(a);
    if (est > S->budget) {
        *status = PB_ERR_BUSY;
        return FAILED;
    }
    if (!wait_reserve(S, primary, est)) return PREEMPTED;
    std::vector<int64_t> flop((size_t)n, 0);
    size_t ws_bytes = 0;
    pb_status e = pb_spgemm_batch_query(hd, n, st.A.data(), st.B.data(), (pb_dtype)dtype, ps, &ws_bytes, flop.data(),
                                        nullptr);
    unreserve(S, est);
    if (e != PB_OK) {
        *status = e;
        return FAILED;
    }
    auto out_bytes = [&](int32_t i) {
        const size_t c = (size_t)std::max<int64_t>(flop[(size_t)i], 1);
        return r256((st.rp32[(size_t)i] ? 4 : 8) * ((size_t)st.A[(size_t)i].nrows + 1)) + r256(4 * c) + r256(vb * c);
    };
    size_t need = r256(ws_bytes) + r256(8 * (size_t)n) + 256;
    for (int32_t i = 0; i < n; ++i) need += out_bytes(i);
    if (need > S->budget) {
        *status = PB_ERR_BUSY;
        return FAILED;
    }
    if (!wait_reserve(S, primary, need)) return PREEMPTED;
    size_t left = need;
    Buf ws, nnz, dstat;
    st.rowptr.assign((size_t)n, Buf{});
    st.colidx.assign((size_t)n, Buf{});
    st.val.assign((size_t)n, Buf{});
    auto release = [&]() {
        (void)cudaStreamSynchronize(s);
        unreserve(S, left);
        left = 0;
        for (Buf *b : {&ws, &nnz, &dstat}) put(S, s, *b);
    };
    pb_status a = PB_OK;
    if ((a = alloc(S, s, ws, r256(ws_bytes), &left)) != PB_OK || (a = alloc(S, s, nnz, r256(8 * (size_t)n), &left)) != PB_OK ||
        (a = alloc(S, s, dstat, 256, &left)) != PB_OK) {
        release();
        drop_step(S, s, st);
        *status = a;
        return FAILED;
    }
    std::vector<pb_csr_out> C((size_t)n);
    for (int32_t i = 0; i < n && a == PB_OK; ++i) {
        const size_t k = (size_t)i, c = (size_t)std::max<int64_t>(flop[k], 1);
        if ((a = alloc(S, s, st.rowptr[k], r256((st.rp32[k] ? 4 : 8) * ((size_t)st.A[k].nrows + 1)), &left)) != PB_OK ||
            (a = alloc(S, s, st.colidx[k], r256(4 * c), &left)) != PB_OK ||
            (a = alloc(S, s, st.val[k], r256(vb * c), &left)) != PB_OK)
            break;
        C[k] = pb_csr_out{st.A[k].nrows, st.B[k].ncols, flop[k],
                          st.rp32[k] ? nullptr : static_cast<int64_t *>(st.rowptr[k].p),
                          st.rp32[k] ? static_cast<int32_t *>(st.rowptr[k].p) : nullptr,
                          static_cast<int32_t *>(st.colidx[k].p), st.val[k].p, static_cast<int64_t *>(nnz.p) + i};
    }
    int32_t dev = PB_OK;
    st.nnz.assign((size_t)n, 0);
    if (a == PB_OK)
        a = pb_spgemm_batch(hd, n, st.A.data(), st.B.data(), C.data(), (pb_dtype)dtype, ws.p, ws.bytes, ps,
                            static_cast<int32_t *>(dstat.p));
    if (a == PB_OK && (cudaMemcpyAsync(&dev, dstat.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaMemcpyAsync(st.nnz.data(), nnz.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaStreamSynchronize(s) != cudaSuccess))
        a = PB_ERR_CUDA;
    if (a == PB_OK) a = (pb_status)dev;
    release();
    if (a != PB_OK) {
        drop_step(S, s, st);
        *status = a;
        return FAILED;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->batch_launches;
    }
    return OK_DONE;
}

// Run a group of small requests as batched launches.  On success every member
// owns its final C; otherwise nothing is held.
Outcome run_group(pb_server *S, int slot, std::vector<Req *> &g, pb_status *status) {
    cudaStream_t s = S->streams[slot];
    const int32_t dtype = g[0]->r.dtype;
    BatchStep s1, s2;
    for (Req *q : g) s1.add(q, q->r.A, q->r.B, q->r.kind == PB_REQ_GALERKIN);  // Galerkin: AP = A * P
    Outcome o = run_batch_step(S, slot, g[0], dtype, s1, status);
    if (o != OK_DONE) return o;
    for (size_t i = 0; i < g.size(); ++i) {
        const pb_request &r = g[i]->r;
        if (r.kind != PB_REQ_GALERKIN) continue;
        // P^T as CSC is P's CSR arrays read column-wise; AP is step 1's C
        s2.add(g[i], pb_csc{r.B.ncols, r.B.nrows, r.B.nnz, r.B.rowptr, r.B.colidx, r.B.val},
               pb_csr{r.A.nrows, r.B.ncols, s1.nnz[i], static_cast<const int32_t *>(s1.rowptr[i].p),
                      static_cast<const int32_t *>(s1.colidx[i].p), s1.val[i].p},
               false);
    }
    if (!s2.A.empty()) {
        o = run_batch_step(S, slot, g[0], dtype, s2, status);
        // the intermediates AP are no longer needed either way
        (void)cudaStreamSynchronize(s);
        for (size_t i = 0; i < g.size(); ++i)
            if (g[i]->r.kind == PB_REQ_GALERKIN)
                for (Buf *b : {&s1.rowptr[i], &s1.colidx[i], &s1.val[i]}) put(S, s, *b);
        if (o != OK_DONE) {
            drop_step(S, s, s1);
            return o;
        }
    }
    size_t j = 0;
    for (size_t i = 0; i < g.size(); ++i) {
        Req *q = g[i];
        if (q->r.kind == PB_REQ_GALERKIN) {
            q->out_rowptr = s2.rowptr[j];
            q->out_colidx = s2.colidx[j];
            q->out_val = s2.val[j];
            q->nnz = s2.nnz[j];
            ++j;
        } else {
            q->out_rowptr = s1.rowptr[i];
            q->out_colidx = s1.colidx[i];
            q->out_val = s1.val[i];
            q->nnz = s1.nnz[i];
        }
    }
    *status = PB_OK;
    return OK_DONE;
}

void slot_main(SlotCtx c) {
    pb_server *S = c.S;
    const int slot = c.slot;
    (void)cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->queue.empty() || S->waiting > 0) {
            if (S->stop && S->queue.empty()) break;
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        // least estimated work first, within a bounded bypass of the oldest request
        size_t pick = 0;
        if (S->queue.front()->bypassed < MAX_BYPASS) {
            for (size_t i = 1; i < S->queue.size(); ++i)
                if (S->queue[i]->est < S->queue[pick]->est) pick = i;
        }
        Req *q = S->queue[pick];
        for (size_t i = 0; i < pick; ++i) ++S->queue[i]->bypassed;
        S->queue.erase(S->queue.begin() + (std::ptrdiff_t)pick);
        // a small request takes the other queued small requests of its value type along
        std::vector<Req *> group{q};
        if (S->batch_max > 1 && q->est <= S->batch_work) {
            for (size_t i = 0; i < S->queue.size() && (int)group.size() < S->batch_max;) {
                Req *x = S->queue[i];
                if (x->est <= S->batch_work && x->r.dtype == q->r.dtype) {
                    group.push_back(x);
                    S->queue.erase(S->queue.begin() + (std::ptrdiff_t)i);
                } else {
                    ++i;
                }
            }
        }
        S->active[slot] = q;
        const Clock::time_point now = Clock::now();
        for (Req *x : group) {
            x->preempt = false;
            x->t_admit = now;
            if (!x->admitted_once) {
                x->admitted_once = true;
                x->t_first_admit = now;
            }
        }
        lk.unlock();
        std::vector<Req *> requeue;
        if (group.size() > 1) {
            pb_status st = PB_OK;
            const Outcome o = run_group(S, slot, group, &st);
            if (o == OK_DONE) {
                for (Req *x : group) finish(S, x, PB_OK);
                std::lock_guard<std::mutex> g(S->mu);
                S->batched_requests += (int64_t)group.size();
            } else if (o == PREEMPTED) {
                requeue = group;
            } else {
                // one by one
                for (Req *x : group) {
                    {
                        std::lock_guard<std::mutex> g(S->mu);
                        S->active[slot] = x;
                        x->preempt = false;
                    }
                    pb_status sx = PB_OK;
                    const Outcome ox = run(S, slot, x, &sx);
                    if (ox == PREEMPTED)
                        requeue.push_back(x);
                    else
                        finish(S, x, sx);
                }
            }
        } else {
            pb_status st = PB_OK;
            const Outcome o = run(S, slot, q, &st);
            if (o != PREEMPTED)
                finish(S, q, st);
            else
                requeue.push_back(q);
        }
        lk.lock();
        S->active[slot] = nullptr;
        for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) {
            ++(*it)->restarts;
            ++S->preempted;
            S->queue.push_front(*it);
        }
        S->cv_work.notify_all();
    }
}

pb_status check_request(pb_server *S, const pb_request *r) {
    if (!r) return host_fail(S->user, PB_ERR_INVALID_ARG, "request must not be NULL");
    if (r->dtype != PB_F64 && r->dtype != PB_F32 && r->dtype != PB_F64_F32TUPLE)
        return host_fail(S->user, PB_ERR_UNSUPPORTED_DTYPE, "unknown dtype");
    pb_status st = host_check_operands(S->user, &r->A, &r->B);
    if (st != PB_OK) return st;
    if (r->kind == PB_REQ_GALERKIN) {
        if (r->A.nrows != r->A.ncols) return host_fail(S->user, PB_ERR_SHAPE, "Galerkin: A must be square");
    } else if (r->kind != PB_REQ_PRODUCT) {
        return host_fail(S->user, PB_ERR_INVALID_ARG, "unknown request kind");
    }
    return PB_OK;
}

Req *find(pb_server *S, uint64_t id) {
    auto it = S->reqs.find(id);
    return it == S->reqs.end() ? nullptr : it->second;
}

void free_result(pb_server *S, Req *q) {
    for (Buf *b : {&q->out_rowptr, &q->out_colidx, &q->out_val})
        if (b->p) {
            (void)cudaFreeAsync(b->p, S->streams[0]);
            S->in_use -= std::min(b->bytes, S->in_use);
            *b = Buf{};
        }
}

}  // namespace

extern "C" {

pb_status pb_server_create(pb_handle *h, size_t hbm_budget, int32_t max_slots, pb_server **out) {
    if (!h || !out || hbm_budget == 0 || max_slots < 1 || max_slots > 64) return PB_ERR_INVALID_ARG;
    *out = nullptr;
    pb_server *S = new (std::nothrow) pb_server();
    if (!S) return PB_ERR_OOM;
    S->user = h;
    S->device = h->device;
    S->budget = hbm_budget;
    S->max_slots = max_slots;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    cudaError_t e = cudaMemPoolCreate(&S->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = hbm_budget;  // keep freed memory in the pool up to the budget
        e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pb_status st = PB_OK;
    for (int i = 0; e == cudaSuccess && st == PB_OK && i < max_slots; ++i) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        S->streams.push_back(s);
        pb_handle *hs = nullptr;
        st = pb_create(&hs);
        if (st == PB_OK) st = pb_set_allocator(hs, pool_alloc, pool_free, S);
        if (hs) S->hs.push_back(hs);
    }
    cudaSetDevice(prev);
    if (e != cudaSuccess || st != PB_OK) {
        for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
        for (pb_handle *x : S->hs) pb_destroy(x);
        if (S->pool) cudaMemPoolDestroy(S->pool);
        delete S;
        if (e != cudaSuccess) return host_cuda_fail(h, e, "pb_server_create");
        return st;
    }
    S->active.assign(max_slots, nullptr);
    for (int i = 0; i < max_slots; ++i) S->threads.emplace_back(slot_main, SlotCtx{S, i});
    *out = S;
    return PB_OK;
}

pb_status pb_server_destroy(pb_server *S) {
    if (!S) return PB_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->threads) t.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto &kv : S->reqs) {
        free_result(S, kv.second);
        delete kv.second;
    }
    for (cudaStream_t s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (pb_handle *x : S->hs) pb_destroy(x);
    cudaMemPoolDestroy(S->pool);
    cudaSetDevice(prev);
    delete S;
    return PB_OK;
}

pb_status pb_serve_submit(pb_server *S, const pb_request *r, uint64_t *req_id) {
    if (!S || !req_id) return PB_ERR_INVALID_ARG;
    pb_status st = check_request(S, r);
    if (st != PB_OK) return st;
    const size_t lower = 12 * (size_t)r->A.nnz + 8 * ((size_t)r->A.nrows + (size_t)r->A.ncols);
    if (lower > S->budget) return host_fail(S->user, PB_ERR_BUSY, "request can never fit the server budget");
    Req *q = new (std::nothrow) Req();
    if (!q) return PB_ERR_OOM;
    q->r = *r;
    q->nsteps = r->kind == PB_REQ_GALERKIN ? 2 : 1;
    const double rowB = r->B.nrows > 0 ? (double)r->B.nnz / (double)r->B.nrows : 0.0;
    q->est = (double)r->A.nnz * std::max(rowB, 1.0) * q->nsteps;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->id = S->next_id++;
        S->reqs[q->id] = q;
        S->queue.push_back(q);
    }
    S->cv_work.notify_all();
    *req_id = q->id;
    return PB_OK;
}

pb_status pb_serve_poll(pb_server *S, uint64_t id, int32_t *done, pb_status *result) {
    if (!S || !done) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Req *q = find(S, id);
    if (!q) return PB_ERR_INVALID_ARG;
    *done = q->done ? 1 : 0;
    if (result) *result = q->done ? q->result : PB_OK;
    return PB_OK;
}

pb_status pb_serve_wait(pb_server *S, uint64_t id, pb_status *result) {
    if (!S) return PB_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    Req *q = find(S, id);
    if (!q) return PB_ERR_INVALID_ARG;
    S->cv_done.wait(lk, [&] { return q->done; });
    if (result) *result = q->result;
    return PB_OK;
}

pb_status pb_serve_result(pb_server *S, uint64_t id, pb_csr_out *C) {
    if (!S || !C) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Req *q = find(S, id);
    if (!q || !q->done || q->result != PB_OK) return PB_ERR_INVALID_ARG;
    const pb_request &r = q->r;
    std::memset(C, 0, sizeof(*C));
    C->nrows = r.kind == PB_REQ_GALERKIN ? r.B.ncols : r.A.nrows;
    C->ncols = r.B.ncols;
    C->cap = q->nnz;
    C->rowptr64 = static_cast<int64_t *>(q->out_rowptr.p);
    C->colidx = static_cast<int32_t *>(q->out_colidx.p);
    C->val = q->out_val.p;
    return PB_OK;
}

pb_status pb_serve_timing(pb_server *S, uint64_t id, double *queued_ms, double *total_ms) {
    if (!S) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Req *q = find(S, id);
    if (!q || !q->done) return PB_ERR_INVALID_ARG;
    using ms = std::chrono::duration<double, std::milli>;
    if (queued_ms) *queued_ms = q->admitted_once ? ms(q->t_first_admit - q->t_submit).count() : 0.0;
    if (total_ms) *total_ms = ms(q->t_done - q->t_submit).count();
    return PB_OK;
}

pb_status pb_serve_release(pb_server *S, uint64_t id) {
    if (!S) return PB_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        Req *q = find(S, id);
        if (!q || !q->done) {
            cudaSetDevice(prev);
            return PB_ERR_INVALID_ARG;
        }
        free_result(S, q);  // the slot that ran q no longer touches it once it is done
        S->reqs.erase(id);
        delete q;
    }
    cudaSetDevice(prev);
    S->cv_work.notify_all();
    return PB_OK;
}

pb_status pb_server_set_batching(pb_server *S, int32_t max_requests, double max_request_work) {
    if (!S || max_requests < 1 || max_requests > 4096 || !(max_request_work >= 0)) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->batch_max = max_requests;
    S->batch_work = max_request_work;
    return PB_OK;
}

pb_status pb_serve_batch_stats(pb_server *S, int64_t *requests, int64_t *launches) {
    if (!S) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (requests) *requests = S->batched_requests;
    if (launches) *launches = S->batch_launches;
    return PB_OK;
}

pb_status pb_serve_stats(pb_server *S, int64_t *completed, int64_t *preempted, size_t *bytes_in_use,
                         size_t *peak_bytes) {
    if (!S) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (completed) *completed = S->completed;
    if (preempted) *preempted = S->preempted;
    if (bytes_in_use) *bytes_in_use = S->in_use;
    if (peak_bytes) *peak_bytes = S->peak;
    return PB_OK;
}

}  // extern "C"
