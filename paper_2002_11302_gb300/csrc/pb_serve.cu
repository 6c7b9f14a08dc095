// Serving loop with continuous batching over the PB-SpGEMM entry points.
//
// One worker thread drives `max_slots` CUDA streams.  A request is a short
// chain of products (one for C = A*B, two for the Galerkin product P^T (A P)),
// each run as: symbolic phase (Alg. 3; synchronises only the slot's stream),
// optionally a counting run (when a flop-sized C would take more than a quarter
// of the budget), then the numeric phase (Alg. 2).  The worker admits queued
// requests in arrival order while a slot is free and their memory fits the
// budget, and advances every admitted request when its stream's event fires, so
// requests arriving while others run on the GPU overlap with them.
//
// Every device byte the server holds (plans, workspaces, intermediates and
// results) comes from the server's own memory pool and is counted against the
// budget.  When all admitted requests wait for memory, the most recently
// admitted one is preempted (its memory released, the request queued again).
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

enum Phase { QUEUED, PLAN, MEM, COUNTING, RUNNING, DONE };

struct Req {
    uint64_t id = 0;
    pb_request r{};
    int step = 0, nsteps = 1;
    Phase phase = QUEUED;
    bool waiting = false;  // the last attempt to advance found too little memory
    bool counted = false;  // a counting run sized this step's output exactly
    pb_status result = PB_OK;
    int slot = -1;
    int restarts = 0;
    bool admitted_once = false;
    Clock::time_point t_submit, t_first_admit, t_admit, t_done;
    pb_plan *plan = nullptr;
    size_t plan_bytes = 0;   // reserved for the plan
    int64_t flop = 0, nnz = 0;
    Buf ws, nnz_dev;
    Buf out_rowptr, out_colidx, out_val;  // this step's C
    Buf prev_rowptr, prev_colidx, prev_val;  // the previous step's C (Galerkin: AP)
    int64_t prev_nnz = 0;
    cudaEvent_t ev = nullptr;
};

size_t val_bytes(int32_t dtype) { return dtype == PB_F32 ? 4 : 8; }

}  // namespace

struct pb_server {
    pb_handle *user = nullptr;
    pb_handle *h = nullptr;  // the worker's own handle (plans come from the server pool)
    int device = 0;
    cudaMemPool_t pool = nullptr;
    size_t budget = 0, in_use = 0, peak = 0;
    int max_slots = 0;
    std::vector<cudaStream_t> streams;
    std::vector<Req *> slots;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::vector<Buf> to_free;     // released results, freed by the worker
    std::vector<Req *> to_delete; // released requests: only the worker deletes requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t completed = 0, preempted = 0;
};

namespace {

// ---- budget -----------------------------------------------------------------
bool reserve(pb_server *S, size_t b) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->in_use + b > S->budget) return false;
    S->in_use += b;
    S->peak = std::max(S->peak, S->in_use);
    return true;
}

void force_reserve(pb_server *S, size_t b) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use += b;
    S->peak = std::max(S->peak, S->in_use);
}

void unreserve(pb_server *S, size_t b) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= std::min(b, S->in_use);
}

cudaStream_t stream_of(pb_server *S, const Req *q) { return S->streams[q->slot >= 0 ? q->slot : 0]; }

// Reserve and allocate; false when the budget has no room (nothing allocated).
bool get(pb_server *S, Req *q, Buf &b, size_t bytes, pb_status *err) {
    bytes = std::max<size_t>(bytes, 256);
    if (!reserve(S, bytes)) return false;
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, S->pool, stream_of(S, q)) != cudaSuccess) {
        (void)cudaGetLastError();
        unreserve(S, bytes);
        *err = PB_ERR_OOM;
        return true;
    }
    b.p = p;
    b.bytes = bytes;
    return true;
}

void put(pb_server *S, cudaStream_t s, Buf &b) {
    if (!b.p) return;
    (void)cudaFreeAsync(b.p, s);
    unreserve(S, b.bytes);
    b = Buf{};
}

// Allocator of the worker's handle: plan arrays from the server pool.  Plans
// are only destroyed after their stream's work has completed, so freeing on
// the first server stream is safe.
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

void pool_free(void *p, size_t, pb_stream_t stream, void *ctx) {
    pb_server *S = static_cast<pb_server *>(ctx);
    if (p) (void)cudaFreeAsync(p, stream ? reinterpret_cast<cudaStream_t>(stream) : S->streams[0]);
}

// ---- one product step ----------------------------------------------------------
struct Operands {
    pb_csc A;
    pb_csr B;
    bool intermediate;  // output feeds the next step (int32 row pointer)
};

Operands operands(const Req *q) {
    const pb_request &r = q->r;
    if (r.kind == PB_REQ_PRODUCT) return {r.A, r.B, false};
    if (q->step == 0) return {r.A, r.B, true};  // AP = A * P
    // P^T as CSC is P's CSR arrays read column-wise; AP is the previous step's C
    pb_csc Pt{r.B.ncols, r.B.nrows, r.B.nnz, r.B.rowptr, r.B.colidx, r.B.val};
    pb_csr AP{r.A.nrows, r.B.ncols, q->prev_nnz, static_cast<const int32_t *>(q->prev_rowptr.p),
              static_cast<const int32_t *>(q->prev_colidx.p), q->prev_val.p};
    return {Pt, AP, false};
}

// Upper estimate of a plan's device bytes, reserved while the plan is built.
size_t plan_estimate(const Operands &o) {
    const size_t m = (size_t)o.A.nrows, k = (size_t)o.A.ncols, e = (size_t)o.A.nnz;
    return 16 * (k + 2) + 96 * (m + 2) + 12 * e + (1u << 20);
}

void release_step(pb_server *S, Req *q) {
    cudaStream_t s = stream_of(S, q);
    put(S, s, q->ws);
    put(S, s, q->nnz_dev);
    if (q->plan) {
        pb_plan_destroy(q->plan);
        q->plan = nullptr;
    }
    unreserve(S, q->plan_bytes);
    q->plan_bytes = 0;
}

void release_all(pb_server *S, Req *q) {
    cudaStream_t s = stream_of(S, q);
    release_step(S, q);
    put(S, s, q->out_rowptr);
    put(S, s, q->out_colidx);
    put(S, s, q->out_val);
    put(S, s, q->prev_rowptr);
    put(S, s, q->prev_colidx);
    put(S, s, q->prev_val);
}

void finish(pb_server *S, Req *q, pb_status st) {
    q->result = st;
    if (st != PB_OK) {
        release_all(S, q);
    } else {
        release_step(S, q);
        cudaStream_t s = stream_of(S, q);
        put(S, s, q->prev_rowptr);
        put(S, s, q->prev_colidx);
        put(S, s, q->prev_val);
    }
    q->t_done = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    q->phase = DONE;
    q->waiting = false;
    if (q->slot >= 0) S->slots[q->slot] = nullptr;
    q->slot = -1;
    ++S->completed;
    S->cv_done.notify_all();
}

// Advance a request by one action.  Returns false when it must wait for memory.
bool advance(pb_server *S, Req *q) {
    cudaStream_t s = stream_of(S, q);
    const int32_t dtype = q->r.dtype;
    const size_t vb = val_bytes(dtype);
    pb_status err = PB_OK;
    for (;;) {
        switch (q->phase) {
            case PLAN: {
                const Operands o = operands(q);
                const size_t est = plan_estimate(o);
                if (est > S->budget) {
                    finish(S, q, PB_ERR_BUSY);
                    return true;
                }
                if (!reserve(S, est)) return false;
                pb_config cfg{};
                cfg.max_tuple_bytes = (int64_t)(S->budget / 4);  // larger products run in row panels
                pb_status st = pb_spgemm_symbolic(S->h, &o.A, &o.B, (pb_dtype)dtype, &cfg,
                                                  reinterpret_cast<pb_stream_t>(s), &q->plan);
                unreserve(S, est);
                if (st != PB_OK) {
                    q->plan = nullptr;
                    finish(S, q, st);
                    return true;
                }
                q->plan_bytes = plan_device_bytes(q->plan);
                force_reserve(S, q->plan_bytes);
                pb_plan_query(q->plan, &q->flop, nullptr, nullptr, nullptr, nullptr);
                q->counted = false;
                q->phase = MEM;
                break;
            }
            case MEM: {
                size_t ws_bytes = 0;
                pb_plan_query(q->plan, nullptr, nullptr, &ws_bytes, nullptr, nullptr);
                const Operands o = operands(q);
                const size_t m = (size_t)o.A.nrows;
                const size_t rp = o.intermediate ? 4 : 8;
                const int64_t cap = q->counted ? q->nnz : q->flop;
                const size_t out_bytes = rp * (m + 1) + (size_t)std::max<int64_t>(cap, 1) * (4 + vb);
                const size_t held_other = q->prev_rowptr.bytes + q->prev_colidx.bytes + q->prev_val.bytes;
                if (!q->counted && out_bytes > S->budget / 4) {
                    // size C exactly first: a counting run needs only the workspace
                    if (q->plan_bytes + held_other + ws_bytes + 256 > S->budget) {
                        finish(S, q, PB_ERR_BUSY);
                        return true;
                    }
                    if (!q->ws.p && !get(S, q, q->ws, ws_bytes, &err)) return false;
                    if (!q->nnz_dev.p && err == PB_OK && !get(S, q, q->nnz_dev, 8, &err)) return false;
                    if (err != PB_OK) {
                        finish(S, q, err);
                        return true;
                    }
                    pb_csr_out C{o.A.nrows, o.B.ncols, 0, nullptr, nullptr, nullptr, nullptr,
                                 static_cast<int64_t *>(q->nnz_dev.p)};
                    pb_status st = pb_spgemm_numeric(S->h, q->plan, &o.A, &o.B, &C, q->ws.p, q->ws.bytes,
                                                     reinterpret_cast<pb_stream_t>(s));
                    if (st == PB_OK && cudaEventRecord(q->ev, s) != cudaSuccess) st = PB_ERR_CUDA;
                    if (st != PB_OK) {
                        finish(S, q, st);
                        return true;
                    }
                    q->phase = COUNTING;
                    return true;
                }
                if (q->plan_bytes + held_other + ws_bytes + out_bytes + 256 > S->budget) {
                    finish(S, q, PB_ERR_BUSY);
                    return true;
                }
                // all or nothing: what this step still lacks must fit together
                const size_t lack = (q->ws.p ? 0 : std::max<size_t>(ws_bytes, 256)) + (q->nnz_dev.p ? 0 : 256) +
                                    std::max<size_t>(rp * (m + 1), 256) +
                                    std::max<size_t>((size_t)std::max<int64_t>(cap, 1) * 4, 256) +
                                    std::max<size_t>((size_t)std::max<int64_t>(cap, 1) * vb, 256);
                if (!reserve(S, lack)) return false;
                unreserve(S, lack);
                if (!q->ws.p) get(S, q, q->ws, ws_bytes, &err);
                if (err == PB_OK && !q->nnz_dev.p) get(S, q, q->nnz_dev, 8, &err);
                if (err == PB_OK) get(S, q, q->out_rowptr, rp * (m + 1), &err);
                if (err == PB_OK) get(S, q, q->out_colidx, (size_t)std::max<int64_t>(cap, 1) * 4, &err);
                if (err == PB_OK) get(S, q, q->out_val, (size_t)std::max<int64_t>(cap, 1) * vb, &err);
                if (err != PB_OK || !q->out_val.p) {
                    finish(S, q, err != PB_OK ? err : PB_ERR_OOM);
                    return true;
                }
                pb_csr_out C{o.A.nrows, o.B.ncols, cap,
                             o.intermediate ? nullptr : static_cast<int64_t *>(q->out_rowptr.p),
                             o.intermediate ? static_cast<int32_t *>(q->out_rowptr.p) : nullptr,
                             static_cast<int32_t *>(q->out_colidx.p), q->out_val.p,
                             static_cast<int64_t *>(q->nnz_dev.p)};
                pb_status st = pb_spgemm_numeric(S->h, q->plan, &o.A, &o.B, &C, q->ws.p, q->ws.bytes,
                                                 reinterpret_cast<pb_stream_t>(s));
                if (st == PB_OK && cudaEventRecord(q->ev, s) != cudaSuccess) st = PB_ERR_CUDA;
                if (st != PB_OK) {
                    finish(S, q, st);
                    return true;
                }
                q->phase = RUNNING;
                return true;
            }
            case COUNTING:
            case RUNNING: {
                // the step's event has fired: read its device status and nnz(C)
                pb_status dev = PB_OK;
                pb_status st = pb_plan_status(q->plan, reinterpret_cast<pb_stream_t>(s), &dev);
                int64_t nnz = 0;
                if (st == PB_OK && cudaMemcpy(&nnz, q->nnz_dev.p, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                    st = PB_ERR_CUDA;
                if (st == PB_OK) st = dev;
                if (st != PB_OK) {
                    finish(S, q, st);
                    return true;
                }
                q->nnz = nnz;
                if (q->phase == COUNTING) {
                    q->counted = true;
                    q->phase = MEM;
                    break;
                }
                const bool intermediate = operands(q).intermediate;
                release_step(S, q);
                if (intermediate) {
                    // keep this step's C as the next step's B; drop the step before it
                    put(S, s, q->prev_rowptr);
                    put(S, s, q->prev_colidx);
                    put(S, s, q->prev_val);
                    q->prev_rowptr = q->out_rowptr;
                    q->prev_colidx = q->out_colidx;
                    q->prev_val = q->out_val;
                    q->prev_nnz = nnz;
                    q->out_rowptr = q->out_colidx = q->out_val = Buf{};
                }
                if (++q->step < q->nsteps) {
                    q->phase = PLAN;
                    break;
                }
                finish(S, q, PB_OK);
                return true;
            }
            default:
                return true;
        }
    }
}

void preempt(pb_server *S, Req *q) {
    release_all(S, q);
    std::lock_guard<std::mutex> lk(S->mu);
    if (q->slot >= 0) S->slots[q->slot] = nullptr;
    q->slot = -1;
    q->step = 0;
    q->phase = QUEUED;
    q->waiting = false;
    q->counted = false;
    q->prev_nnz = 0;
    ++q->restarts;
    ++S->preempted;
    S->queue.push_front(q);
}

void worker_main(pb_server *S) {
    (void)cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        // results and requests released by callers (no request is referenced here)
        if (!S->to_free.empty() || !S->to_delete.empty()) {
            std::vector<Buf> fr;
            std::vector<Req *> dl;
            fr.swap(S->to_free);
            dl.swap(S->to_delete);
            lk.unlock();
            for (Buf &b : fr) (void)cudaFreeAsync(b.p, S->streams[0]);
            for (Req *q : dl) {
                if (q->ev) (void)cudaEventDestroy(q->ev);
                delete q;
            }
            lk.lock();
            progress = true;
        }
        // admitted requests: completed events and retries after waiting for memory
        for (int i = 0; i < S->max_slots; ++i) {
            Req *q = S->slots[i];
            if (!q) continue;
            if (q->phase == COUNTING || q->phase == RUNNING) {
                lk.unlock();
                const cudaError_t e = cudaEventQuery(q->ev);
                bool fired = e == cudaSuccess;
                if (e != cudaSuccess && e != cudaErrorNotReady) {
                    (void)cudaGetLastError();
                    finish(S, q, PB_ERR_CUDA);
                    fired = false;
                    progress = true;
                }
                if (fired) {
                    advance(S, q);
                    progress = true;
                }
                lk.lock();
            } else if (q->phase == PLAN || q->phase == MEM) {
                lk.unlock();
                const bool moved = advance(S, q);
                lk.lock();
                q->waiting = !moved && q->phase != DONE;
                progress |= moved;
            }
        }
        // preemption: every admitted request waits for memory
        int active = 0, waiting = 0;
        Req *youngest = nullptr;
        for (Req *q : S->slots) {
            if (!q) continue;
            ++active;
            if (q->waiting) {
                ++waiting;
                if (!youngest || q->t_admit > youngest->t_admit) youngest = q;
            }
        }
        if (active >= 2 && waiting == active) {
            lk.unlock();
            preempt(S, youngest);
            lk.lock();
            progress = true;
            continue;
        }
        // admissions, in arrival order, while nobody waits for memory
        while (waiting == 0 && !S->queue.empty()) {
            int free_slot = -1;
            for (int i = 0; i < S->max_slots; ++i)
                if (!S->slots[i]) {
                    free_slot = i;
                    break;
                }
            if (free_slot < 0) break;
            Req *q = S->queue.front();
            S->queue.pop_front();
            S->slots[free_slot] = q;
            q->slot = free_slot;
            q->phase = PLAN;
            q->t_admit = Clock::now();
            if (!q->admitted_once) {
                q->admitted_once = true;
                q->t_first_admit = q->t_admit;
            }
            lk.unlock();
            const bool moved = advance(S, q);
            lk.lock();
            q->waiting = !moved && q->phase != DONE;
            if (q->waiting) waiting = 1;
            progress = true;
        }
        bool busy = !S->queue.empty();
        for (Req *q : S->slots) busy |= q != nullptr;
        if (S->stop && !busy && S->to_free.empty() && S->to_delete.empty()) break;
        if (!progress) S->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
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
    for (int i = 0; e == cudaSuccess && i < max_slots; ++i) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) S->streams.push_back(s);
    }
    pb_status st = PB_OK;
    if (e == cudaSuccess) st = pb_create(&S->h);
    if (e == cudaSuccess && st == PB_OK) st = pb_set_allocator(S->h, pool_alloc, pool_free, S);
    cudaSetDevice(prev);
    if (e != cudaSuccess || st != PB_OK) {
        for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
        if (S->pool) cudaMemPoolDestroy(S->pool);
        if (S->h) pb_destroy(S->h);
        delete S;
        if (e != cudaSuccess) return host_cuda_fail(h, e, "pb_server_create");
        return st;
    }
    S->slots.assign(max_slots, nullptr);
    S->worker = std::thread(worker_main, S);
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
    S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto &kv : S->reqs) {
        Req *q = kv.second;
        for (Buf *b : {&q->out_rowptr, &q->out_colidx, &q->out_val})
            if (b->p) cudaFreeAsync(b->p, S->streams[0]);
        if (q->ev) cudaEventDestroy(q->ev);
        delete q;
    }
    for (cudaStream_t s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    pb_destroy(S->h);
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
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    cudaError_t e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        delete q;
        return host_cuda_fail(S->user, e, "pb_serve_submit");
    }
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
    *done = q->phase == DONE ? 1 : 0;
    if (result) *result = q->phase == DONE ? q->result : PB_OK;
    return PB_OK;
}

pb_status pb_serve_wait(pb_server *S, uint64_t id, pb_status *result) {
    if (!S) return PB_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    Req *q = find(S, id);
    if (!q) return PB_ERR_INVALID_ARG;
    S->cv_done.wait(lk, [&] { return q->phase == DONE; });
    if (result) *result = q->result;
    return PB_OK;
}

pb_status pb_serve_result(pb_server *S, uint64_t id, pb_csr_out *C) {
    if (!S || !C) return PB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Req *q = find(S, id);
    if (!q || q->phase != DONE || q->result != PB_OK) return PB_ERR_INVALID_ARG;
    const pb_request &r = q->r;
    const int32_t nrows = r.kind == PB_REQ_GALERKIN ? r.B.ncols : r.A.nrows;
    std::memset(C, 0, sizeof(*C));
    C->nrows = nrows;
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
    if (!q || q->phase != DONE) return PB_ERR_INVALID_ARG;
    using ms = std::chrono::duration<double, std::milli>;
    if (queued_ms) *queued_ms = q->admitted_once ? ms(q->t_first_admit - q->t_submit).count() : 0.0;
    if (total_ms) *total_ms = ms(q->t_done - q->t_submit).count();
    return PB_OK;
}

pb_status pb_serve_release(pb_server *S, uint64_t id) {
    if (!S) return PB_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        Req *q = find(S, id);
        if (!q || q->phase != DONE) return PB_ERR_INVALID_ARG;
        for (Buf *b : {&q->out_rowptr, &q->out_colidx, &q->out_val})
            if (b->p) {
                S->to_free.push_back(*b);
                S->in_use -= std::min(b->bytes, S->in_use);
            }
        S->reqs.erase(id);
        S->to_delete.push_back(q);
    }
    S->cv_work.notify_all();
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
