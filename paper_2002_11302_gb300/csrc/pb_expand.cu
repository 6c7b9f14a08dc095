// Expand phase with propagation blocking (Alg. 2 expand loop, Sec. III-C).
//
// Alg. 2 walks column k of A (and row k of B), each (rowid, aval) of A(:,k)
// and each (colid, bval) of B(k,:), emitting (rowid, colid, aval*bval).  The
// tuples of one A entry form a run of nnz(B(k,:)) tuples, all for the same
// row, hence the same bin.
//
// Work split: expand work items are ranges of A entries (CSC order) holding
// about `chunk` tuples each (flop-balanced, so hub columns of skewed inputs
// spread over many warps); a persistent grid of warps takes them one at a
// time from a counter.  A warp takes 32 consecutive A entries at a time, one
// per lane, in a three-stage software pipeline: the entries of batch i + 2
// are loaded and the runs of batch i + 1 are reserved in their bins (one
// atomic on the bin's cursor per run) while batch i is written, so neither
// load nor atomic latency sits between a batch's B loads and its stores.
// Runs shorter than 32 tuples are written as one flattened stream: lane l of
// window w handles tuple 32w + l of the concatenated runs.  Its run is found
// without a search: one warp-wide OR-reduction per window marks the runs
// starting in the window, and the run is the number of runs started at or
// before the lane's tuple; the runs' descriptors (B offset, key high part,
// A value, bin position) sit in shared memory in that order.  Consecutive
// lanes thus load consecutive entries of B's rows and write consecutive slots
// of a run.  Several windows' B loads are issued together.  Runs of 32 or
// more tuples are written one at a time by the whole warp.
// Propagation blocking: tuple (i, j, a*b) goes to the bin holding row i (row
// ranges from the symbolic phase) as key = (i - first row of bin) << colbits | j
// and value a*b.  Reserving at a bin's cursor appends at the bin's frontier,
// so partially written sectors stay few and L2-resident until completed.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int LONG_RUN = 32;
constexpr int EXP_THREADS = 256;
constexpr int EXP_WARPS = EXP_THREADS / 32;
constexpr int64_t NO_POS = INT64_MIN;  // a run whose reservation failed: not written

#ifndef PB_EXPAND_U
#define PB_EXPAND_U 4  // 32-tuple windows whose B loads are issued together
#endif
#ifndef PB_EXPAND_MINB
#define PB_EXPAND_MINB 4  // resident blocks per SM the register budget must allow (64 registers, no spills)
#endif

#ifndef PB_EXPAND_PREFETCH
#define PB_EXPAND_PREFETCH 1  // L2 prefetch of the next batch's B rows
#endif

__device__ inline void prefetch_l2(const void *ptr) { asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr)); }

template <class TV, class IV>
__device__ inline TV tuple_product(IV a, IV b) {
    return static_cast<TV>(a * b);
}

template <class IV>
struct Entry {  // one A entry per lane
    uint64_t info;  // bin << 32 | key high part of the entry's row
    IV av;
    int32_t b0, lb;  // B(k,:) = [b0, b0 + lb); lb = 0: nothing to write
    int64_t apos;    // deterministic mode: the run's fixed first position
};

// The entry's three loads are independent and unconditional (the panel test
// comes after them), so a batch's loads are all in flight before any is used.
template <class IV, bool DET>
__device__ inline Entry<IV> load_entry(const NumericArgs &p, const IV *__restrict__ valA, int32_t e, bool valid) {
    Entry<IV> x;
    x.info = 0;
    x.av = IV(0);
    x.b0 = 0;
    x.lb = 0;
    x.apos = 0;
    if (valid) {
        x.info = p.ainfo[e];
        const int2 sp = p.aspan[e];
        x.av = valA[e];
        x.b0 = sp.x;
        x.lb = sp.y;
        if (DET) x.apos = p.apos[e];
    }
    return x;
}

// A run's reservation: the atomic on the bin's cursor and the bin's end are
// issued here; their values are first used one batch later (resolve), so the
// warp does not wait for the atomic's round trip.
struct Resv {
    int64_t pos;  // first absolute position (or the fixed one in deterministic mode)
    int64_t end;  // the bin's end: a run past it means the operands differ from the plan
};

template <class IV, bool DET>
__device__ inline Resv reserve_run(const NumericArgs &p, Entry<IV> &x) {
    Resv r{NO_POS, 0};
    const int64_t bin = (int64_t)(x.info >> 32);
    if (bin < p.bin_lo || bin >= p.bin_hi) x.lb = 0;  // the entry's row belongs to another panel
    if (x.lb <= 0) return r;
    if (DET) {
        r.pos = x.apos;
        r.end = INT64_MAX;
        return r;
    }
    r.pos = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&p.cursor[bin * p.cursor_stride]),
                               (unsigned long long)x.lb);
    r.end = p.bin_off[bin + 1];
    return r;
}

__device__ inline int64_t resolve(const NumericArgs &p, const Resv &r, int32_t lb) {
    if (r.pos == NO_POS) return NO_POS;
    if (r.pos + lb > r.end) {
        atomicOr(p.err, DEV_ERR_CAPACITY);
        return NO_POS;
    }
    return r.pos;
}

struct RunDesc {  // a short run of the flattened stream, indexed by run order
    int32_t boff;     // B index of the run's tuple t is boff + t (t: stream position)
    uint32_t keyhi;   // key high part (in-bin row << colbits)
    int64_t poff;     // bin position of tuple t is poff + t (NO_POS: not written)
};

// BATCH: the work items of all products of a batch, one product per item;
// A entries are indexed in the batch's global entry space and the operand
// arrays of the item's product are taken from its descriptor.
// DET: runs go to positions fixed in the plan (deterministic mode) instead of
// being reserved at the bins' cursors.
// PACK: 4-byte values written with their keys as one 8-byte pair per tuple
// (one store, half the scattered write requests of separate key and value arrays).
template <class TV>
__device__ inline uint2 packed_tuple(uint32_t key, TV v) {
    static_assert(sizeof(TV) == 4, "packed tuples hold 4-byte values");
    return make_uint2(key, __float_as_uint((float)v));
}

template <class IV, class TV, bool BATCH, bool DET, bool PACK>
__global__ void __launch_bounds__(EXP_THREADS, PB_EXPAND_MINB) k_expand(const NumericArgs p) {
    __shared__ RunDesc sdesc[EXP_WARPS][32];
    __shared__ IV sav[EXP_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    RunDesc *desc = sdesc[wid];
    IV *avs = sav[wid];
    const IV *__restrict__ valA = static_cast<const IV *>(p.valA);
    const IV *__restrict__ valB = static_cast<const IV *>(p.valB);
    const int32_t *__restrict__ colidxB = p.colidxB;
    // reserved positions are absolute tuple indices of the whole product; the
    // buffer holds this panel's tuples from tuple_base on
    uint32_t *__restrict__ keys = p.keys - p.tuple_base;
    TV *__restrict__ vals = static_cast<TV *>(p.vals) - p.tuple_base;
    uint2 *__restrict__ tup = reinterpret_cast<uint2 *>(p.keys) - p.tuple_base;  // PACK
    int64_t nchunks = p.nchunks;
    if constexpr (BATCH) {
        if (*p.err & DEV_ERR_BATCH_FATAL) return;
        nchunks = p.bhdr->nchunks;
    }
    const uint32_t le = lanemask_lt() | (1u << lane);

    while (true) {
        int64_t c = 0;
        if (lane == 0) c = (int64_t)atomicAdd(p.work, 1u);
        c = __shfl_sync(FULL, c, 0);
        if (c >= nchunks) break;
        int32_t e_begin = p.chunk_e[c], e_end = p.chunk_e[c + 1];
        if constexpr (BATCH) {
            const BatchDesc &d = p.desc[p.chunk_prod[c]];
            // global entry e of this product is its local entry e - estart
            valA = static_cast<const IV *>(d.valA) - d.estart;
            valB = static_cast<const IV *>(d.valB);
            colidxB = d.colidxB;
            const int32_t e_last = d.estart + d.nnzA;
            e_begin = min(e_begin, e_last);
            e_end = min(e_end, e_last);
        }
        // pipeline: cur is written, nxt is reserved, nx2 is loaded
        Entry<IV> cur = load_entry<IV, DET>(p, valA, e_begin + lane, e_begin + lane < e_end);
        Entry<IV> nxt = load_entry<IV, DET>(p, valA, e_begin + 32 + lane, e_begin + 32 + lane < e_end);
        Resv cur_r = reserve_run<IV, DET>(p, cur);
        for (int32_t e0 = e_begin; e0 < e_end; e0 += 32) {
            const int32_t e2 = e0 + 64 + lane;
            const Entry<IV> nx2 = load_entry<IV, DET>(p, valA, e2, e2 < e_end);
            const Resv nxt_r = reserve_run<IV, DET>(p, nxt);
            const int64_t cur_pos = resolve(p, cur_r, cur.lb);
#if PB_EXPAND_PREFETCH
            if (nxt.lb > 0) {  // the next batch's B rows into L2 while this batch is written
                prefetch_l2(colidxB + nxt.b0);
                prefetch_l2(colidxB + nxt.b0 + nxt.lb - 1);
                prefetch_l2(valB + nxt.b0);
                prefetch_l2(valB + nxt.b0 + nxt.lb - 1);
            }
#endif
            // ---- short runs of cur: descriptors in run order ----------------------------
            const bool is_long = cur.lb >= LONG_RUN;
            const int32_t sl = is_long ? 0 : cur.lb;
            const int32_t incl = warp_inclusive_scan(sl);
            const int32_t start = incl - sl;
            const int32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t nonempty = __ballot_sync(FULL, sl > 0);
            if (sl > 0) {
                const int k = __popc(nonempty & lanemask_lt());
                RunDesc d;
                d.boff = cur.b0 - start;
                d.keyhi = (uint32_t)cur.info;
                d.poff = cur_pos == NO_POS ? NO_POS : cur_pos - start;
                desc[k] = d;
                avs[k] = cur.av;
            }
            __syncwarp();
            int runs_before = 0;  // runs started before the current window
            for (int32_t t0 = 0; t0 < total; t0 += 32 * PB_EXPAND_U) {
                int r[PB_EXPAND_U];
#pragma unroll
                for (int u = 0; u < PB_EXPAND_U; ++u) {
                    const int32_t w0 = t0 + 32 * u;
                    const int32_t off = start - w0;
                    const uint32_t mine = (sl > 0 && off >= 0 && off < 32) ? (1u << off) : 0u;
                    const uint32_t starts = __reduce_or_sync(FULL, mine);  // runs starting in this window
                    r[u] = runs_before + __popc(starts & le) - 1;
                    runs_before += __popc(starts);
                }
                RunDesc d[PB_EXPAND_U];
#pragma unroll
                for (int u = 0; u < PB_EXPAND_U; ++u) d[u] = RunDesc{0, 0u, NO_POS};
                uint32_t col[PB_EXPAND_U];
                IV bv[PB_EXPAND_U];
#pragma unroll
                for (int u = 0; u < PB_EXPAND_U; ++u) {
                    const int32_t t = t0 + 32 * u + lane;
                    col[u] = 0;
                    bv[u] = IV(0);
                    if (t < total) {
                        d[u] = desc[r[u]];
                        col[u] = (uint32_t)colidxB[d[u].boff + t];
                        bv[u] = valB[d[u].boff + t];
                    }
                }
#pragma unroll
                for (int u = 0; u < PB_EXPAND_U; ++u) {
                    const int32_t t = t0 + 32 * u + lane;
                    if (t < total && d[u].poff != NO_POS) {
                        const TV v = tuple_product<TV, IV>(avs[r[u]], bv[u]);
                        if constexpr (PACK) {
                            tup[d[u].poff + t] = packed_tuple<TV>(d[u].keyhi | col[u], v);
                        } else {
                            keys[d[u].poff + t] = d[u].keyhi | col[u];
                            vals[d[u].poff + t] = v;
                        }
                    }
                }
            }
            // ---- long runs, one per warp step -------------------------------------------
            uint32_t lm = __ballot_sync(FULL, is_long);
            while (lm) {
                const int rl = __ffs(lm) - 1;
                lm &= lm - 1;
                const uint32_t keyhi = (uint32_t)__shfl_sync(FULL, cur.info, rl);
                const IV ar = __shfl_sync(FULL, cur.av, rl);
                const int32_t br = __shfl_sync(FULL, cur.b0, rl);
                const int32_t lr = __shfl_sync(FULL, cur.lb, rl);
                const int64_t pr = __shfl_sync(FULL, cur_pos, rl);
                if (pr == NO_POS) continue;
                for (int32_t ib = lane; ib < lr; ib += 32) {
                    const uint32_t key = keyhi | (uint32_t)colidxB[br + ib];
                    const TV v = tuple_product<TV, IV>(ar, valB[br + ib]);
                    if constexpr (PACK) {
                        tup[pr + ib] = packed_tuple<TV>(key, v);
                    } else {
                        keys[pr + ib] = key;
                        vals[pr + ib] = v;
                    }
                }
            }
            __syncwarp();  // the descriptors are rewritten by the next batch
            cur = nxt;
            cur_r = nxt_r;
            nxt = nx2;
        }
    }
}

template <class IV, class TV, bool BATCH, bool DET, bool PACK = false>
cudaError_t run_expand(const NumericArgs &a, cudaStream_t s) {
    auto kern = k_expand<IV, TV, BATCH, DET, PACK>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, EXP_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)a.num_sms * per_sm;  // one wave; work items are taken from a counter
    const int64_t need = ceil_div<int64_t>(a.nchunks, EXP_WARPS);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, EXP_THREADS, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <bool BATCH, bool DET>
cudaError_t dispatch_expand(const NumericArgs &a, cudaStream_t s) {
    switch (a.dtype) {
        case PB_F64: return run_expand<double, double, BATCH, DET>(a, s);
        case PB_F32: return run_expand<float, float, BATCH, DET>(a, s);
        case PB_F64_F32TUPLE: return run_expand<double, float, BATCH, DET>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_expand(const NumericArgs &a, cudaStream_t s) {
    if (a.flop <= 0) return cudaSuccess;
    if (a.packed) {
        switch (a.dtype) {
            case PB_F32: return run_expand<float, float, false, false, true>(a, s);
            case PB_F64_F32TUPLE: return run_expand<double, float, false, false, true>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    return a.apos ? dispatch_expand<false, true>(a, s) : dispatch_expand<false, false>(a, s);
}

// a.nchunks is an upper bound on the work items (it only sizes the grid).
cudaError_t launch_expand_batch(const NumericArgs &a, cudaStream_t s) { return dispatch_expand<true, false>(a, s); }

}  // namespace pb
