// Expand phase with propagation blocking (Alg. 2 expand loop, Sec. III-C).
//
// Alg. 2 walks column k of A (and row k of B), each (rowid, aval) of A(:,k)
// and each (colid, bval) of B(k,:), emitting (rowid, colid, aval*bval).  The
// tuples of one A entry form a run of nnz(B(k,:)) tuples, all for the same
// row, hence the same bin.
//
// Work split: expand work items are ranges of A entries (CSC order) holding
// about `chunk` tuples each (flop-balanced, so hub columns of skewed inputs
// spread over many warps).  A warp takes 32 consecutive A entries at a time,
// one per lane:
//   1. each lane loads its entry's column, bin info and value and the extent
//      of B(k,:), then reserves its whole run in its bin with one atomic on
//      the bin's cursor (32 independent reservations in flight per warp);
//   2. runs shorter than 32 tuples are written as one flattened stream: lane
//      l of step s handles tuple 32s + l of the concatenated runs, found by a
//      shuffle search over the runs' prefix sums, so consecutive lanes write
//      consecutive slots of the same run;
//   3. runs of 32 or more tuples are written one at a time by the whole warp.
// Propagation blocking: tuple (i, j, a*b) goes to the bin holding row i (row
// ranges from the symbolic phase) as key = (i - first row of bin) << colbits | j
// and value a*b.  Reserving at a bin's cursor appends at the bin's frontier,
// so partially written sectors stay few and L2-resident until completed.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int LONG_RUN = 32;

template <class TV, class IV>
__device__ inline TV tuple_product(IV a, IV b) {
    return static_cast<TV>(a * b);
}

// Reserve `len` slots of `bin`; returns the first absolute position or -1.
__device__ inline int64_t reserve(const NumericArgs &p, uint32_t bin, uint32_t len) {
    const int64_t pos = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&p.cursor[bin]),
                                           (unsigned long long)len);
    if (pos + len > p.bin_off[bin + 1]) {  // operands differ from the plan's structure
        atomicOr(p.err, DEV_ERR_CAPACITY);
        return -1;
    }
    return pos;
}

template <class IV>
struct Batch {  // one A entry per lane
    uint64_t info;
    IV av;
    int32_t b0, lb;
    int64_t apos;  // deterministic mode: the run's fixed first position
};

template <class IV, bool DET>
__device__ inline Batch<IV> load_batch(const NumericArgs &p, const IV *__restrict__ valA,
                                      const int32_t *__restrict__ rowptrB, int32_t e, bool valid) {
    Batch<IV> x;
    x.info = 0;
    x.av = IV(0);
    x.b0 = 0;
    x.lb = 0;
    x.apos = 0;
    if (valid) {
        const int32_t k = p.acol[e];
        x.info = p.ainfo[e];
        const int64_t bin = (int64_t)(x.info >> 32);
        if (bin >= p.bin_lo && bin < p.bin_hi) {  // the entry's row belongs to this panel
            x.av = valA[e];
            x.b0 = rowptrB[k];
            x.lb = rowptrB[k + 1] - x.b0;
            if (DET) x.apos = p.apos[e];
        }
    }
    return x;
}

#ifndef PB_EXPAND_U
#define PB_EXPAND_U 1  // 32-tuple steps whose B loads are issued together
#endif
#ifndef PB_EXPAND_MINB
#define PB_EXPAND_MINB 5  // resident blocks per SM the register budget must allow (measured best on GB300)
#endif

// BATCH: the work items of all products of a batch, one product per item;
// A entries are indexed in the batch's global entry space and the operand
// arrays of the item's product are taken from its descriptor.
// DET: runs go to positions fixed in the plan (deterministic mode) instead of
// being reserved at the bins' cursors.
template <class IV, class TV, bool BATCH, bool DET>
__global__ void __launch_bounds__(256, PB_EXPAND_MINB) k_expand(const NumericArgs p) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const IV *__restrict__ valA = static_cast<const IV *>(p.valA);
    const IV *__restrict__ valB = static_cast<const IV *>(p.valB);
    const int32_t *__restrict__ colidxB = p.colidxB;
    const int32_t *__restrict__ rowptrB = p.rowptrB;
    // reserved positions are absolute tuple indices of the whole product; the
    // buffer holds this panel's tuples from tuple_base on
    uint32_t *__restrict__ keys = p.keys - p.tuple_base;
    TV *__restrict__ vals = static_cast<TV *>(p.vals) - p.tuple_base;
    int64_t nchunks = p.nchunks;
    if constexpr (BATCH) {
        if (*p.err & DEV_ERR_BATCH_FATAL) return;
        nchunks = p.bhdr->nchunks;
    }

    for (int64_t c = gwarp; c < nchunks; c += nwarps) {
        int32_t e_begin = p.chunk_e[c], e_end = p.chunk_e[c + 1];
        if constexpr (BATCH) {
            const BatchDesc &d = p.desc[p.chunk_prod[c]];
            // global entry e of this product is its local entry e - estart
            valA = static_cast<const IV *>(d.valA) - d.estart;
            valB = static_cast<const IV *>(d.valB);
            colidxB = d.colidxB;
            rowptrB = d.rowptrB;
            const int32_t e_last = d.estart + d.nnzA;
            e_begin = min(e_begin, e_last);
            e_end = min(e_end, e_last);
        }
        Batch<IV> cur = load_batch<IV, DET>(p, valA, rowptrB, e_begin + lane, e_begin + lane < e_end);
        for (int32_t e0 = e_begin; e0 < e_end; e0 += 32) {
            const bool valid = e0 + lane < e_end;
            const bool is_long = cur.lb >= LONG_RUN;
            const int32_t sl = is_long ? 0 : cur.lb;
            int64_t pos = -1;
            if (sl > 0) pos = DET ? cur.apos : reserve(p, (uint32_t)(cur.info >> 32), (uint32_t)sl);
            // software pipeline: the next batch's loads overlap this batch's reservations and writes
            const int32_t en = e0 + 32 + lane;
            const Batch<IV> nxt = load_batch<IV, DET>(p, valA, rowptrB, en, en < e_end);
            // ---- short runs as one flattened stream --------------------------------
            const int32_t incl = warp_inclusive_scan(sl);
            const int32_t total = __shfl_sync(FULL, incl, 31);
            // Steps of 32 tuples in groups of PB_EXPAND_U: the B loads of a group
            // are all issued before any of its stores, so their latencies overlap.
            for (int32_t t0 = 0; t0 < total; t0 += 32 * PB_EXPAND_U) {
                uint32_t col[PB_EXPAND_U];
                IV bv[PB_EXPAND_U];
                int rr[PB_EXPAND_U];
                int32_t ibs[PB_EXPAND_U];
#pragma unroll
                for (int u = 0; u < PB_EXPAND_U; ++u) {
                    const int32_t t = t0 + 32 * u + lane;
                    int r = 0;  // the run holding tuple t: number of runs ending at or before t
#pragma unroll
                    for (int s = 16; s >= 1; s >>= 1)
                        if (__shfl_sync(FULL, incl, r + s - 1) <= t) r += s;
                    const int32_t ib = t - (__shfl_sync(FULL, incl, r) - __shfl_sync(FULL, sl, r));
                    const int32_t br = __shfl_sync(FULL, cur.b0, r);
                    col[u] = 0;
                    bv[u] = IV(0);
                    if (t < total) {
                        col[u] = (uint32_t)colidxB[br + ib];
                        bv[u] = valB[br + ib];
                    }
                    rr[u] = r;
                    ibs[u] = ib;
                }
#pragma unroll
                for (int u = 0; u < PB_EXPAND_U; ++u) {
                    const int32_t t = t0 + 32 * u + lane;
                    const int r = rr[u];
                    const uint32_t keyhi = (uint32_t)__shfl_sync(FULL, (uint32_t)cur.info, r);
                    const IV ar = __shfl_sync(FULL, cur.av, r);
                    const int64_t pr = __shfl_sync(FULL, pos, r);
                    if (t < total && pr >= 0) {
                        keys[pr + ibs[u]] = keyhi | col[u];
                        vals[pr + ibs[u]] = tuple_product<TV, IV>(ar, bv[u]);
                    }
                }
            }
            // ---- long runs, one per warp step -------------------------------------
            uint32_t lm = __ballot_sync(FULL, valid && is_long);
            while (lm) {
                const int r = __ffs(lm) - 1;
                lm &= lm - 1;
                const uint64_t ir = __shfl_sync(FULL, cur.info, r);
                const IV ar = __shfl_sync(FULL, cur.av, r);
                const int32_t br = __shfl_sync(FULL, cur.b0, r);
                const int32_t lr = __shfl_sync(FULL, cur.lb, r);
                int64_t pr = 0;
                if (DET) {
                    pr = __shfl_sync(FULL, cur.apos, r);
                } else {
                    if (lane == 0) pr = reserve(p, (uint32_t)(ir >> 32), (uint32_t)lr);
                    pr = __shfl_sync(FULL, pr, 0);
                }
                if (pr < 0) continue;
                const uint32_t keyhi = (uint32_t)ir;
                for (int32_t ib = lane; ib < lr; ib += 32) {
                    keys[pr + ib] = keyhi | (uint32_t)colidxB[br + ib];
                    vals[pr + ib] = tuple_product<TV, IV>(ar, valB[br + ib]);
                }
            }
            cur = nxt;
        }
    }
}

}  // namespace

cudaError_t launch_expand(const NumericArgs &a, cudaStream_t s) {
    if (a.flop <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (int64_t)a.num_sms * 8;
    const int64_t need = ceil_div<int64_t>(a.nchunks * 32, threads);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    const unsigned b = (unsigned)blocks;
    if (a.apos) {
        switch (a.dtype) {
            case PB_F64: k_expand<double, double, false, true><<<b, threads, 0, s>>>(a); break;
            case PB_F32: k_expand<float, float, false, true><<<b, threads, 0, s>>>(a); break;
            case PB_F64_F32TUPLE: k_expand<double, float, false, true><<<b, threads, 0, s>>>(a); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (a.dtype) {
            case PB_F64: k_expand<double, double, false, false><<<b, threads, 0, s>>>(a); break;
            case PB_F32: k_expand<float, float, false, false><<<b, threads, 0, s>>>(a); break;
            case PB_F64_F32TUPLE: k_expand<double, float, false, false><<<b, threads, 0, s>>>(a); break;
            default: return cudaErrorInvalidValue;
        }
    }
    count_launches(1);
    return cudaGetLastError();
}

// a.nchunks is an upper bound on the work items (it only sizes the grid).
cudaError_t launch_expand_batch(const NumericArgs &a, cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (int64_t)a.num_sms * 8;
    const int64_t need = ceil_div<int64_t>(a.nchunks * 32, threads);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    switch (a.dtype) {
        case PB_F64: k_expand<double, double, true, false><<<(unsigned)blocks, threads, 0, s>>>(a); break;
        case PB_F32: k_expand<float, float, true, false><<<(unsigned)blocks, threads, 0, s>>>(a); break;
        case PB_F64_F32TUPLE: k_expand<double, float, true, false><<<(unsigned)blocks, threads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pb
