// Sort, compress and ConvertCSR of Alg. 2, one bin per CTA pass.
//
// For each bin (a range of consecutive rows, Sec. III-A/III-D):
//   load     the bin's keys and values with two bulk global->shared copies
//            (the bin is read from DRAM exactly once: "in-cache sorting",
//            Sec. III-D, with shared memory playing the cache);
//   sort     by the packed (in-bin row, column) key (Sec. III-D).  A bucket
//            pass on the top bits of (key - min key) with shared-memory atomic
//            counters places every tuple in its bucket.  When no bucket holds
//            more than SMALL_BUCKET tuples (the common case for ER-like
//            inputs), each thread owns a contiguous run of buckets and
//            finishes them by insertion sort.  Otherwise a stable LSD radix
//            sort over 8-bit digits (warp-level multisplit ranking with
//            ballots) sorts the whole bin.  Both give ascending keys; equal
//            keys are merged next, so their relative order does not matter;
//   compress equal adjacent keys are summed (Sec. III-E: one pass over the
//            sorted tuples; sums accumulate in double);
//   ConvertCSR the bins are concatenated in row order: the bin's number of
//            merged entries is published and the exclusive prefix over all
//            earlier bins is found by a warp-parallel decoupled look-back
//            (bins are taken in increasing order through a ticket counter, so
//            every bin a CTA waits for is owned by a running CTA); then the
//            column indices, values and row pointers of the bin are written.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int RMAX = 1 << RMAX_LOG2;  // max rows of one bin (symbolic cuts bins at multiples of this)
constexpr int SMALL_BUCKET = 32;

// Bucket-offset scan: 1 = contiguous per-thread runs with vector accesses
// (measured faster on GB300), 0 = lane-striped runs with warp shuffles.
#ifndef PB_SORT_VSCAN
#define PB_SORT_VSCAN 1
#endif

// Output of the bin being processed, for batched products (the product's C).
struct BinOut {
    int64_t *rowptr64;
    int32_t *rowptr32;
    int32_t *colidx;
    void *valC;
    int64_t *nnz_dev;
    int64_t cap;
    int64_t first;   // the product's first bin: its look-back chain starts there
    int32_t rbase;   // global row of the product's row 0
    int32_t m;
    int32_t colbits;
    int32_t last;    // the product's last bin
};

template <int CAP, int THREADS, class TV>
struct SortSmem {
    static constexpr int NW = THREADS / 32;
    static constexpr int CNTN = (CAP + 4 > 256 * NW) ? CAP + 4 : 256 * NW;
    uint32_t kin[CAP];
    TV vin[CAP];
    uint32_t skey[CAP];
    uint16_t sidx[CAP];
    uint16_t sidx2[CAP];
    uint32_t cnt[CNTN];     // bucket counters / offsets, LSD digit counters
    uint32_t rowcnt[RMAX];  // merged entries per in-bin row
    int64_t scratch[40];
    uint32_t wtot[NW];      // merged entries per warp segment
    int32_t marks[2];       // look-back: nearest inclusive prefix / unpublished bin
    uint64_t bar;
    int64_t bin;
    int64_t prefix;
    uint32_t big;
    int32_t ok;
    BinOut out;
};

__device__ inline void write_rowptr(const NumericArgs &p, int64_t row, int64_t v) {
    if (p.rowptr64)
        p.rowptr64[row] = v;
    else
        p.rowptr32[row] = (int32_t)v;
}

__device__ inline void write_rowptr(const BinOut &o, int64_t row, int64_t v) {
    if (o.rowptr64)
        o.rowptr64[row] = v;
    else
        o.rowptr32[row] = (int32_t)v;
}

// Exclusive scan in place of cnt[0..n), blocked per thread; all threads.
template <int THREADS>
__device__ inline void smem_exclusive_scan(uint32_t *cnt, int n, int64_t *scratch) {
    const int per = (n + THREADS - 1) / THREADS;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, n);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    int64_t total;
    int64_t pre = block_exclusive_scan<int64_t, THREADS>((int64_t)s, scratch, &total);
    uint32_t run = (uint32_t)pre;
    for (int i = lo; i < hi; ++i) {
        uint32_t c = cnt[i];
        cnt[i] = run;
        run += c;
    }
    __syncthreads();
}

// Exclusive scan in place of cnt[0..n) with n = NW * 32 * V: warp w owns the
// contiguous segment [w*32V, (w+1)*32V), loads it lane-striped (conflict-free,
// all V loads in flight), scans the V rows with interleaved warp scans, then
// the warp totals are combined.
template <int THREADS, int V>
__device__ inline void smem_exclusive_scan_striped(uint32_t *cnt, int64_t *scratch) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *seg = cnt + warp * 32 * V;
    uint32_t v[V], inc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] = seg[j * 32 + lane];
#pragma unroll
    for (int j = 0; j < V; ++j) inc[j] = v[j];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const uint32_t t = __shfl_up_sync(FULL, inc[j], o);
            if (lane >= o) inc[j] += t;
        }
    }
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const uint32_t tot = __shfl_sync(FULL, inc[j], 31);
        v[j] = run + inc[j] - v[j];
        run += tot;
    }
    uint32_t *wsum = reinterpret_cast<uint32_t *>(scratch);
    if (lane == 0) wsum[warp] = run;
    __syncthreads();
    uint32_t base = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) base += (w < warp) ? wsum[w] : 0u;
#pragma unroll
    for (int j = 0; j < V; ++j) seg[j * 32 + lane] = v[j] + base;
    __syncthreads();
}

// Exclusive scan in place of cnt[0..THREADS*V): thread t owns the contiguous
// run [t*V, (t+1)*V), read and written with 16-byte vector accesses.
template <int THREADS, int V>
__device__ inline void smem_exclusive_scan_runs(uint32_t *cnt, int64_t *scratch) {
    static_assert(V % 4 == 0, "runs of whole uint4");
    uint4 *run = reinterpret_cast<uint4 *>(cnt + threadIdx.x * V);
    uint4 v[V / 4];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < V / 4; ++j) {
        v[j] = run[j];
        s += v[j].x + v[j].y + v[j].z + v[j].w;
    }
    int64_t total;
    uint32_t pre = (uint32_t)block_exclusive_scan<int64_t, THREADS>((int64_t)s, scratch, &total);
#pragma unroll
    for (int j = 0; j < V / 4; ++j) {
        uint4 o;
        o.x = pre;
        pre += v[j].x;
        o.y = pre;
        pre += v[j].y;
        o.z = pre;
        pre += v[j].z;
        o.w = pre;
        pre += v[j].w;
        run[j] = o;
    }
    __syncthreads();
}

__device__ inline uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Decoupled look-back, executed by one full warp.  Lane i inspects bin j - i,
// so each poll covers 32 predecessors.  Returns the exclusive prefix.
__device__ inline int64_t lookback_warp(uint64_t *status, int64_t b, uint64_t agg, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    if (b == 0) {
        if (lane == 0) st_release_u64(&status[0], LB_PREFIX | agg);
        return 0;
    }
    if (lane == 0) st_release_u64(&status[b], LB_AGGREGATE | agg);
    uint64_t prefix = 0;
    int64_t j = b - 1;
    bool timed_out = false;
    while (true) {
        const int64_t idx = j - lane;
        uint64_t v = LB_PREFIX;  // before bin 0 the prefix is 0
        if (idx >= 0) {
            uint32_t spins = 0;
            while (true) {
                v = ld_acquire_u64(&status[idx]);
                if (v >> LB_FLAG_SHIFT) break;
                if (++spins > SPIN_LIMIT) {
                    timed_out = true;
                    v = LB_PREFIX;  // give up: treat as prefix 0 so the chain keeps moving
                    break;
                }
                __nanosleep(32);
            }
        }
        const uint32_t pmask = __ballot_sync(FULL, (v & ~LB_VALUE_MASK) == LB_PREFIX);
        if (pmask) {
            const int first = __ffs(pmask) - 1;  // closest predecessor holding an inclusive prefix
            prefix += warp_sum_u64(lane <= first ? (v & LB_VALUE_MASK) : 0ull);
            break;
        }
        prefix += warp_sum_u64(v & LB_VALUE_MASK);
        j -= 32;
    }
    if (__any_sync(FULL, timed_out) && lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
    if (lane == 0) st_release_u64(&status[b], LB_PREFIX | (prefix + agg));
    return (int64_t)prefix;
}

// Decoupled look-back by the whole CTA: thread t inspects bin j - t, so one
// round covers THREADS predecessors.  A round is accepted when every bin
// closer than the nearest inclusive prefix has published its count; the
// counts up to that prefix are then summed.  Returns the exclusive prefix
// (all threads); thread 0 publishes this bin's aggregate and inclusive prefix.
// The chain starts at bin `first` (0 for one product; a product's first bin in
// a batch): bins before it count as an inclusive prefix of 0.
template <int THREADS>
__device__ inline int64_t lookback_block(uint64_t *status, int64_t b, uint64_t agg, uint32_t *err, int64_t *scratch,
                                         int32_t *marks, int64_t first) {
    const int tid = threadIdx.x;
    if (b == first) {
        if (tid == 0) st_release_u64(&status[b], LB_PREFIX | agg);
        return 0;
    }
    if (tid == 0) st_release_u64(&status[b], LB_AGGREGATE | agg);
    uint64_t prefix = 0;
    int64_t j = b - 1;
    int64_t wait_for = b - 1;  // a bin whose count is needed and may be unpublished
    while (true) {
        // One lane waits (with backoff) until that bin has published; the other
        // threads sleep at the barrier instead of polling.
        if (tid == 0) {
            uint32_t spins = 0, ns = 32;
            while ((ld_acquire_u64(&status[wait_for]) >> LB_FLAG_SHIFT) == 0) {
                if (++spins > SPIN_LIMIT) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns <<= 1;
            }
            marks[0] = THREADS;  // nearest inclusive prefix
            marks[1] = THREADS;  // nearest unpublished bin
        }
        __syncthreads();
        const int64_t idx = j - tid;
        const uint64_t v = (idx >= first) ? ld_acquire_u64(&status[idx]) : LB_PREFIX;  // before the chain: 0
        if ((v & ~LB_VALUE_MASK) == LB_PREFIX) atomicMin(&marks[0], tid);
        if ((v >> LB_FLAG_SHIFT) == 0) atomicMin(&marks[1], tid);
        __syncthreads();
        const int fp = marks[0], fz = marks[1];
        if (fz < fp) {  // a bin in front of the nearest prefix has not published yet
            wait_for = j - fz;
            __syncthreads();
            continue;
        }
        const uint64_t mine = (tid <= fp) ? (v & LB_VALUE_MASK) : 0ull;
        prefix += (uint64_t)block_reduce_sum<int64_t, THREADS>((int64_t)mine, scratch);
        if (fp < THREADS) break;
        j -= THREADS;
        wait_for = j;
    }
    if (tid == 0) st_release_u64(&status[b], LB_PREFIX | (prefix + agg));
    return (int64_t)prefix;
}

// Warp 0: publish this bin's merged count, find its prefix, check C's capacity,
// and let the last bin write nnz(C) and the final row pointer.
__device__ inline void publish_and_check(const NumericArgs &p, int64_t b, int64_t U, int64_t *prefix, int32_t *ok) {
    const int64_t P = lookback_warp(p.status, b, (uint64_t)U, p.err);
    if ((threadIdx.x & 31) != 0) return;
    *prefix = P;
    int32_t good = p.count_only ? 0 : 1;
    if (!p.count_only && (P + U > p.cap || (p.rowptr32 && P + U > 0x7fffffffll))) {
        atomicOr(p.err, DEV_ERR_OVERFLOW);
        good = 0;
    }
    *ok = good;
    if (b == p.nbins - 1) {
        if (good) write_rowptr(p, p.m, P + U);
        if (p.nnz_dev) *p.nnz_dev = P + U;
    }
}

// An oversize bin (one row, more tuples than the on-chip capacity) was sorted
// in global memory before this kernel and its merged count is known: publish
// it at once, then stream the sorted run and write the merged entries.
template <int THREADS, class TV, class OV>
__device__ void stream_oversize_bin(const NumericArgs &p, int64_t b, int32_t row0, int32_t row1, int64_t off,
                                    int64_t N, uint32_t colmask, int64_t *scratch, int64_t *prefix, int32_t *okp) {
    const int tid = threadIdx.x;
    const int64_t o = p.over_scan[b];
    const bool in_scratch = (p.over_passes & 1) != 0;
    const uint32_t *k = in_scratch ? p.skeys + (p.over_tuple_off[o] - p.over_base) : p.keys + off;
    const TV *v = in_scratch ? static_cast<const TV *>(p.svals) + (p.over_tuple_off[o] - p.over_base)
                             : static_cast<const TV *>(p.vals) + off;
    OV *valC = static_cast<OV *>(p.valC);
    if (tid < 32) publish_and_check(p, b, p.over_u[o], prefix, okp);
    __syncthreads();
    const int64_t P = *prefix;
    const bool ok = *okp != 0;
    if (ok)
        for (int32_t r = row0 + tid; r < row1; r += THREADS) write_rowptr(p, r, r == row0 ? P : P + p.over_u[o]);
    if (p.over_dense) {
        // merged in dense tiles already: record where the row goes; a later kernel copies it
        if (tid == 0) p.over_p[o] = ok ? P : -1;
        __syncthreads();
        return;
    }
    int64_t running = 0;
    for (int64_t base = 0; base < N; base += THREADS) {
        const int64_t q = base + tid;
        const bool valid = q < N;
        const uint32_t key = valid ? k[q] : 0u;
        const bool head = valid && (q == 0 || k[q - 1] != key);
        int64_t chunk_total;
        const int64_t u = block_exclusive_scan<int64_t, THREADS>(head ? 1 : 0, scratch, &chunk_total);
        if (head && ok) {
            double acc = (double)v[q];
            for (int64_t r = q + 1; r < N && k[r] == key; ++r) acc += (double)v[r];
            p.colidx[P + running + u] = (int32_t)(key & colmask);
            valC[P + running + u] = (OV)acc;
        }
        running += chunk_total;
    }
    __syncthreads();
}

// BATCH: bins of the products of a batch that share one capacity level; each
// bin writes into its own product's C (taken from the product's descriptor).
template <int CAP, int THREADS, class TV, class OV, bool BATCH>
__global__ void __launch_bounds__(THREADS, (THREADS <= 256 ? 4 : (THREADS <= 512 ? 2 : 1))) k_binsort(const NumericArgs p) {
    using S = SortSmem<CAP, THREADS, TV>;
    constexpr int NW = THREADS / 32;
    constexpr int E = CAP / THREADS;  // tuples per thread; also buckets per thread
    constexpr int WS = CAP / NW;      // positions per warp in the LSD ranking
    constexpr int LOG_CAP = (CAP == 2048) ? 11 : (CAP == 4096) ? 12 : 13;
    static_assert(WS % 32 == 0 && WS / 32 == E, "layout");
    static_assert((1 << LOG_CAP) == CAP, "capacity");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TV *__restrict__ gvals = static_cast<const TV *>(p.vals);
    OV *__restrict__ valC = static_cast<OV *>(p.valC);
    const bool stable_ties = p.apos != nullptr;
    int colbits = p.colbits;
    uint32_t colmask = (p.colbits >= 32) ? 0xffffffffu : ((1u << p.colbits) - 1u);

    if (tid == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    int64_t bin_lo = p.bin_lo, bin_hi = p.bin_hi, nbins = p.nbins;
    if constexpr (BATCH) {
        if (*p.err & DEV_ERR_BATCH_FATAL) return;
        bin_lo = p.bhdr->level_bins[p.level];
        bin_hi = p.bhdr->level_bins[p.level + 1];
        nbins = p.bhdr->nbins;
    }

    while (true) {
        if (tid == 0) sm.bin = bin_lo + (int64_t)atomicAdd(p.ticket, 1u);
        fence_proxy_async_smem();  // earlier generic smem accesses before the next bulk copy
        __syncthreads();
        const int64_t b = sm.bin;
        if (b >= bin_hi) break;
        const int32_t row0 = p.bin_row[b], row1 = p.bin_row[b + 1];
        const int64_t off = p.bin_off[b] - p.tuple_base;  // the buffer holds this panel's tuples
        int64_t Nfull = p.R[row1] - p.R[row0];
        if (Nfull > CAP) {
            if constexpr (BATCH) {
                // the symbolic phase never cuts such a bin for a batch; record it and skip the tuples
                if (tid == 0) atomicOr(p.err, DEV_ERR_CAPACITY);
                Nfull = 0;
            } else {
                stream_oversize_bin<THREADS, TV, OV>(p, b, row0, row1, off, Nfull, colmask, sm.scratch,
                                                     &sm.prefix, &sm.ok);
                continue;
            }
        }
        int N = (int)Nfull;
        const int rows_b = row1 - row0;
        // ---- load the bin (bulk copies, 16-byte granules) -----------------------
        bool loaded = true;
        if (N > 0 && tid == 0) {
            const uint32_t n4 = (uint32_t)((N + 3) & ~3);
            mbar_arrive_expect_tx(&sm.bar, n4 * 4u + n4 * (uint32_t)sizeof(TV));
            bulk_g2s(sm.kin, p.keys + off, n4 * 4u, &sm.bar);
            bulk_g2s(sm.vin, gvals + off, n4 * (uint32_t)sizeof(TV), &sm.bar);
        }
        if constexpr (BATCH) {
            if (tid == 0) {  // the bin's product, fetched while the copies are in flight
                const int32_t q = p.bin_prod[b];
                const BatchDesc &d = p.desc[q];
                BinOut &o = sm.out;
                o.rowptr64 = d.rowptr64;
                o.rowptr32 = d.rowptr32;
                o.colidx = d.colidxC;
                o.valC = d.valC;
                o.nnz_dev = d.nnz_dev;
                o.cap = d.capC;
                o.first = p.prod[q].first_bin;
                o.rbase = d.mstart;
                o.m = d.m;
                o.colbits = d.colbits;
                o.last = (b + 1 == nbins || p.bin_prod[b + 1] != q) ? 1 : 0;
            }
        }
        for (int r = tid; r < rows_b; r += THREADS) sm.rowcnt[r] = 0;
        for (int i = tid; i <= CAP; i += THREADS) sm.cnt[i] = 0;
        if (tid == 0) sm.big = 0;
        if (N > 0) {
            loaded = mbar_wait_bounded(&sm.bar, phase);
            phase ^= 1u;
        }
        if (!__syncthreads_and(loaded)) {
            if (tid == 0) atomicOr(p.err, DEV_ERR_TIMEOUT);
            // a bulk copy may still be landing: wait for it (bounded) before the buffer is reused
            (void)mbar_wait_bounded(&sm.bar, phase ^ 1u);
            N = 0;
        }

        if constexpr (BATCH) {
            colbits = sm.out.colbits;
            colmask = (colbits >= 32) ? 0xffffffffu : ((1u << colbits) - 1u);
        }
        const uint32_t *sk = sm.skey;
        const uint16_t *si = sm.sidx;
        if (N > 0) {
            // Keys lie in [0, rows_b << colbits): the bucket of a key is its top
            // LOG_CAP significant bits.
            const uint32_t kmax = (uint32_t)((((uint64_t)rows_b) << colbits) - 1u);
            const int rbits = kmax ? 32 - __clz(kmax) : 0;
            const int shift = rbits > LOG_CAP ? rbits - LOG_CAP : 0;
            // ---- bucket pass (MSD on the top bits) -----------------------------------
            uint32_t kr[E], rk[E];
            bool mine_big = false;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int q = tid + j * THREADS;
                if (q < N) {
                    kr[j] = sm.kin[q];
                    rk[j] = atomicAdd(&sm.cnt[kr[j] >> shift], 1u);
                    mine_big |= rk[j] >= SMALL_BUCKET;
                }
            }
            if (mine_big) sm.big = 1;
            __syncthreads();
            if (sm.big == 0) {
                if (PB_SORT_VSCAN)
                    smem_exclusive_scan_runs<THREADS, CAP / THREADS>(sm.cnt, sm.scratch);
                else
                    smem_exclusive_scan_striped<THREADS, CAP / THREADS>(sm.cnt, sm.scratch);
                if (tid == 0) sm.cnt[CAP] = N;
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int q = tid + j * THREADS;
                    if (q < N) {
                        const uint32_t pos = sm.cnt[kr[j] >> shift] + rk[j];
                        sm.skey[pos] = kr[j];
                        sm.sidx[pos] = (uint16_t)q;
                    }
                }
                __syncthreads();
                // Each tuple's final slot: its bucket's start plus the number of
                // tuples of the same bucket with a smaller key, ties broken by the
                // order in the bin in deterministic mode (fixed positions: equal
                // keys then merge in that order) and by bucket slot otherwise.
                // Buckets hold a few tuples, so this is a short loop per tuple.
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int q = tid + j * THREADS;
                    if (q < N) {
                        const uint32_t key = sm.skey[q];
                        const uint16_t iq = sm.sidx[q];
                        const uint32_t bk = key >> shift;
                        const int lo = (int)sm.cnt[bk], hi = (int)sm.cnt[bk + 1];
                        int rank = lo;
                        if (stable_ties) {  // equal keys keep their order in the bin
                            for (int r = lo; r < hi; ++r) {
                                const uint32_t o = sm.skey[r];
                                rank += (o < key) || (o == key && sm.sidx[r] < iq);
                            }
                        } else {
                            for (int r = lo; r < hi; ++r) {
                                const uint32_t o = sm.skey[r];
                                rank += (o < key) || (o == key && r < q);
                            }
                        }
                        sm.kin[rank] = key;
                        sm.sidx2[rank] = iq;
                    }
                }
                __syncthreads();
                sk = sm.kin;
                si = sm.sidx2;
            } else {
                // ---- stable LSD radix sort, 8-bit digits ---------------------------------
                uint32_t *srck = sm.kin;
                const uint16_t *srci = nullptr;  // identity on the first pass
                uint32_t *dstk = sm.skey;
                uint16_t *dsti = sm.sidx;
                const int passes_bits = rbits > 0 ? rbits : 1;
                for (int sh = 0; sh < passes_bits; sh += 8) {
                    for (int i = tid; i < 256 * NW; i += THREADS) sm.cnt[i] = 0;
                    __syncthreads();
                    uint32_t kk[E], lr[E];
                    uint16_t ii[E];
                    uint8_t dd[E];
#pragma unroll
                    for (int j = 0; j < E; ++j) {
                        const int q = warp * WS + j * 32 + lane;
                        const bool valid = q < N;
                        const uint32_t key = valid ? srck[q] : 0u;
                        const uint32_t d = (key >> sh) & 255u;
                        uint32_t peers = __ballot_sync(FULL, valid);
#pragma unroll
                        for (int bit = 0; bit < 8; ++bit) {
                            const bool on = (d >> bit) & 1u;
                            const uint32_t bb = __ballot_sync(FULL, on);
                            peers &= on ? bb : ~bb;
                        }
                        const int leader = valid ? (__ffs(peers) - 1) : lane;
                        uint32_t old = 0;
                        if (valid && lane == leader) {
                            old = sm.cnt[d * NW + warp];
                            sm.cnt[d * NW + warp] = old + __popc(peers);
                        }
                        old = __shfl_sync(FULL, old, leader);
                        __syncwarp();
                        lr[j] = old + __popc(peers & lanemask_lt());
                        kk[j] = key;
                        ii[j] = valid ? (srci ? srci[q] : (uint16_t)q) : 0;
                        dd[j] = (uint8_t)d;
                    }
                    __syncthreads();
                    smem_exclusive_scan<THREADS>(sm.cnt, 256 * NW, sm.scratch);
#pragma unroll
                    for (int j = 0; j < E; ++j) {
                        const int q = warp * WS + j * 32 + lane;
                        if (q < N) {
                            const uint32_t pos = sm.cnt[(uint32_t)dd[j] * NW + warp] + lr[j];
                            dstk[pos] = kk[j];
                            dsti[pos] = ii[j];
                        }
                    }
                    __syncthreads();
                    srck = dstk;
                    srci = dsti;
                    dstk = (dstk == sm.skey) ? sm.kin : sm.skey;
                    dsti = (dsti == sm.sidx) ? sm.sidx2 : sm.sidx;
                }
                sk = srck;
                si = srci;
            }
        }
        // ---- compress: each warp counts the merged entries of its segment ------------
        const int seg = ((((N + NW - 1) / NW) + 31) / 32) * 32;
        const int s0 = min(warp * seg, N), s1 = min(s0 + seg, N);
        uint32_t wheads = 0;
        for (int base = s0; base < s1; base += 32) {
            const int q = base + lane;
            const bool head = q < s1 && (q == 0 || sk[q - 1] != sk[q]);
            wheads += __popc(__ballot_sync(FULL, head));
            if (head) atomicAdd(&sm.rowcnt[sk[q] >> colbits], 1u);
        }
        if (lane == 0) sm.wtot[warp] = wheads;
        __syncthreads();
        int64_t U = 0, wbase = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t t = sm.wtot[w];
            wbase += (w < warp) ? t : 0;
            U += t;
        }
        {
            const int64_t first = BATCH ? sm.out.first : 0;
            const int64_t P = lookback_block<THREADS>(p.status, b, (uint64_t)U, p.err, sm.scratch, sm.marks, first);
            if (tid == 0) {
                if constexpr (BATCH) {
                    const BinOut &o = sm.out;
                    int32_t good = 1;
                    if (P + U > o.cap || (o.rowptr32 && P + U > 0x7fffffffll)) {
                        atomicOr(p.err, DEV_ERR_OVERFLOW);
                        good = 0;
                    }
                    sm.prefix = P;
                    sm.ok = good;
                    if (o.last) {
                        if (good) write_rowptr(o, o.m, P + U);
                        if (o.nnz_dev) *o.nnz_dev = P + U;
                    }
                } else {
                    int32_t good = p.count_only ? 0 : 1;
                    if (!p.count_only && (P + U > p.cap || (p.rowptr32 && P + U > 0x7fffffffll))) {
                        atomicOr(p.err, DEV_ERR_OVERFLOW);
                        good = 0;
                    }
                    sm.prefix = P;
                    sm.ok = good;
                    if (b == p.nbins - 1) {
                        if (good) write_rowptr(p, p.m, P + U);
                        if (p.nnz_dev) *p.nnz_dev = P + U;
                    }
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
            // row pointers of this bin's rows: exclusive scan of the per-row counts
            if (sm.ok) {
                const int64_t P = sm.prefix;
                uint32_t carry = 0;
                for (int r0 = 0; r0 < rows_b; r0 += 32) {
                    const int r = r0 + lane;
                    const uint32_t c = (r < rows_b) ? sm.rowcnt[r] : 0u;
                    const uint32_t inc = warp_inclusive_scan(c);
                    if (r < rows_b) {
                        if constexpr (BATCH)
                            write_rowptr(sm.out, row0 - sm.out.rbase + r, P + carry + inc - c);
                        else
                            write_rowptr(p, row0 + r, P + carry + inc - c);
                    }
                    carry += __shfl_sync(FULL, inc, 31);
                }
            }
        }
        __syncthreads();
        const int64_t P = sm.prefix;
        if (sm.ok) {
            // ---- merged entries in key order, coalesced across the warp ----------------
            int32_t *colidxC = p.colidx;
            if constexpr (BATCH) {
                colidxC = sm.out.colidx;
                valC = static_cast<OV *>(sm.out.valC);
            }
            int64_t out = P + wbase;
            for (int base = s0; base < s1; base += 32) {
                const int q = base + lane;
                const bool head = q < s1 && (q == 0 || sk[q - 1] != sk[q]);
                const uint32_t hm = __ballot_sync(FULL, head);
                if (head) {
                    const uint32_t key = sk[q];
                    double acc = (double)sm.vin[si[q]];
                    for (int r = q + 1; r < N && sk[r] == key; ++r) acc += (double)sm.vin[si[r]];
                    const int64_t o = out + __popc(hm & lanemask_lt());
                    colidxC[o] = (int32_t)(key & colmask);
                    valC[o] = (OV)acc;
                }
                out += __popc(hm);
            }
        }
        __syncthreads();
    }
}

template <int CAP, int THREADS, class TV, class OV, bool BATCH>
cudaError_t run_binsort(const NumericArgs &a, cudaStream_t s) {
    using S = SortSmem<CAP, THREADS, TV>;
    auto kern = k_binsort<CAP, THREADS, TV, OV, BATCH>;
    const size_t smem = sizeof(S);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)a.num_sms * per_sm;
    // a batch's bin count is only known on the device: a.bin_hi - a.bin_lo bounds it
    if (grid > a.bin_hi - a.bin_lo) grid = a.bin_hi - a.bin_lo;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, THREADS, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <class TV, class OV, bool BATCH>
cudaError_t dispatch_cap(const NumericArgs &a, cudaStream_t s) {
    switch (a.capacity) {
        case 2048: return run_binsort<2048, 256, TV, OV, BATCH>(a, s);
        case 4096: return run_binsort<4096, 512, TV, OV, BATCH>(a, s);
        case 8192: return run_binsort<8192, 1024, TV, OV, BATCH>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool BATCH>
cudaError_t dispatch_dtype(const NumericArgs &a, cudaStream_t s) {
    if (a.bin_hi <= a.bin_lo) return cudaSuccess;
    switch (a.dtype) {
        case PB_F64: return dispatch_cap<double, double, BATCH>(a, s);
        case PB_F32: return dispatch_cap<float, float, BATCH>(a, s);
        case PB_F64_F32TUPLE: return dispatch_cap<float, double, BATCH>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_binsort(const NumericArgs &a, cudaStream_t s) { return dispatch_dtype<false>(a, s); }

// a.bin_lo / a.bin_hi bound the level's bins (grid size only); the kernel reads
// the exact range from a.bhdr.  a.ticket is the level's own counter.
cudaError_t launch_binsort_batch(const NumericArgs &a, cudaStream_t s) { return dispatch_dtype<true>(a, s); }

}  // namespace pb
