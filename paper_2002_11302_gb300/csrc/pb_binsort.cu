// Sort, compress and ConvertCSR of Alg. 2, one bin per CTA pass.
//
// For each bin (a range of consecutive rows, Sec. III-A/III-D):
//   load     the bin's keys and values with two bulk global->shared copies
//            (the bin is read from DRAM exactly once: "in-cache sorting",
//            Sec. III-D, with shared memory playing the cache);
//   sort     by the packed (in-bin row, column) key (Sec. III-D): a bucket
//            pass on the key's top bits with shared-memory atomic counters,
//            then a rank inside the few multi-tuple buckets; a bin with a
//            bucket above SMALL_BUCKET tuples is sorted by a stable LSD radix
//            sort over 8-bit digits instead;
//   compress equal adjacent keys are summed (Sec. III-E; sums accumulate in
//            double);
//   ConvertCSR the bins are concatenated in row order: the bin's number of
//            merged entries is published and the exclusive prefix over all
//            earlier bins is found by a decoupled look-back (bins are taken in
//            increasing order through a ticket counter, so every bin a CTA
//            waits for is owned by a running CTA); then the column indices,
//            values and row pointers of the bin are written.
// Two kernels: k_binsort for single products (phases described above it) and
// k_binsort_batch for batched products (bins of many products in one launch,
// each bin writing into its own product's C).
#include <type_traits>

#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int RMAX = 1 << RMAX_LOG2;  // max rows of one bin (symbolic cuts bins at multiples of this)

// Test builds only: the sort kernels never take the first bin of their range,
// so the next bin's look-back waits on a bin that never publishes and must end
// by its spin bound (DEV_ERR_TIMEOUT).  0 in every product build.
#ifndef PB_TEST_SKIP_FIRST_BIN
#define PB_TEST_SKIP_FIRST_BIN 0
#endif
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
    int32_t marks[3];       // look-back: nearest inclusive prefix / unpublished bin / gave up
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
// Bounded: a lane gives up on a bin after SPIN_LIMIT polls, records
// DEV_ERR_TIMEOUT and treats the bin as an inclusive prefix of 0, so the walk
// always ends.
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
// Bounded: thread 0 waits at most SPIN_LIMIT polls in the whole look-back.
// When that budget runs out it records DEV_ERR_TIMEOUT and the look-back stops
// waiting: every bin still unpublished counts as 0 (its status word is 0), so
// each later round either ends the walk or moves THREADS bins further back,
// and the walk ends at bin `first` at the latest.
template <int THREADS>
__device__ inline int64_t lookback_block(uint64_t *status, int64_t b, uint64_t agg, uint32_t *err, int64_t *scratch,
                                         int32_t *marks, int64_t first) {
    const int tid = threadIdx.x;
    if (b == first) {
        if (tid == 0) st_release_u64(&status[b], LB_PREFIX | agg);
        return 0;
    }
    if (tid == 0) {
        st_release_u64(&status[b], LB_AGGREGATE | agg);
        marks[2] = 0;  // set once the wait budget is spent
    }
    uint64_t prefix = 0;
    int64_t j = b - 1;
    int64_t wait_for = b - 1;  // a bin whose count is needed and may be unpublished
    uint32_t spins = 0;        // thread 0: polls so far in this look-back
    while (true) {
        // One lane waits (with backoff) until that bin has published; the other
        // threads sleep at the barrier instead of polling.
        if (tid == 0) {
            uint32_t ns = 32;
            while (marks[2] == 0 && (ld_acquire_u64(&status[wait_for]) >> LB_FLAG_SHIFT) == 0) {
                if (++spins > SPIN_LIMIT) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
                    marks[2] = 1;
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns <<= 1;
            }
            marks[0] = THREADS;  // nearest inclusive prefix
            marks[1] = THREADS;  // nearest unpublished bin
        }
        __syncthreads();
        const bool gave_up = marks[2] != 0;
        const int64_t idx = j - tid;
        const uint64_t v = (idx >= first) ? ld_acquire_u64(&status[idx]) : LB_PREFIX;  // before the chain: 0
        if ((v & ~LB_VALUE_MASK) == LB_PREFIX) atomicMin(&marks[0], tid);
        if ((v >> LB_FLAG_SHIFT) == 0) atomicMin(&marks[1], tid);
        __syncthreads();
        const int fp = marks[0], fz = marks[1];
        if (fz < fp && !gave_up) {  // a bin in front of the nearest prefix has not published yet
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

// ---------------------------------------------------------------------------
// Single-product sort kernel (one bin per CTA pass, bins taken by ticket).
//
// Phases of one bin of N <= CAP tuples (THREADS threads, E = CAP / THREADS
// tuples per thread, bucket b = key >> shift with shift chosen so that the
// bin's key range spans at most CAP buckets):
//   A  count: thread t takes tuples t, t + THREADS, ...; one shared-memory
//      atomic per tuple gives its bucket's count and its arrival rank there.
//   B  bucket starts: thread t owns buckets [4t, 4t+4) and [CAP/2 + 4t, ...);
//      both halves are scanned at once as the two 16-bit halves of one word
//      (counts never exceed CAP <= 8192).  Each counter becomes the packed word
//      start | size << 16, so one load later gives both.
//   C  place: a tuple alone in its bucket is at its final position (its
//      bucket's start); the others write (key bits below the bucket, position
//      in the bin) into their bucket's slots.
//   D  rank: a tuple of a multi-tuple bucket counts the smaller packed words
//      of its bucket; equal keys order by position in the bin (a stable sort).
//   A bucket above SMALL_BUCKET tuples switches the bin to a stable LSD radix
//   sort (8-bit digits, warp multisplit ranking) instead of B-D.
//   E  heads: warp w owns sorted positions [w*CAP/NW, (w+1)*CAP/NW) in
//      32-position chunks; a head is a key different from its predecessor,
//      one ballot per chunk marks them and the warp's count of merged entries
//      goes to shared memory.  Warp 0 then publishes the bin's count and finds
//      its prefix by the decoupled look-back.
//   F  write C: the merged entry of a run goes to prefix + (heads before it).
//      Chunks without duplicates write every tuple directly; a chunk with
//      duplicates sums each run by a segmented warp-shuffle reduction
//      (Sec. III-E's merge), or sequentially from its head when duplicates are
//      few or the order of the sum is fixed (deterministic mode: equal keys
//      then sum in position order, i.e. ascending k).  Row pointers are written
//      where the row changes.
// ---------------------------------------------------------------------------
// PACK: the bin arrives as packed {key, value bits} pairs (4-byte values) in
// pin; phase A keeps each key in a register and stores the value into vin at
// the tuple's position, so everything after phase A is as for separate arrays
// (the radix path's first pass reads the keys from pin).
template <int CAP, int THREADS, class TV, bool PACK = false>
struct BinSmem {
    static constexpr int NW = THREADS / 32;
    uint32_t kin[CAP];     // the bin's keys (bulk copy), then its sorted keys
    TV vin[CAP];           // the bin's values (bulk copy; PACK: written by phase A)
    uint32_t pk[CAP];      // multi-tuple buckets: low key bits << log2(CAP) | position; radix: keys
    uint16_t fidx[CAP];    // position in the bin of each sorted tuple
    uint16_t sidx2[CAP];   // radix: positions
    alignas(16) uint32_t cnt[CAP];  // bucket counters, then start | size << 16; radix digit counters (uint4 access)
    int64_t scratch[40];
    uint32_t wtot[NW];     // per warp: bucket-count sums (B), merged entries (E)
    uint64_t bar;
    int64_t bin;
    int64_t prefix;
    uint32_t big;
    int32_t ok;
    alignas(16) uint2 pin[PACK ? CAP : 1];  // PACK: the bin's {key, value bits} pairs (bulk copy)
};

__device__ inline uint32_t lanemask_le() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

template <int CAP, int THREADS>
__device__ inline void zero_counters(uint32_t *cnt) {
    static_assert(CAP % (4 * THREADS) == 0, "whole uint4 per thread");
#pragma unroll
    for (int i = 4 * threadIdx.x; i < CAP; i += 4 * THREADS) *reinterpret_cast<uint4 *>(cnt + i) = make_uint4(0, 0, 0, 0);
}

// Bucket of a key.  Keys of a bin lie below rows << colbits, so key >> shift
// is below CAP; the clamp only keeps a malformed key (a column of B outside
// [0, n)) inside the counter array.
__device__ inline uint32_t bucket_of(uint32_t key, int shift, int cap) { return min(key >> shift, (uint32_t)cap - 1u); }

// Packed bucket words of 4 consecutive counters starting at offset `s`.
__device__ inline uint4 bucket_words(uint4 c, uint32_t s) {
    uint4 o;
    o.x = s | (c.x << 16);
    s += c.x;
    o.y = s | (c.y << 16);
    s += c.y;
    o.z = s | (c.z << 16);
    s += c.z;
    o.w = s | (c.w << 16);
    return o;
}

// Bring bin nb's tuples into L2 (bulk prefetch; one thread).  A CTA calls this
// for the bin one grid ahead of the one it takes, about the bin it takes next,
// without taking its ticket (the look-back chain is not lengthened).  Bin
// regions start at multiples of 4 tuples and are padded to them (16-byte
// granules); bins above the capacity are left alone.
template <class TV, bool PACK>
__device__ inline void prefetch_bin_l2(const NumericArgs &p, int64_t nb, int cap) {
    const int64_t o0 = p.bin_off[nb] - p.tuple_base, n = p.bin_off[nb + 1] - p.bin_off[nb];
    if (n <= 0 || n > cap) return;
    if constexpr (PACK) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const uint2 *>(p.keys) + o0),
                     "r"((uint32_t)(n * 8)) : "memory");
    } else {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p.keys + o0), "r"((uint32_t)(n * 4)) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const TV *>(p.vals) + o0),
                     "r"((uint32_t)(n * sizeof(TV))) : "memory");
    }
}


template <int CAP, int THREADS, class TV, class OV, bool PACK>
__global__ void __launch_bounds__(THREADS, (THREADS <= 256 ? 4 : (THREADS <= 512 ? 2 : 1))) k_binsort(const NumericArgs p) {
    using S = BinSmem<CAP, THREADS, TV, PACK>;
    static_assert(!PACK || sizeof(TV) == 4, "packed tuples hold 4-byte values");
    static_assert(offsetof(S, cnt) % 16 == 0 && offsetof(S, vin) % 16 == 0 && offsetof(S, pin) % 16 == 0,
                  "16-byte accesses and bulk-copy destinations");
    constexpr int NW = THREADS / 32;
    constexpr int E = CAP / THREADS;  // tuples per thread in A-D
    constexpr int WS = CAP / NW;      // sorted positions per warp in E-F
    constexpr int CH = WS / 32;       // chunks per warp
    constexpr int HALF = CAP / 2;
    constexpr int LOG_CAP = (CAP == 2048) ? 11 : (CAP == 4096) ? 12 : 13;
    static_assert((1 << LOG_CAP) == CAP && E == 8 && CH == 8 && 256 * NW == CAP, "layout");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TV *__restrict__ gvals = static_cast<const TV *>(p.vals);
    OV *__restrict__ valC = static_cast<OV *>(p.valC);
    int32_t *__restrict__ colidxC = p.colidx;
    const bool det = p.apos != nullptr;
    const int colbits = p.colbits;
    const uint32_t colmask = (colbits >= 32) ? 0xffffffffu : ((1u << colbits) - 1u);

    if (tid == 0) {
        mbar_init(&sm.bar, 1);
        sm.big = 0;
    }
    zero_counters<CAP, THREADS>(sm.cnt);
    uint32_t phase = 0;
    while (true) {
        if (tid == 0) sm.bin = p.bin_lo + PB_TEST_SKIP_FIRST_BIN + (int64_t)atomicAdd(p.ticket, 1u);
        fence_proxy_async_smem();  // this thread's reads of the last bin before the next bulk copy
        __syncthreads();
        const int64_t b = sm.bin;
        if (b >= p.bin_hi) break;
        const int32_t row0 = p.bin_row[b], row1 = p.bin_row[b + 1];
        const int64_t off = p.bin_off[b] - p.tuple_base;  // the buffer holds this panel's tuples
        int64_t Nfull = p.R[row1] - p.R[row0];
        if (Nfull > CAP) {
            if constexpr (PACK) {
                // packed plans have no oversize bins; record it and skip the tuples
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
        if (tid == 32 && b + gridDim.x < p.bin_hi) prefetch_bin_l2<TV, PACK>(p, b + gridDim.x, CAP);
        // ---- load the bin (bulk copies, 16-byte granules) ---------------------------
        bool loaded = true;
        if (N > 0) {
            if (tid == 0) {
                const uint32_t n4 = (uint32_t)((N + 3) & ~3);
                if constexpr (PACK) {
                    mbar_arrive_expect_tx(&sm.bar, n4 * 8u);
                    bulk_g2s(sm.pin, reinterpret_cast<const uint2 *>(p.keys) + off, n4 * 8u, &sm.bar);
                } else {
                    mbar_arrive_expect_tx(&sm.bar, n4 * 4u + n4 * (uint32_t)sizeof(TV));
                    bulk_g2s(sm.kin, p.keys + off, n4 * 4u, &sm.bar);
                    bulk_g2s(sm.vin, gvals + off, n4 * (uint32_t)sizeof(TV), &sm.bar);
                }
            }
            loaded = mbar_wait_bounded(&sm.bar, phase);
            phase ^= 1u;
        }
        if (!__syncthreads_and(loaded)) {
            if (tid == 0) atomicOr(p.err, DEV_ERR_TIMEOUT);
            // a bulk copy may still be landing: wait for it (bounded) before the buffer is reused
            (void)mbar_wait_bounded(&sm.bar, phase ^ 1u);
            N = 0;
        }
        const uint32_t *sk = sm.kin;   // sorted keys
        const uint16_t *si = sm.fidx;  // their positions in the bin
        if (N > 0) {
            const uint32_t kmax = (uint32_t)((((uint64_t)rows_b) << colbits) - 1u);
            const int rbits = kmax ? 32 - __clz(kmax) : 0;
            const int shift = rbits > LOG_CAP ? rbits - LOG_CAP : 0;  // <= 32 - LOG_CAP
            const uint32_t lowmask = (1u << shift) - 1u;
            // ---- A: bucket counts and arrival ranks ------------------------------------
            uint32_t kr[E], rk[E];
            bool mine_big = false;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int q = tid + j * THREADS;
                kr[j] = 0;
                rk[j] = 0;
                if (q < N) {
                    if constexpr (PACK) {
                        const uint2 t = sm.pin[q];
                        kr[j] = t.x;
                        sm.vin[q] = __uint_as_float(t.y);
                    } else {
                        kr[j] = sm.kin[q];
                    }
                    rk[j] = atomicAdd(&sm.cnt[bucket_of(kr[j], shift, CAP)], 1u);
                    mine_big |= rk[j] >= SMALL_BUCKET;
                }
            }
            if (mine_big) sm.big = 1;
            __syncthreads();
            if (sm.big == 0) {
                // ---- B: bucket starts ---------------------------------------------------
                {
                    uint4 *c0 = reinterpret_cast<uint4 *>(sm.cnt + 4 * tid);
                    uint4 *c1 = reinterpret_cast<uint4 *>(sm.cnt + HALF + 4 * tid);
                    const uint4 a0 = *c0, a1 = *c1;
                    const uint32_t v = (a0.x + a0.y + a0.z + a0.w) | ((a1.x + a1.y + a1.z + a1.w) << 16);
                    const uint32_t inc = warp_inclusive_scan(v);
                    if (lane == 31) sm.wtot[warp] = inc;
                    __syncthreads();
                    uint32_t base = 0, total = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const uint32_t t = sm.wtot[w];
                        base += (w < warp) ? t : 0u;
                        total += t;
                    }
                    const uint32_t ex = base + inc - v;
                    *c0 = bucket_words(a0, ex & 0xffffu);
                    *c1 = bucket_words(a1, (total & 0xffffu) + (ex >> 16));
                }
                __syncthreads();
                // ---- C: singletons to their final slot, the rest into their bucket ------
                uint32_t multi = 0;
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int q = tid + j * THREADS;
                    if (q < N) {
                        const uint32_t w = sm.cnt[bucket_of(kr[j], shift, CAP)];
                        const uint32_t start = w & 0xffffu;
                        if ((w >> 16) == 1u) {
                            sm.kin[start] = kr[j];
                            sm.fidx[start] = (uint16_t)q;
                        } else {
                            sm.pk[start + rk[j]] = ((kr[j] & lowmask) << LOG_CAP) | (uint32_t)q;
                            multi |= 1u << j;
                        }
                    }
                }
                __syncthreads();
                // ---- D: rank inside multi-tuple buckets ---------------------------------
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    if (multi & (1u << j)) {
                        const int q = tid + j * THREADS;
                        const uint32_t w = sm.cnt[bucket_of(kr[j], shift, CAP)];
                        const int start = (int)(w & 0xffffu), end = start + (int)(w >> 16);
                        const uint32_t mine = ((kr[j] & lowmask) << LOG_CAP) | (uint32_t)q;
                        int rank = start;
                        for (int r = start; r < end; ++r) rank += sm.pk[r] < mine;
                        sm.kin[rank] = kr[j];
                        sm.fidx[rank] = (uint16_t)q;
                    }
                }
                __syncthreads();
            } else {
                // ---- stable LSD radix sort, 8-bit digits --------------------------------
                const uint32_t *srck = sm.kin;
                const uint16_t *srci = nullptr;  // identity on the first pass
                uint32_t *dstk = sm.pk;
                uint16_t *dsti = sm.fidx;
                const int passes_bits = rbits > 0 ? rbits : 1;
                for (int sh = 0; sh < passes_bits; sh += 8) {
                    zero_counters<CAP, THREADS>(sm.cnt);
                    __syncthreads();
                    uint32_t kk[E], lr[E];
                    uint16_t ii[E];
                    uint8_t dd[E];
#pragma unroll
                    for (int j = 0; j < E; ++j) {
                        const int q = warp * WS + j * 32 + lane;
                        const bool valid = q < N;
                        uint32_t key = 0u;
                        if constexpr (PACK) {  // the first pass reads the packed input
                            if (valid) key = srci ? srck[q] : sm.pin[q].x;
                        } else {
                            if (valid) key = srck[q];
                        }
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
                    dstk = (dstk == sm.pk) ? sm.kin : sm.pk;
                    dsti = (dsti == sm.fidx) ? sm.sidx2 : sm.fidx;
                }
                sk = srck;
                si = srci;
            }
        }
        // counters of the next bin (buckets and digits are no longer read)
        zero_counters<CAP, THREADS>(sm.cnt);
        if (tid == 0) sm.big = 0;
        // ---- E: heads (first tuple of each run of equal keys), per warp segment --------
        const int sbase = warp * WS;
        const uint32_t before = (sbase > 0 && sbase - 1 < N) ? sk[sbase - 1] : 0u;  // key ahead of the segment
        uint32_t keyc[CH], hmc[CH];
        uint32_t heads = 0;
        {
            uint32_t last = before;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int q = sbase + c * 32 + lane;
                const bool valid = q < N;
                const uint32_t key = valid ? sk[q] : 0u;
                uint32_t prev = __shfl_up_sync(FULL, key, 1);
                if (lane == 0) prev = last;
                hmc[c] = __ballot_sync(FULL, valid && (q == 0 || key != prev));
                heads += __popc(hmc[c]);
                keyc[c] = key;
                last = __shfl_sync(FULL, key, 31);
            }
        }
        if (lane == 0) sm.wtot[warp] = heads;
        __syncthreads();
        int64_t U = 0, wbase = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t t = sm.wtot[w];
            wbase += (w < warp) ? t : 0u;
            U += t;
        }
        if (warp == 0) publish_and_check(p, b, U, &sm.prefix, &sm.ok);
        __syncthreads();
        if (!sm.ok) continue;
        // ---- F: merged entries and row pointers ---------------------------------------
        // value of the tuple at sorted position i
        auto value_at = [&](int i) -> double { return (double)sm.vin[si[i]]; };
        const int64_t P = sm.prefix;
        int64_t running = P + wbase;  // C position of the segment's first head
        uint32_t last = before;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int q = sbase + c * 32 + lane;
            const bool valid = q < N;
            const uint32_t vm = __ballot_sync(FULL, valid);
            if (vm == 0) break;
            const uint32_t key = keyc[c], hm = hmc[c];
            uint32_t prev = __shfl_up_sync(FULL, key, 1);
            if (lane == 0) prev = last;
            last = __shfl_sync(FULL, key, 31);
            const bool head = (hm >> lane) & 1u;
            const int64_t idx = running + __popc(hm & lanemask_le()) - 1;  // this tuple's merged entry
            if (head) {  // rows from the one after the previous tuple's row up to this row start here
                const int rh = (int)(key >> colbits);
                const int rp = (q == 0) ? -1 : (int)(prev >> colbits);
                for (int r = rp + 1; r <= rh; ++r) write_rowptr(p, row0 + r, idx);
            }
            // does the run holding lane 31 end inside this chunk?
            bool ends = true;
            const int qn = sbase + c * 32 + 32;
            if (vm == FULL && qn < N) ends = (c + 1 < CH) ? ((hmc[c + 1 < CH ? c + 1 : c] & 1u) != 0) : (sk[qn] != last);
            const int dups = __popc(vm & ~hm);
            if (hm == vm && ends) {
                if (valid) {  // no duplicates: every tuple is its own entry
                    colidxC[idx] = (int32_t)(key & colmask);
                    valC[idx] = (OV)value_at(q);
                }
            } else if (det || dups <= 4) {
                if (head) {  // the run summed in sorted order from its head
                    double acc = value_at(q);
                    for (int r = q + 1; r < N && sk[r] == key; ++r) acc += value_at(r);
                    colidxC[idx] = (int32_t)(key & colmask);
                    valC[idx] = (OV)acc;
                }
            } else {
                // segmented suffix sums: lane l adds lanes (l, end of its run in the chunk]
                double v = valid ? value_at(q) : 0.0;
                const uint32_t after = hm & ~lanemask_le();
                const int endl = after ? __ffs(after) - 2 : 31;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double t = __shfl_down_sync(FULL, v, o);
                    if (lane + o <= endl) v += t;
                }
                if (head) {
                    if (endl == 31 && !ends)  // the run goes on past the chunk
                        for (int r = qn; r < N && sk[r] == key; ++r) v += value_at(r);
                    colidxC[idx] = (int32_t)(key & colmask);
                    valC[idx] = (OV)v;
                }
            }
            running += __popc(hm);
        }
        if (warp == 0) {  // rows after the bin's last tuple (all rows of an empty bin)
            const int rl = N > 0 ? (int)(sk[N - 1] >> colbits) : -1;
            for (int r = rl + 1 + lane; r < rows_b; r += 32) write_rowptr(p, row0 + r, P + U);
        }
    }
}

// The product of batch bin b: where its merged entries go (thread 0).
__device__ inline void load_bin_out(const NumericArgs &p, int64_t b, int64_t nbins, BinOut &o) {
    const int32_t q = p.bin_prod[b];
    const BatchDesc &d = p.desc[q];
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

// Batch bin b is one row above the capacity, merged in dense tiles before this
// kernel (its merged count is known): publish the count in its product's
// look-back chain, write the row pointer(s) and record the row's C offset for
// the copy kernel that runs after the sort.
template <int THREADS>
__device__ void batch_oversize_bin(const NumericArgs &p, int64_t b, int32_t row0, int64_t nbins, BinOut &out,
                                   int64_t *scratch, int32_t *marks) {
    const int tid = threadIdx.x;
    if (tid == 0) load_bin_out(p, b, nbins, out);
    __syncthreads();
    const int64_t o = p.over_scan[b];
    const int64_t U = p.over_u[o];
    const int64_t P = lookback_block<THREADS>(p.status, b, (uint64_t)U, p.err, scratch, marks, out.first);
    if (tid == 0) {
        const bool good = !(P + U > out.cap || (out.rowptr32 && P + U > 0x7fffffffll));
        if (!good) atomicOr(p.err, DEV_ERR_OVERFLOW);
        if (good) write_rowptr(out, row0 - out.rbase, P);
        if (out.last) {
            if (good) write_rowptr(out, out.m, P + U);
            if (out.nnz_dev) *out.nnz_dev = P + U;
        }
        p.over_p[o] = good ? P : -1;
    }
    __syncthreads();  // the shared descriptor and look-back words are reused by the next bin
}

// BATCH: bins of the products of a batch that share one capacity level; each
// bin writes into its own product's C (taken from the product's descriptor).
template <int CAP, int THREADS, class TV, class OV, bool BATCH>
__global__ void __launch_bounds__(THREADS, (THREADS <= 256 ? 4 : (THREADS <= 512 ? 2 : 1))) k_binsort_batch(const NumericArgs p) {
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
        if (tid == 0) sm.bin = bin_lo + PB_TEST_SKIP_FIRST_BIN + (int64_t)atomicAdd(p.ticket, 1u);
        fence_proxy_async_smem();  // earlier generic smem accesses before the next bulk copy
        __syncthreads();
        const int64_t b = sm.bin;
        if (b >= bin_hi) break;
        const int32_t row0 = p.bin_row[b], row1 = p.bin_row[b + 1];
        const int64_t off = p.bin_off[b] - p.tuple_base;  // the buffer holds this panel's tuples
        int64_t Nfull = p.R[row1] - p.R[row0];
        if (Nfull > CAP) {
            if constexpr (BATCH) {
                batch_oversize_bin<THREADS>(p, b, row0, nbins, sm.out, sm.scratch, sm.marks);
                continue;
            } else {
                stream_oversize_bin<THREADS, TV, OV>(p, b, row0, row1, off, Nfull, colmask, sm.scratch,
                                                     &sm.prefix, &sm.ok);
                continue;
            }
        }
        int N = (int)Nfull;
        const int rows_b = row1 - row0;
        if (tid == 32 && b + gridDim.x < bin_hi) prefetch_bin_l2<TV, false>(p, b + gridDim.x, CAP);
        // ---- load the bin (bulk copies, 16-byte granules) -----------------------
        bool loaded = true;
        if (N > 0 && tid == 0) {
            const uint32_t n4 = (uint32_t)((N + 3) & ~3);
            mbar_arrive_expect_tx(&sm.bar, n4 * 4u + n4 * (uint32_t)sizeof(TV));
            bulk_g2s(sm.kin, p.keys + off, n4 * 4u, &sm.bar);
            bulk_g2s(sm.vin, gvals + off, n4 * (uint32_t)sizeof(TV), &sm.bar);
        }
        if constexpr (BATCH) {
            if (tid == 0) load_bin_out(p, b, nbins, sm.out);  // fetched while the copies are in flight
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

template <int CAP, int THREADS, class TV, class OV, bool BATCH, bool PACK = false>
cudaError_t run_binsort(const NumericArgs &a, cudaStream_t s) {
    auto kern = BATCH ? k_binsort_batch<CAP, THREADS, TV, OV, true> : k_binsort<CAP, THREADS, TV, OV, PACK>;
    const size_t smem = BATCH ? sizeof(SortSmem<CAP, THREADS, TV>) : sizeof(BinSmem<CAP, THREADS, TV, PACK>);
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

template <class TV, class OV, bool BATCH, bool PACK = false>
cudaError_t dispatch_cap(const NumericArgs &a, cudaStream_t s) {
    switch (a.capacity) {
        case 2048: return run_binsort<2048, 256, TV, OV, BATCH, PACK>(a, s);
        case 4096: return run_binsort<4096, 512, TV, OV, BATCH, PACK>(a, s);
        case 8192: return run_binsort<8192, 1024, TV, OV, BATCH, PACK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool BATCH>
cudaError_t dispatch_dtype(const NumericArgs &a, cudaStream_t s) {
    if (a.bin_hi <= a.bin_lo) return cudaSuccess;
    if (!BATCH && a.packed) {
        switch (a.dtype) {
            case PB_F32: return dispatch_cap<float, float, false, true>(a, s);
            case PB_F64_F32TUPLE: return dispatch_cap<float, double, false, true>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
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
