// Oversize bins: single heavy rows whose tuples exceed the on-chip sort capacity.
//
// The paper keeps every bin sortable in cache by using more bins or variable
// row ranges (Sec. III-D); a single row cannot be split by rows, so its tuples
// (all with in-bin row 0, key = column) are merged here in global memory.
// Both paths start from the same stable partition in chunks of OVER_CHUNK tuples:
//   histogram  per chunk, counts of each 8-bit digit value;
//   offsets    per oversize row, for every (digit, chunk) the destination of
//              the chunk's first tuple with that digit (digit-major order);
//   scatter    each chunk ranks its tuples stably (warp multisplit over the
//              digit with ballots, per-warp counters), stages them in shared
//              memory in digit order and writes them out coalesced.
// Dense path (default): one pass on the column's top 8 bits, then each row is
// merged in dense shared-memory tiles in column order (k_over_dense) and later
// copied into C at the offset the sort kernel found (k_over_emit).
// Radix path (deterministic mode, or columns too wide for a tile): LSD passes
// over all key bits alternate between the row's region of the tuple buffer and
// a scratch region; a head count then gives each row's merged size, so the
// look-back chain of the sort phase never waits for the merge itself, and the
// sort kernel streams the sorted run into C.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int OT = 512;             // threads per CTA
constexpr int OE = OVER_CHUNK / OT;  // tuples per thread in a chunk
constexpr int ONW = OT / 32;
constexpr int OWS = OVER_CHUNK / ONW;  // tuples per warp in a chunk

struct ChunkRef {
    int64_t o, start, len;
    int64_t main_base, scr_base;  // the bin's first tuple in the main and scratch buffers
};

// End of the oversize bins and of their work items: the launch's values, or
// for a batch the counts its symbolic phase found on the device.
__device__ inline int64_t over_o_hi(const OversizeArgs &a) { return a.dev_count ? a.dev_count[0] : a.o_hi; }
__device__ inline int64_t over_c_hi(const OversizeArgs &a) { return a.dev_count ? a.dev_count[1] : a.c_hi; }
// Per-work-item digit histograms: a batch keeps them in its tuple buffer.
__device__ inline uint32_t *over_hist(const OversizeArgs &a) {
    return a.dev_count ? a.keys + a.dev_count[2] : a.hist;
}

// Work item c from the lists (four levels of dependent loads).
__device__ inline ChunkRef chunk_lookup(const OversizeArgs &a, int64_t c) {
    ChunkRef r;
    r.o = a.over_chunk_bin[c];
    const int64_t bin = a.over_bin[r.o];
    const int64_t N = a.R[a.bin_row[bin + 1]] - a.R[a.bin_row[bin]];
    r.start = (c - a.over_chunk_off[r.o]) * OVER_CHUNK;
    r.len = (N - r.start < OVER_CHUNK) ? N - r.start : OVER_CHUNK;
    r.main_base = a.bin_off[bin] - a.tuple_base;
    r.scr_base = a.over_tuple_off[r.o] - a.over_base;
    return r;
}

__device__ inline ChunkRef chunk_ref(const OversizeArgs &a, int64_t c) {
    if (!a.cinfo) return chunk_lookup(a, c);
    const OverChunk x = a.cinfo[c - a.c_lo];
    return ChunkRef{x.o, x.start, x.len, x.main_base, x.scr_base};
}

__global__ void k_over_chunk_info(const OversizeArgs a) {
    for (int64_t c = a.c_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.c_hi;
         c += (int64_t)gridDim.x * blockDim.x) {
        const ChunkRef r = chunk_lookup(a, c);
        a.cinfo[c - a.c_lo] = OverChunk{r.main_base, r.scr_base, r.start, (int32_t)r.len, (int32_t)r.o};
    }
}

// Bring the `len` tuples from index t of a bin's region into L2 (bulk prefetch).
// Regions start at multiples of 4 tuples and are padded to them, so rounding
// len up keeps to 16-byte granules inside the region.
template <class T>
__device__ inline void prefetch_tuples_l2(const T *base, int64_t t, int64_t len) {
    const uint32_t bytes = (uint32_t)(((len + 3) & ~int64_t(3)) * (int64_t)sizeof(T));
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + t), "r"(bytes) : "memory");
}

template <class TV>
__device__ inline void pass_buffers(const OversizeArgs &a, int pass, const ChunkRef &r, const uint32_t *&sk,
                                    const TV *&sv, uint32_t *&dk, TV *&dv) {
    uint32_t *mk = a.keys + r.main_base;
    TV *mv = static_cast<TV *>(a.vals) + r.main_base;
    uint32_t *xk = a.skeys + r.scr_base;
    TV *xv = static_cast<TV *>(a.svals) + r.scr_base;
    if ((pass & 1) == 0) {
        sk = mk; sv = mv; dk = xk; dv = xv;
    } else {
        sk = xk; sv = xv; dk = mk; dv = mv;
    }
}

template <class TV>
__global__ void __launch_bounds__(OT) k_over_hist(const OversizeArgs a, int pass, int shift) {
    __shared__ uint32_t h[256];
    const int64_t c_hi = over_c_hi(a);
    uint32_t *hist = over_hist(a);
    for (int64_t c = a.c_lo + blockIdx.x; c < c_hi; c += gridDim.x) {
        const ChunkRef r = chunk_ref(a, c);
        const bool has_next = c + gridDim.x < c_hi;
        ChunkRef rn{};
        if (threadIdx.x == 0 && has_next) rn = chunk_ref(a, c + gridDim.x);  // used after the count
        const uint32_t *sk;
        const TV *sv;
        uint32_t *dk;
        TV *dv;
        pass_buffers<TV>(a, pass, r, sk, sv, dk, dv);
        for (int i = threadIdx.x; i < 256; i += OT) h[i] = 0;
        __syncthreads();
        for (int64_t q = threadIdx.x; q < r.len; q += OT) atomicAdd(&h[(sk[r.start + q] >> shift) & 255u], 1u);
        if (threadIdx.x == 0 && has_next) {  // the CTA's next work item into L2
            const uint32_t *nk;
            const TV *nv;
            uint32_t *dk2;
            TV *dv2;
            pass_buffers<TV>(a, pass, rn, nk, nv, dk2, dv2);
            prefetch_tuples_l2(nk, rn.start, rn.len);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += OT) hist[(c - a.c_lo) * 256 + i] = h[i];
        __syncthreads();
    }
}

// One CTA per oversize bin: hist[c][d] becomes the destination offset (within
// the bin) of chunk c's first tuple with digit d.
__global__ void __launch_bounds__(256) k_over_offsets(const OversizeArgs a) {
    __shared__ int64_t scratch[40];
    const int d = threadIdx.x;  // one digit value per thread
    const int64_t o_hi = over_o_hi(a);
    uint32_t *hist = over_hist(a);
    for (int64_t o = a.o_lo + blockIdx.x; o < o_hi; o += gridDim.x) {
        const int64_t c0 = a.over_chunk_off[o] - a.c_lo, c1 = a.over_chunk_off[o + 1] - a.c_lo;
        uint32_t run = 0;
        for (int64_t c = c0; c < c1; ++c) {
            const uint32_t v = hist[c * 256 + d];
            hist[c * 256 + d] = run;
            run += v;
        }
        int64_t total;
        const int64_t base = block_exclusive_scan<int64_t, 256>((int64_t)run, scratch, &total);
        for (int64_t c = c0; c < c1; ++c) hist[c * 256 + d] += (uint32_t)base;
        __syncthreads();
    }
}

template <class TV>
struct ScatterSmem {
    uint32_t wc[256 * ONW];   // per (digit, warp) counts, then offsets inside the digit's run
    uint32_t cbase[256];      // first position of each digit in the chunk's staged order
    int64_t gbase[256];       // destination of a staged position i with digit d: gbase[d] + i
    uint32_t hrow[256];       // the work item's digit offsets (loaded before the ranking)
    uint32_t sk[OVER_CHUNK];  // the chunk, staged in digit order
    TV sv[OVER_CHUNK];
};

// Stable scatter of one chunk: ranks inside the chunk (warp multisplit), the
// chunk staged in shared memory in digit order, then written out so that
// consecutive threads write consecutive slots of each digit's run.
template <class TV>
__global__ void __launch_bounds__(OT, 2) k_over_scatter(const OversizeArgs a, int pass, int shift) {
    extern __shared__ __align__(16) unsigned char smraw[];
    ScatterSmem<TV> &m = *reinterpret_cast<ScatterSmem<TV> *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c_hi = over_c_hi(a);
    const uint32_t *hist = over_hist(a);
    for (int64_t c = a.c_lo + blockIdx.x; c < c_hi; c += gridDim.x) {
        const ChunkRef r = chunk_ref(a, c);
        const uint32_t *sk;
        const TV *sv;
        uint32_t *dk;
        TV *dv;
        pass_buffers<TV>(a, pass, r, sk, sv, dk, dv);
        // loaded now, used after the ranking: this work item's digit offsets and
        // where the CTA's next work item lies (its tuples are then brought into L2)
        uint32_t hv = 0;
        if (threadIdx.x < 256) hv = hist[(c - a.c_lo) * 256 + threadIdx.x];
        const bool has_next = c + gridDim.x < c_hi;
        ChunkRef rn{};
        if (threadIdx.x == 0 && has_next) rn = chunk_ref(a, c + gridDim.x);
        for (int i = threadIdx.x; i < 256 * ONW; i += OT) m.wc[i] = 0;
        __syncthreads();
        uint32_t kk[OE], lr[OE];
        TV vv[OE];
#pragma unroll
        for (int j = 0; j < OE; ++j) {
            const int64_t q = warp * OWS + j * 32 + lane;
            const bool valid = q < r.len;
            const uint32_t key = valid ? sk[r.start + q] : 0u;
            vv[j] = valid ? sv[r.start + q] : TV(0);
            const uint32_t dg = (key >> shift) & 255u;
            uint32_t peers = __ballot_sync(FULL, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool on = (dg >> bit) & 1u;
                const uint32_t bb = __ballot_sync(FULL, on);
                peers &= on ? bb : ~bb;
            }
            const int leader = valid ? (__ffs(peers) - 1) : lane;
            uint32_t old = 0;
            if (valid && lane == leader) {
                old = m.wc[dg * ONW + warp];
                m.wc[dg * ONW + warp] = old + __popc(peers);
            }
            old = __shfl_sync(FULL, old, leader);
            __syncwarp();
            lr[j] = old + __popc(peers & lanemask_lt());
            kk[j] = key;
        }
        if (threadIdx.x < 256) m.hrow[threadIdx.x] = hv;
        if (threadIdx.x == 0 && has_next) {
            const uint32_t *nk;
            const TV *nv;
            uint32_t *dk2;
            TV *dv2;
            pass_buffers<TV>(a, pass, rn, nk, nv, dk2, dv2);
            prefetch_tuples_l2(nk, rn.start, rn.len);
            prefetch_tuples_l2(nv, rn.start, rn.len);
        }
        __syncthreads();
        // per digit: exclusive prefix over warps (stable order inside the chunk), digit total
        if (threadIdx.x < 256) {
            uint32_t run = 0;
            for (int w = 0; w < ONW; ++w) {
                const uint32_t v = m.wc[threadIdx.x * ONW + w];
                m.wc[threadIdx.x * ONW + w] = run;
                run += v;
            }
            m.cbase[threadIdx.x] = run;
        }
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the digit totals: 8 digits per lane
            uint32_t t[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                t[j] = m.cbase[lane * 8 + j];
                sum += t[j];
            }
            uint32_t pre = warp_inclusive_scan(sum) - sum;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int d = lane * 8 + j;
                m.cbase[d] = pre;
                m.gbase[d] = (int64_t)m.hrow[d] - pre;
                pre += t[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < OE; ++j) {
            const int64_t q = warp * OWS + j * 32 + lane;
            if (q < r.len) {
                const uint32_t dg = (kk[j] >> shift) & 255u;
                const uint32_t local = m.cbase[dg] + m.wc[dg * ONW + warp] + lr[j];
                m.sk[local] = kk[j];
                m.sv[local] = vv[j];
            }
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < r.len; i += OT) {
            const uint32_t key = m.sk[i];
            const int64_t g = m.gbase[(key >> shift) & 255u] + i;
            dk[g] = key;
            dv[g] = m.sv[i];
        }
        __syncthreads();
    }
}

// Number of merged entries of each oversize bin = number of run heads.
__global__ void __launch_bounds__(OT) k_over_heads(const OversizeArgs a, int passes) {
    __shared__ int64_t scratch[40];
    const int64_t c_hi = over_c_hi(a);
    for (int64_t c = a.c_lo + blockIdx.x; c < c_hi; c += gridDim.x) {
        const ChunkRef r = chunk_ref(a, c);
        const uint32_t *k = (passes & 1) ? a.skeys + r.scr_base : a.keys + r.main_base;
        int64_t heads = 0;
        for (int64_t q = threadIdx.x; q < r.len; q += OT) {
            const int64_t p = r.start + q;
            heads += (p == 0 || k[p] != k[p - 1]) ? 1 : 0;
        }
        heads = block_reduce_sum<int64_t, OT>(heads, scratch);
        if (threadIdx.x == 0 && heads) atomicAdd(reinterpret_cast<unsigned long long *>(&a.over_u[r.o]),
                                                 (unsigned long long)heads);
    }
}


// Rows of the panel by decreasing size class (leading zeros of the tuple count):
// the dense and emit kernels take rows in this order through a ticket, so the
// largest start first and the rest fill in around them (longest-first list
// scheduling within a factor of two).
__device__ inline int over_size_class(const OversizeArgs &a, int64_t o) {
    const int64_t bin = a.over_bin[o];
    const int64_t N = a.R[a.bin_row[bin + 1]] - a.R[a.bin_row[bin]];
    return __clzll((long long)(N > 0 ? N : 1));
}

__global__ void k_over_order_count(const OversizeArgs a) {
    const int64_t o_hi = over_o_hi(a);
    for (int64_t o = a.o_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < o_hi;
         o += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&a.order_cnt[over_size_class(a, o)], 1u);
}

__global__ void k_over_order_place(const OversizeArgs a) {
    __shared__ uint32_t start[64];
    if (threadIdx.x < 64) {
        uint32_t s = 0;
        for (int k = 0; k < (int)threadIdx.x; ++k) s += a.order_cnt[k];
        start[threadIdx.x] = s;
    }
    __syncthreads();
    const int64_t o_hi = over_o_hi(a);
    for (int64_t o = a.o_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < o_hi;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int c = over_size_class(a, o);
        a.row_order[start[c] + atomicAdd(&a.order_cnt[64 + c], 1u)] = (int32_t)(o - a.o_lo);
    }
}

// ---------------------------------------------------------------------------
// Dense tiles for oversize rows.  After one partition pass on the column's top
// digit (column >> dense_shift), the tuples of an oversize row with digit d form
// one contiguous segment of the scratch buffer.  A CTA takes one row at a time
// (through a ticket, largest size class first) and walks its segments in digit
// order, a round of whole digits of up to 4096 columns at a time; it sums each
// round into a dense shared-memory tile of FP64 accumulators with presence flags
// (every structural entry is kept, exact-zero sums included) and writes the
// merged entries back in column order right after those of the previous rounds.
// The compaction goes by warp and slab (lanes on consecutive columns), so it
// reads the tile without bank conflicts and writes coalesced.  The row's merged,
// sorted entries (Sec. III-E) thus end up contiguous at the start of its
// scratch region without a sort (with FP32 tuples the FP64 sums go to the row's
// free region of the main tuple buffer instead; see OversizeArgs::wide).  The
// order of the sums within a column is not fixed (shared-memory atomics), so
// deterministic mode keeps the radix sort.
// ---------------------------------------------------------------------------
constexpr int DT = 256;  // threads per CTA of the dense kernels
// (slab, warp) counters of the compaction: up to 2^OVER_DENSE_MAX_SHIFT columns per round
constexpr int DENSE_WCNT = ((1 << OVER_DENSE_MAX_SHIFT) / DT) * (DT / 32);

template <class TV>
__global__ void __launch_bounds__(DT) k_over_dense(const OversizeArgs a, int group) {
    extern __shared__ __align__(16) unsigned char sraw[];
    const int w = a.dense_shift;
    const int W = group << w;  // a round covers `group` consecutive digits
    double *acc = reinterpret_cast<double *>(sraw);
    int64_t *offs = reinterpret_cast<int64_t *>(acc + W);           // [257] segment starts of the row
    int64_t *scratch = offs + 264;
    uint32_t *wtot = reinterpret_cast<uint32_t *>(scratch);          // merged entries of the round
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(scratch + 40);     // [W / DT * NWD] per (slab, warp)
    uint8_t *seen = reinterpret_cast<uint8_t *>(wcnt + DENSE_WCNT);  // presence of each column of the tile
    constexpr int NWD = DT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < W; i += DT) {
        acc[i] = 0.0;
        seen[i] = 0;
    }
    const int nslab = W / DT;  // W is a multiple of DT
    const int64_t o_hi = over_o_hi(a);
    __shared__ int64_t next_row;
    while (true) {
        // rows are taken through a ticket, largest size class first
        if (tid == 0) {
            const int64_t t = (int64_t)atomicAdd(&a.row_ticket[0], 1u);
            next_row = t < o_hi - a.o_lo ? a.o_lo + a.row_order[t] : o_hi;
        }
        __syncthreads();
        const int64_t o = next_row;
        if (o >= o_hi) break;
        const int64_t bin = a.over_bin[o];
        const int64_t N = a.R[a.bin_row[bin + 1]] - a.R[a.bin_row[bin]];
        const int64_t c0 = a.over_chunk_off[o] - a.c_lo;  // the bin's first work item holds its digit offsets
        offs[tid] = over_hist(a)[c0 * 256 + tid];
        if (tid == 0) offs[256] = N;
        __syncthreads();
        uint32_t *xk = a.skeys + (a.over_tuple_off[o] - a.over_base);
        TV *xv = static_cast<TV *>(a.svals) + (a.over_tuple_off[o] - a.over_base);
        // FP64 merged values of FP32 tuples: the row's main-buffer region (see OversizeArgs::wide)
        const int64_t half = (N + 1) / 2;
        double *wa = reinterpret_cast<double *>(a.keys + (a.bin_off[bin] - a.tuple_base));
        double *wb = reinterpret_cast<double *>(static_cast<TV *>(a.vals) + (a.bin_off[bin] - a.tuple_base));
        int64_t run = 0;  // merged entries written so far (the row's output is compacted to its start)
        for (int d = 0; d < 256; d += group) {
            const int64_t start = offs[d], end = offs[min(d + group, 256)];
            if (start >= end) continue;
            const uint32_t base = (uint32_t)d << w;
            for (int64_t q = start + tid; q < end; q += DT) {
                const uint32_t loc = xk[q] - base;
                atomicAdd(&acc[loc], (double)xv[q]);
                seen[loc] = 1;  // every writer stores the same value
            }
            __syncthreads();
            // Compaction in column order.  Warp v owns column sl*DT + v*32 + lane of
            // each slab sl of DT columns: lanes touch consecutive flags and
            // accumulators (no bank conflicts) and write consecutive output slots.
            for (int sl = 0; sl < nslab; ++sl) {
                const uint32_t m = __ballot_sync(FULL, seen[sl * DT + tid] != 0);
                if (lane == 0) wcnt[sl * NWD + wid] = (uint32_t)__popc(m);
            }
            __syncthreads();
            if (wid == 0) {  // exclusive scan of the (slab, warp) counts, i.e. in column order
                const int n = nslab * NWD, k = (n + 31) / 32;
                uint32_t sum = 0;
                for (int j = 0; j < k; ++j) sum += (lane * k + j < n) ? wcnt[lane * k + j] : 0u;
                uint32_t pre = warp_inclusive_scan(sum) - sum;
                for (int j = 0; j < k; ++j) {
                    if (lane * k + j < n) {
                        const uint32_t v = wcnt[lane * k + j];
                        wcnt[lane * k + j] = pre;
                        pre += v;
                    }
                }
                if (lane == 31) *wtot = pre;
            }
            __syncthreads();
            // output positions never pass the round's own end: run + *wtot <= end
            for (int sl = 0; sl < nslab; ++sl) {
                const int i = sl * DT + tid;
                const bool on = seen[i] != 0;
                const uint32_t m = __ballot_sync(FULL, on);
                if (on) {
                    const int64_t pos = run + wcnt[sl * NWD + wid] + __popc(m & lanemask_lt());
                    xk[pos] = base + (uint32_t)i;
                    if (a.wide)
                        *(pos < half ? wa + pos : wb + (pos - half)) = acc[i];
                    else
                        xv[pos] = (TV)acc[i];
                    acc[i] = 0.0;
                    seen[i] = 0;
                }
            }
            run += *wtot;
            __syncthreads();
        }
        if (tid == 0) a.over_u[o] = run;
        // every thread has read this row's offsets (trailing empty rounds included)
        // and its ticket before the next row's are stored
        __syncthreads();
    }
}

// Position of the r-th (from 0) set bit of x; x has more than r set bits.
__device__ inline uint32_t select_bit(uint32_t x, uint32_t r) {
    uint32_t pos = 0, c = __popc(x & 0xffffu);
    if (r >= c) { r -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xffu);
    if (r >= c) { r -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xfu);
    if (r >= c) { r -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (r >= c) { r -= c; x >>= 2; pos += 2; }
    if (r >= (x & 1u)) pos += 1;
    return pos;
}

// First round at or after digit d that holds tuples (256 when none is left).
__device__ inline int next_round(const int64_t *offs, int d, int group) {
    while (d < 256 && offs[d] >= offs[min(d + group, 256)]) d += group;
    return d;
}

constexpr int DPF = 4;  // tuples per thread of the next round loaded during a compaction

// The dense tiles for rounds of at most 8192 columns, with a presence bitmap
// (one 32-column word per thread) instead of a flag per column.  Compaction
// costs what the round holds, not the tile width: the words' set-bit counts
// are scanned, and output entry j (written by thread j mod DT, so the stores
// are coalesced) finds its word by binary search over the prefix and its
// column by selecting the bit.  The first tuples of the next round are loaded
// into registers before the compaction, so their latency overlaps it.  (R-MAT
// hub rows spread over many sparse rounds: at scale 20 a 4096-column round
// holds a few hundred tuples.)
template <class TV>
__global__ void __launch_bounds__(DT) k_over_dense_bm(const OversizeArgs a, int group) {
    extern __shared__ __align__(16) unsigned char sraw[];
    const int w = a.dense_shift;
    const int W = group << w;  // a round covers `group` consecutive digits; W <= 8192
    const int NWORD = W >> 5;  // <= DT
    constexpr int NWD = DT / 32;
    double *acc = reinterpret_cast<double *>(sraw);
    int64_t *offs = reinterpret_cast<int64_t *>(acc + W);      // [257] segment starts of the row
    uint32_t *bm = reinterpret_cast<uint32_t *>(offs + 264);   // [NWORD] columns touched by the round
    uint32_t *bmc = bm + DT;                                   // [NWORD] the round's words, for the compaction
    uint32_t *pre = bmc + DT;                                  // [NWORD + 1] set bits before each word
    uint32_t *wsum = pre + DT + 8;                             // [NWD] per-warp totals of the word scan
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < W; i += DT) acc[i] = 0.0;
    if (tid < NWORD) bm[tid] = 0;
    const int64_t o_hi = over_o_hi(a);
    __shared__ int64_t next_row;
    while (true) {
        // rows are taken through a ticket, largest size class first
        if (tid == 0) {
            const int64_t t = (int64_t)atomicAdd(&a.row_ticket[0], 1u);
            next_row = t < o_hi - a.o_lo ? a.o_lo + a.row_order[t] : o_hi;
        }
        __syncthreads();
        const int64_t o = next_row;
        if (o >= o_hi) break;
        const int64_t bin = a.over_bin[o];
        const int64_t N = a.R[a.bin_row[bin + 1]] - a.R[a.bin_row[bin]];
        const int64_t c0 = a.over_chunk_off[o] - a.c_lo;  // the bin's first work item holds its digit offsets
        offs[tid] = over_hist(a)[c0 * 256 + tid];
        if (tid == 0) offs[256] = N;
        __syncthreads();
        uint32_t *xk = a.skeys + (a.over_tuple_off[o] - a.over_base);
        TV *xv = static_cast<TV *>(a.svals) + (a.over_tuple_off[o] - a.over_base);
        // FP64 merged values of FP32 tuples: the row's main-buffer region (see OversizeArgs::wide)
        const int64_t half = (N + 1) / 2;
        double *wa = reinterpret_cast<double *>(a.keys + (a.bin_off[bin] - a.tuple_base));
        double *wb = reinterpret_cast<double *>(static_cast<TV *>(a.vals) + (a.bin_off[bin] - a.tuple_base));
        int64_t run = 0;  // merged entries written so far (the row's output is compacted to its start)
        uint32_t pk[DPF];
        TV pv[DPF];
        auto prefetch = [&](int d) {
#pragma unroll
            for (int j = 0; j < DPF; ++j) {
                const int64_t q = offs[d] + j * DT + tid;
                if (d < 256 && q < offs[min(d + group, 256)]) {
                    pk[j] = xk[q];
                    pv[j] = xv[q];
                }
            }
        };
        int d = next_round(offs, 0, group);
        prefetch(d);
        while (d < 256) {
            const int64_t start = offs[d], end = offs[min(d + group, 256)];
            const uint32_t base = (uint32_t)d << w;
#pragma unroll
            for (int j = 0; j < DPF; ++j) {
                if (start + j * DT + tid < end) {
                    const uint32_t loc = pk[j] - base;
                    atomicAdd(&acc[loc], (double)pv[j]);
                    atomicOr(&bm[loc >> 5], 1u << (loc & 31u));
                }
            }
            for (int64_t q = start + DPF * DT + tid; q < end; q += DT) {
                const uint32_t loc = xk[q] - base;
                atomicAdd(&acc[loc], (double)xv[q]);
                atomicOr(&bm[loc >> 5], 1u << (loc & 31u));
            }
            // the next round's first tuples lie past this round's end, where no output goes
            const int d2 = next_round(offs, d + group, group);
            prefetch(d2);
            __syncthreads();
            // compaction: exclusive scan of the words' set-bit counts
            uint32_t c = 0;
            if (tid < NWORD) {
                const uint32_t bits = bm[tid];
                bm[tid] = 0;
                bmc[tid] = bits;
                c = (uint32_t)__popc(bits);
            }
            const uint32_t inc = warp_inclusive_scan(c);
            if (lane == 31) wsum[wid] = inc;
            __syncthreads();
            uint32_t wbase = 0, tot = 0;
#pragma unroll
            for (int k = 0; k < NWD; ++k) {
                const uint32_t t = wsum[k];
                wbase += (k < wid) ? t : 0u;
                tot += t;
            }
            if (tid < NWORD) pre[tid] = wbase + inc - c;
            if (tid == 0) pre[NWORD] = tot;
            __syncthreads();
            // output positions never pass the round's own end: run + tot <= end
            for (uint32_t j = tid; j < tot; j += DT) {
                int lo = 0, hi = NWORD;  // pre[lo] <= j < pre[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[mid] <= j)
                        lo = mid;
                    else
                        hi = mid;
                }
                const uint32_t col = ((uint32_t)lo << 5) + select_bit(bmc[lo], j - pre[lo]);
                const int64_t pos = run + j;
                xk[pos] = base + col;
                if (a.wide)
                    *(pos < half ? wa + pos : wb + (pos - half)) = acc[col];
                else
                    xv[pos] = (TV)acc[col];
                acc[col] = 0.0;
            }
            run += tot;
            d = d2;
            __syncthreads();  // the tile is clear and the words are free for the next round
        }
        if (tid == 0) a.over_u[o] = run;
        // every thread has read this row's offsets and its ticket before the next row's are stored
        __syncthreads();
    }
}

// Columns of one dense round: consecutive digits grouped up to this width.
constexpr int DENSE_ROUND_COLUMNS = 4096;

template <class TV>
cudaError_t run_dense(const OversizeArgs &a, int num_sms, cudaStream_t s) {
    int group = DENSE_ROUND_COLUMNS >> a.dense_shift;
    if (group < 1) group = 1;
    if (group > 256) group = 256;
    const int W = group << a.dense_shift;
    // rounds of up to 8192 columns use the bitmap form (one word per thread)
    const bool bitmap = W <= 32 * DT;
    const size_t smem = bitmap ? 8 * (size_t)W + 8 * 264 + 4 * (3 * (size_t)DT + 8 + 32)
                               : 8 * (size_t)W + 8 * (264 + 40) + 4 * (size_t)DENSE_WCNT + (size_t)((W + 15) & ~15);
    auto kern = bitmap ? k_over_dense_bm<TV> : k_over_dense<TV>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    const int64_t rows = a.o_hi - a.o_lo;
    if (grid > rows) grid = rows;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, DT, smem, s>>>(a, group);
    count_launches(1);
    return cudaGetLastError();
}

// Copy each oversize row's merged entries (compacted to the start of its
// scratch region) to C at the offset the sort kernel recorded; CTA per row.
template <class TV, class OV, bool WIDE>
__global__ void __launch_bounds__(256) k_over_emit(const OversizeArgs a) {
    const int64_t o_hi = over_o_hi(a);
    __shared__ int64_t next_row;
    while (true) {
        if (threadIdx.x == 0) {
            const int64_t t = (int64_t)atomicAdd(&a.row_ticket[1], 1u);
            next_row = t < o_hi - a.o_lo ? a.o_lo + a.row_order[t] : o_hi;
        }
        __syncthreads();
        const int64_t o = next_row;
        __syncthreads();  // every thread has its row before the ticket word is reused
        if (o >= o_hi) break;
        const int64_t P = a.over_p[o];
        if (P < 0) continue;
        const int64_t U = a.over_u[o];
        const int64_t bin = a.over_bin[o];
        const uint32_t *xk = a.skeys + (a.over_tuple_off[o] - a.over_base);
        int32_t *colidxC = a.colidxC;
        OV *valC = static_cast<OV *>(a.valC);
        if (a.desc) {  // batch: the row's product's C
            const BatchDesc &d = a.desc[a.bin_prod[bin]];
            colidxC = d.colidxC;
            valC = static_cast<OV *>(d.valC);
        }
        if (WIDE) {
            const int64_t half = (a.R[a.bin_row[bin + 1]] - a.R[a.bin_row[bin]] + 1) / 2;
            const double *wa = reinterpret_cast<const double *>(a.keys + (a.bin_off[bin] - a.tuple_base));
            const double *wb =
                reinterpret_cast<const double *>(static_cast<const TV *>(a.vals) + (a.bin_off[bin] - a.tuple_base));
            for (int64_t i = threadIdx.x; i < U; i += blockDim.x) {
                colidxC[P + i] = (int32_t)xk[i];
                valC[P + i] = (OV)(i < half ? wa[i] : wb[i - half]);
            }
        } else {
            const TV *xv = static_cast<const TV *>(a.svals) + (a.over_tuple_off[o] - a.over_base);
            for (int64_t i = threadIdx.x; i < U; i += blockDim.x) {
                colidxC[P + i] = (int32_t)xk[i];
                valC[P + i] = (OV)xv[i];
            }
        }
    }
}
template <class TV>
cudaError_t run_oversize(const OversizeArgs &a, int passes, int num_sms, cudaStream_t s) {
    const int64_t g4 = (int64_t)num_sms * 4, g8 = (int64_t)num_sms * 8;
    const int64_t nc = a.c_hi - a.c_lo, no = a.o_hi - a.o_lo;
    const unsigned grid = (unsigned)(nc < g4 ? nc : g4);
    const unsigned ogrid = (unsigned)(no < g8 ? no : g8);
    cudaError_t e = cudaMemsetAsync(a.over_u + a.o_lo, 0, 8 * (size_t)no, s);
    if (e != cudaSuccess) return e;
    if (a.cinfo) {
        k_over_chunk_info<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(a);
        count_launches(1);
    }
    e = cudaFuncSetAttribute(k_over_scatter<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ScatterSmem<TV>));
    if (e != cudaSuccess) return e;
    if (a.dense) {
        // one partition pass on the top digit, then dense accumulation per segment
        k_over_hist<TV><<<grid, OT, 0, s>>>(a, 0, a.dense_shift);
        k_over_offsets<<<ogrid, 256, 0, s>>>(a);
        k_over_scatter<TV><<<grid, OT, sizeof(ScatterSmem<TV>), s>>>(a, 0, a.dense_shift);
        if ((e = cudaMemsetAsync(a.order_cnt, 0, 512, s)) != cudaSuccess) return e;
        k_over_order_count<<<ogrid, 256, 0, s>>>(a);
        k_over_order_place<<<ogrid, 256, 0, s>>>(a);
        count_launches(5);
        return run_dense<TV>(a, num_sms, s);
    }
    for (int pass = 0; pass < passes; ++pass) {
        k_over_hist<TV><<<grid, OT, 0, s>>>(a, pass, 8 * pass);
        k_over_offsets<<<ogrid, 256, 0, s>>>(a);
        k_over_scatter<TV><<<grid, OT, sizeof(ScatterSmem<TV>), s>>>(a, pass, 8 * pass);
        count_launches(3);
    }
    k_over_heads<<<grid, OT, 0, s>>>(a, passes);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_oversize(const OversizeArgs &a, int passes, int dtype, int num_sms, cudaStream_t s) {
    if (a.o_hi <= a.o_lo) return cudaSuccess;
    if (dtype == PB_F64) return run_oversize<double>(a, passes, num_sms, s);
    return run_oversize<float>(a, passes, num_sms, s);
}

cudaError_t launch_oversize_emit(const OversizeArgs &a, int dtype, int num_sms, cudaStream_t s) {
    if (a.o_hi <= a.o_lo || !a.dense) return cudaSuccess;
    const int64_t rows = a.o_hi - a.o_lo;
    int64_t grid = (int64_t)num_sms * 8;
    if (grid > rows) grid = rows;
    switch (dtype) {
        case PB_F64: k_over_emit<double, double, false><<<(unsigned)grid, 256, 0, s>>>(a); break;
        case PB_F32: k_over_emit<float, float, false><<<(unsigned)grid, 256, 0, s>>>(a); break;
        case PB_F64_F32TUPLE: k_over_emit<float, double, true><<<(unsigned)grid, 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pb
