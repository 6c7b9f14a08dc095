// Internal definitions shared by the CUDA translation units of libpbspgemm.
// Nothing here is part of the public ABI (include/pb_spgemm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pb_spgemm.h"

namespace pb {

constexpr unsigned FULL = 0xffffffffu;

// Device status word bits (pb_plan_status maps the lowest set bit to a pb_status).
enum : uint32_t {
    DEV_ERR_OVERFLOW = 1u << 0,   // nnz(C) > C.cap or an int32 row pointer would overflow
    DEV_ERR_TIMEOUT = 1u << 1,    // a bounded wait (look-back, mbarrier) gave up
    DEV_ERR_CAPACITY = 1u << 2,   // a bin held more tuples than the plan sized it for
    DEV_ERR_WORKSPACE = 1u << 3,  // batch: the tuples do not fit the caller's workspace
    DEV_ERR_HEAVY_ROW = 1u << 4,  // batch: one row has more tuples than its bin capacity
};
// Errors after which the batched kernels do no further work.
constexpr uint32_t DEV_ERR_BATCH_FATAL = DEV_ERR_WORKSPACE | DEV_ERR_HEAVY_ROW;

// The pb_status a device status word reports (one mapping for every entry
// point): errors that stop the work first, then overflow, timeout, capacity.
__host__ __device__ inline pb_status status_of_word(uint32_t w) {
    if (w & DEV_ERR_HEAVY_ROW) return PB_ERR_UNSUPPORTED;
    if (w & DEV_ERR_WORKSPACE) return PB_ERR_WORKSPACE;
    if (w & DEV_ERR_OVERFLOW) return PB_ERR_OVERFLOW;
    if (w & DEV_ERR_TIMEOUT) return PB_ERR_TIMEOUT;
    if (w & DEV_ERR_CAPACITY) return PB_ERR_UNSUPPORTED;  // operands differ from the plan's structure
    return PB_OK;
}

// Look-back status of one bin: two flag bits over a 62-bit count.
constexpr uint64_t LB_FLAG_SHIFT = 62;
constexpr uint64_t LB_AGGREGATE = 1ull << LB_FLAG_SHIFT;
constexpr uint64_t LB_PREFIX = 2ull << LB_FLAG_SHIFT;
constexpr uint64_t LB_VALUE_MASK = (1ull << LB_FLAG_SHIFT) - 1;

// Bounded spin: every device wait gives up after this many polls.  A test
// build lowers it (PB_SPIN_LIMIT) to make a wait run out quickly.
#ifndef PB_SPIN_LIMIT
#define PB_SPIN_LIMIT (1u << 24)
#endif
constexpr uint32_t SPIN_LIMIT = PB_SPIN_LIMIT;

// Words between two bins' expand cursors in a single product's workspace.
#ifndef PB_CURSOR_STRIDE
#define PB_CURSOR_STRIDE 1
#endif

// Tuples per work item of the oversize-bin sort.
constexpr int OVER_CHUNK = 4096;

// A bin spans at most 2^RMAX_LOG2 rows (fewer when the column bits leave less
// room in the 32-bit key).
constexpr int RMAX_LOG2 = 11;

// Plan header filled on the device by the symbolic phase, read back once.
struct PlanHeader {
    int64_t flop;
    int64_t nbins;
    int64_t tuples_padded;   // sum over bins of round_up(count, 4)
    unsigned long long max_bin_count;
    unsigned long long max_light_row;  // largest per-row flop among rows <= heavy threshold
    int64_t n_oversize;      // bins holding more than bin_capacity tuples
    int64_t over_chunks;     // OVER_CHUNK-tuple work items over all oversize bins
    int64_t over_tuples;     // sum over oversize bins of round_up(count, 4)
};

// Arguments of the kernels (passed by value).
struct SymbolicArgs {
    int32_t m, k, n;
    const int32_t *colptrA, *rowidxA, *rowptrB;
    int64_t *F;          // [k+1]
    int64_t *R;          // [m+1]
    int64_t *flags;      // [m+1] scratch: bin-start flags, then their exclusive scan
    uint64_t *rowinfo;   // [m]   (bin << 32) | (local_row << colbits)
    uint64_t *ainfo;     // [nnzA] rowinfo of each A entry's row
    int32_t *acol;       // [nnzA] column of each A entry
    int2 *aspan;         // [nnzA] B(k,:) of each A entry (column k): (first entry, length)
    int32_t *long_cols;  // [k] scratch: columns with many entries
    uint32_t *n_long;    // [1] scratch counter
    int64_t nnzA;
    int32_t *bin_row;    // [m+2]
    int64_t *bin_off;    // [m+2]
    PlanHeader *hdr;
    int32_t colbits, rmax_log2;
    int64_t capacity, heavy;
    // oversize-bin lists (upper bound m+1 entries each)
    int64_t *over_scan;       // exclusive index of each bin among oversize bins
    int64_t *over_bin;        // bin id of oversize bin o
    int64_t *over_chunk_off;  // first work item of oversize bin o
    int64_t *over_tuple_off;  // scratch offset of oversize bin o
};

struct BatchDesc;

// Where one OVER_CHUNK-tuple work item of an oversize bin reads and writes
// (one 32-byte load instead of a chain of dependent list lookups).
struct __align__(16) OverChunk {
    int64_t main_base;  // the bin's first tuple in the main buffer (index into keys / vals)
    int64_t scr_base;   // the bin's first tuple in the scratch buffer (index into skeys / svals)
    int64_t start;      // the work item's first tuple within the bin
    int32_t len, o;     // its tuples; its oversize bin
};

struct OversizeArgs {
    const int64_t *R;
    const int32_t *bin_row;
    const int64_t *bin_off;
    const int64_t *over_bin, *over_chunk_off, *over_tuple_off;
    const int32_t *over_chunk_bin;  // [over_chunks] oversize bin of each work item
    int64_t n_over, over_chunks;
    uint32_t *keys;
    void *vals;
    uint32_t *skeys;
    void *svals;
    uint32_t *hist;   // [(c_hi - c_lo) * 256]
    int64_t *over_u;  // [n_over] merged entries of each oversize bin
    // the panel being processed: oversize bins [o_lo, o_hi), their work items
    // [c_lo, c_hi); tuple offsets are relative to tuple_base (main buffer) and
    // over_base (scratch)
    int64_t o_lo, o_hi, c_lo, c_hi, tuple_base, over_base;
    // dense tiles instead of the radix sort: one partition pass on the column's
    // top digit (columns >> dense_shift), then per row a dense accumulation of
    // each tile of 2^dense_shift columns in shared memory
    int dense;
    int dense_shift;
    // FP32 tuples merged into FP64 values (PB_F64_F32TUPLE): the dense kernel
    // writes a row's merged values to the row's region of the main tuple buffer,
    // free after the partition pass, as FP64 positions [0, h) over its key array
    // and [h, U) over its value array, h = (N + 1) / 2 (N tuples, U merged)
    int wide;
    uint32_t *row_ticket;  // [2] zeroed per panel: rows taken in order by the dense and emit kernels
    int32_t *row_order;    // [o_hi - o_lo] the panel's rows (minus o_lo) by decreasing size class
    uint32_t *order_cnt;   // [128] per size class: rows, then rows placed
    int64_t *over_p;    // [n_over] C offset of each oversize row (-1: not written)
    int32_t *colidxC;   // C, for the copy of the segments once the offsets are known
    void *valC;
    // Batches find their oversize rows on the device: dev_count[0] oversize bins,
    // dev_count[1] work items (o_lo = c_lo = 0; o_hi and c_hi are then upper
    // bounds that only size the grids), dev_count[2] the offset in `keys` of
    // the work items' histograms (hist is unused), and each row's C is its
    // product's (desc[bin_prod[bin]]).  Null for a single product.
    const int64_t *dev_count;
    const BatchDesc *desc;
    const int32_t *bin_prod;
    // [c_hi - c_lo] the work items' places, filled by launch_oversize before the
    // passes (null: each pass looks them up in the lists)
    OverChunk *cinfo;
};

template <class T>
__host__ __device__ inline T ceil_div(T a, T b) { return (a + b - 1) / b; }

__device__ inline uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ inline void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ inline uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (TMA, non-tensor form) helpers.
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false on timeout.
__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < SPIN_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    return false;
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses of the same CTA.
__device__ inline void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned,
// bytes a multiple of 16.
__device__ inline void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Prefetch `bytes` (a multiple of 16) at a 16-byte aligned global address into L2.
__device__ inline void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Block-wide scans.
// ---------------------------------------------------------------------------
template <class T>
__device__ inline T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; returns the prefix,
// writes the block total to *total.  `scratch` holds >= 33 elements.
template <class T, int THREADS>
__device__ inline T block_exclusive_scan(T v, T *scratch, T *total) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < NW) ? scratch[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < NW) scratch[lane] = wi - w;
        if (lane == NW - 1) scratch[32] = wi;
    }
    __syncthreads();
    T res = scratch[warp] + inc - v;
    *total = scratch[32];
    __syncthreads();
    return res;
}

template <class T, int THREADS>
__device__ inline T block_reduce_sum(T v, T *scratch) {
    T total;
    (void)block_exclusive_scan<T, THREADS>(v, scratch, &total);
    return total;
}

// Host-side launch of the device-wide int64 exclusive scan (pb_scan.cu).
// Scans x[0..n) in place and writes the total to x[n].  tmp must hold
// scan_tmp_elems(n) int64 elements.
int64_t scan_tmp_elems(int64_t n);
cudaError_t scan_i64(int64_t *x, int64_t n, int64_t *tmp, cudaStream_t s);

// Operand checks of pb_validate_operands; sets bits 1/2 (A.colptr / B.rowptr not
// a valid pointer array), 4 (A.rowidx out of range), 8 (B.colidx out of range).
cudaError_t launch_validate(const pb_csc &A, const pb_csr &B, uint32_t *bad, cudaStream_t s);

// Process-wide count of kernels launched by the library (pb_kernel_launches).
void count_launches(int64_t n);

// Kernel launchers implemented in the other translation units.
cudaError_t launch_symbolic(const SymbolicArgs &a, int64_t *scan_tmp, cudaStream_t s);
cudaError_t launch_symbolic_oversize(const SymbolicArgs &a, int64_t *scan_tmp, cudaStream_t s);
// Per-A-entry pass after the sizes are known: ainfo and the expand work items.
cudaError_t launch_chunk_table(const SymbolicArgs &a, int64_t nchunks, int64_t chunk, int32_t *chunk_e,
                               cudaStream_t s);
cudaError_t launch_over_chunk_map(const int64_t *over_chunk_off, int64_t n_over, int32_t *over_chunk_bin,
                                  cudaStream_t s);
cudaError_t launch_oversize(const OversizeArgs &a, int passes, int dtype, int num_sms, cudaStream_t s);
// Dense mode: copy every oversize row's compacted segments to C at the offsets
// the sort kernel recorded (after the sort kernel of the panel).
cudaError_t launch_oversize_emit(const OversizeArgs &a, int dtype, int num_sms, cudaStream_t s);
// Largest dense_shift (tile of 2^shift columns) the dense oversize path handles.
constexpr int OVER_DENSE_MAX_SHIFT = 14;

// ---------------------------------------------------------------------------
// Batched products (pb_spgemm_batch).  The products are laid out back to back
// in three global index spaces: rows (of A and C), columns of A (= rows of B)
// and A entries.  Each space is cut into tiles of BATCH_TILE elements that never
// straddle two products; tile_*[p] is the first tile of product p.
// ---------------------------------------------------------------------------
constexpr int BATCH_TILE = 1024;
constexpr int BATCH_MIN_CAPACITY = 2048;  // smallest bin capacity a batched product can be tuned to

struct BatchDesc {
    const int32_t *colptrA, *rowidxA;
    const void *valA;
    const int32_t *rowptrB, *colidxB;
    const void *valB;
    int64_t *rowptr64;
    int32_t *rowptr32;
    int32_t *colidxC;
    void *valC;
    int64_t *nnz_dev;
    int64_t capC;
    int32_t m, k, n, nnzA;
    int32_t mstart, kstart, estart;  // first global row, column and A entry
    int32_t colbits, rmax_log2, capacity, chunk, level;
    int32_t over_ok;  // rows above the capacity may be merged in dense tiles (B.ncols <= 2^(8 + OVER_DENSE_MAX_SHIFT))
};

// Per-product values found on the device.
struct BatchProd {
    int64_t flop;
    unsigned long long max_light;  // largest row flop <= capacity / 2
    unsigned long long max_row;    // largest row flop
    int64_t first_bin;
    int64_t chunk_base;            // first expand work item
    int64_t over_bound;            // sum of round_up(r, 4) over rows with r > BATCH_MIN_CAPACITY tuples
};

struct BatchHeader {
    int64_t nbins;
    int64_t nchunks;
    int64_t tuples;                // padded tuple slots used
    int64_t level_bins[8];         // bins of capacity level l: [level_bins[l], level_bins[l+1])
};

struct NumericArgs {
    // inputs
    int32_t m, k, n;
    const int32_t *colptrA, *rowidxA, *rowptrB, *colidxB;
    const void *valA, *valB;
    // plan
    const int64_t *F, *R;
    const uint64_t *ainfo;  // [nnzA] bin << 32 | key high part, per A entry
    const int32_t *acol;    // [nnzA] column of each A entry
    const int2 *aspan;      // [nnzA] B(k,:) of each A entry: (first entry, length)
    const int32_t *bin_row;
    const int64_t *bin_off;
    const int32_t *chunk_e; // [nchunks+1] first A entry of each expand work item
    int64_t flop, nbins, nchunks, chunk;
    int32_t colbits;
    int32_t capacity;
    // the panel being processed: bins [bin_lo, bin_hi); the tuple buffer holds
    // tuples [tuple_base, tuple_base + panel size) of the whole product
    int64_t bin_lo, bin_hi, tuple_base, over_base;
    // workspace
    uint32_t *keys;
    void *vals;
    uint64_t *cursor;    // [nbins * cursor_stride] next free absolute slot of bin b at cursor[b * cursor_stride]
    int32_t cursor_stride;  // words between two bins' cursors (spreads the atomics over cache lines)
    uint64_t *status;    // [nbins] look-back words
    uint32_t *ticket;    // [1]
    uint32_t *work;      // [1] expand work items taken so far (zeroed before the expand)
    uint32_t *err;       // [1] device status word
    // output
    int64_t *rowptr64;
    int32_t *rowptr32;
    int32_t *colidx;
    void *valC;
    int64_t *nnz_dev;
    int64_t cap;
    int count_only;      // compute nnz(C) only: no writes to C except *nnz_dev
    int dtype;
    int num_sms;
    // oversize bins (sorted in global memory before the sort kernel)
    const int64_t *over_scan, *over_tuple_off;
    const int64_t *over_u;
    uint32_t *skeys;
    void *svals;
    int over_passes;
    int over_dense;     // oversize rows were accumulated in dense tiles: publish only
    int64_t *over_p;    // [n_over] C offset of each oversize row, written by the sort kernel
    // deterministic mode: the first tuple position of each A entry's run (null: atomic cursors)
    const int64_t *apos;
    // packed tuples (4-byte values only): tuple t is the 8-byte pair {key, value
    // bits} at keys[2t], keys[2t + 1]; the pairs fill the key and value regions
    // and `vals` is unused
    int packed;
    // batched products (null for a single product)
    const BatchDesc *desc;
    const int32_t *chunk_prod;  // [nchunks] product of each expand work item
    const int32_t *bin_prod;    // [nbins] product of each bin
    const BatchProd *prod;
    const BatchHeader *bhdr;    // device-side counts: nbins, nchunks, bin range of each level
    int32_t level;              // capacity level the sort launch serves
};

cudaError_t launch_expand(const NumericArgs &a, cudaStream_t s);

// Deterministic mode (pb_determ.cu): run positions fixed in CSC order inside each bin.
struct DetArgs {
    int64_t E, nbins;
    const uint64_t *ainfo;
    const int32_t *acol, *rowptrB, *bin_row;
    const int64_t *bin_off, *R;
    int64_t *apos;  // [E] output
};
int64_t det_scratch_bytes(int64_t E);
cudaError_t launch_det_positions(const DetArgs &d, void *scratch, int num_sms, cudaStream_t s);

cudaError_t launch_binsort(const NumericArgs &a, cudaStream_t s);
// Batched forms: work counts are read from a.bhdr on the device; the grids are
// persistent (sized from the SM count).
cudaError_t launch_expand_batch(const NumericArgs &a, cudaStream_t s);
cudaError_t launch_binsort_batch(const NumericArgs &a, cudaStream_t s);
int binsort_max_capacity(int dtype);

}  // namespace pb
