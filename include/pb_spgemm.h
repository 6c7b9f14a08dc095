/*
 * pb_spgemm.h -- C ABI of the GB300 PB-SpGEMM library (libpbspgemm.so).
 *
 * Computes C = A * B for sparse A (m x k, CSC) and B (k x n, CSR) with the
 * propagation-blocking outer-product method of Gu, Moreira, Edelsohn and Azad
 * (arXiv 2002.11302, Alg. 2):
 *   symbolic  Alg. 3 flop count per column/row k, plus the per-row flop count
 *             (Sec. III-B) that cuts rows into bins;
 *   expand    the outer products A(:,k) * B(k,:) become (key, value) tuples
 *             written into row-range bins (propagation blocking, Sec. III-A/C);
 *   sort      each bin is sorted on-chip by its packed (in-bin row, column) key
 *             (Sec. III-D);
 *   compress  equal keys are summed (Sec. III-E) and the merged bins are
 *             written in row order as CSR (ConvertCSR, Alg. 2).
 *
 * Conventions for every entry point:
 *   - All matrix and workspace pointers are DEVICE pointers owned by the
 *     caller.  The library never frees caller memory.  Host pointers are only
 *     the struct arguments themselves and the output scalars of query calls.
 *   - Index arrays are int32.  Input pointer arrays (colptr, rowptr) are int32
 *     and monotone with ptr[0] = 0.  Entry order inside a column of A or a row
 *     of B is arbitrary.  No duplicate (row, col) inside one operand.
 *   - Output C: column indices strictly ascending inside each row; every
 *     structural product is kept, including exact-zero sums (Sec. III-E
 *     merges without dropping).
 *   - Every call returns pb_status; nothing throws across the ABI.  A call
 *     that returns an error leaves its outputs unspecified.
 *     pb_last_error() gives a message for the last failing call on a handle.
 *   - Compute calls are asynchronous on the given stream unless stated.
 *     Errors detected on the device (capacity, overflow, bounded-wait
 *     timeout) are recorded in a device status word read by pb_plan_status
 *     after the stream has been synchronised.
 */
#ifndef PB_SPGEMM_H
#define PB_SPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pb_stream_t; /* same object as cudaStream_t; NULL = legacy default stream */

typedef enum pb_status {
    PB_OK = 0,
    PB_ERR_INVALID_ARG = 1,       /* null pointer, negative size, bad config value */
    PB_ERR_SHAPE = 2,             /* A.ncols != B.nrows, or C shape differs from m x n */
    PB_ERR_UNSUPPORTED_DTYPE = 3,
    PB_ERR_OOM = 4,               /* the allocator returned NULL */
    PB_ERR_OVERFLOW = 5,          /* nnz(C) exceeds C's capacity or an int32 row pointer */
    PB_ERR_CUDA = 6,              /* a CUDA runtime call failed (message in pb_last_error) */
    PB_ERR_TIMEOUT = 7,           /* a bounded device-side wait expired */
    PB_ERR_BUSY = 8,              /* a request can never be admitted under the server budget */
    PB_ERR_UNSUPPORTED = 9,       /* a size outside what this build handles (message says which) */
    PB_ERR_WORKSPACE = 10         /* workspace smaller than pb_plan_query reported */
} pb_status;

/* Value types.  Tuples are the intermediate (key, value) pairs of Alg. 2. */
typedef enum pb_dtype {
    PB_F64 = 0,          /* A, B, C values double; double tuples (12-byte tuples)              */
    PB_F32 = 1,          /* A, B, C values float; float products and tuples, merged in double  */
    PB_F64_F32TUPLE = 2  /* A, B, C values double; products rounded once to float in the tuple
                            (8-byte tuples), merged in double                                  */
} pb_dtype;

typedef struct pb_csc {   /* A: nrows x ncols, column j holds rowidx/val[colptr[j] .. colptr[j+1]) */
    int32_t nrows, ncols;
    int64_t nnz;
    const int32_t *colptr; /* device, ncols + 1 */
    const int32_t *rowidx; /* device, nnz */
    const void *val;       /* device, nnz values of the dtype's input type */
} pb_csc;

typedef struct pb_csr {   /* B: nrows x ncols, row i holds colidx/val[rowptr[i] .. rowptr[i+1]) */
    int32_t nrows, ncols;
    int64_t nnz;
    const int32_t *rowptr; /* device, nrows + 1 */
    const int32_t *colidx; /* device, nnz */
    const void *val;       /* device, nnz */
} pb_csr;

typedef struct pb_csr_out { /* C: nrows x ncols in CSR; exactly one of rowptr64/rowptr32 non-null */
    int32_t nrows, ncols;
    int64_t cap;           /* entries available in colidx / val; c_cap from pb_plan_query always suffices */
    int64_t *rowptr64;     /* device, nrows + 1 (int64 row pointer)                                  */
    int32_t *rowptr32;     /* device, nrows + 1 (int32 row pointer; PB_ERR_OVERFLOW if nnz >= 2^31)   */
    int32_t *colidx;       /* device, cap */
    void *val;             /* device, cap values of the dtype's output type */
    int64_t *nnz_dev;      /* device, 1 element receiving nnz(C); may be NULL */
} pb_csr_out;

/* Tunables.  Zero in any field selects the built-in default. */
typedef struct pb_config {
    int32_t bin_capacity;    /* max tuples of one bin sorted on-chip: 2048, 4096 (default) or 8192;
                                other values give PB_ERR_INVALID_ARG                             */
    int32_t sort_threads;    /* threads of one sort CTA: fixed at bin_capacity / 8 (256, 512, 1024);
                                0 or that value, anything else gives PB_ERR_INVALID_ARG           */
    int32_t expand_chunk;    /* tuples per expand work item                                     */
    int32_t deterministic;   /* nonzero: bitwise-reproducible values.  The plan fixes every A entry's
                                tuple positions (CSC order inside each bin) instead of atomic cursors,
                                and equal keys merge in position order, so every C(i,j) is summed over
                                ascending k, identically on every run (costs a stable sort of A's
                                entries in the symbolic phase and 8 bytes per entry of A in the plan) */
    int64_t max_tuple_bytes; /* cap on the tuple workspace (tuples plus the global-sort scratch of
                                oversize rows); a larger product runs in row panels, consecutive
                                bin ranges processed one after another                            */
    int64_t min_panels;      /* a product of at least min_panels * 2^20 tuples runs in about this many
                                row panels even when its tuples fit (lets pb_spgemm_host copy a
                                panel's rows of C back while the next panel computes); 0 or 1 = off */
} pb_config;

typedef struct pb_handle pb_handle;
typedef struct pb_plan pb_plan;

/* Device-memory provider used for plan-owned arrays.  alloc returns a device
 * pointer (256-byte aligned) or NULL; free releases it.  Both are stream
 * ordered on the stream passed.  Default: cudaMallocAsync / cudaFreeAsync. */
typedef void *(*pb_alloc_fn)(size_t bytes, pb_stream_t stream, void *ctx);
typedef void (*pb_free_fn)(void *ptr, size_t bytes, pb_stream_t stream, void *ctx);

/* Create a handle bound to the current CUDA device.  *h receives the handle. */
pb_status pb_create(pb_handle **h);
pb_status pb_destroy(pb_handle *h);
/* Replace the device-memory provider (NULL alloc restores the default). */
pb_status pb_set_allocator(pb_handle *h, pb_alloc_fn alloc, pb_free_fn free_fn, void *ctx);
/* Message for the last failing call on this handle ("" if none).  Owned by the handle. */
const char *pb_last_error(const pb_handle *h);
/* Library version as major*10000 + minor*100 + patch. */
int32_t pb_version(void);

/*
 * Symbolic phase (Alg. 3 and Sec. III-B): computes flop, the per-row flop
 * histogram and the row-range bins.  Launches on `stream`, then synchronises
 * it ONCE to read the sizes back.  The plan owns device arrays allocated
 * through the handle's allocator; it stays valid for numeric calls on any
 * A, B with the same sparsity structure (values may change).
 * cfg may be NULL.  Errors: INVALID_ARG, SHAPE, UNSUPPORTED_DTYPE, OOM, CUDA,
 * UNSUPPORTED (a key of row offset and column does not fit 32 bits).
 */
pb_status pb_spgemm_symbolic(pb_handle *h, const pb_csc *A, const pb_csr *B, pb_dtype dtype,
                             const pb_config *cfg, pb_stream_t stream, pb_plan **plan);

/* Sizes of a plan.  Any output pointer may be NULL.
 *   flop             total multiplications (Alg. 3)
 *   c_cap            entries C must hold (= flop, since nnz(C) <= flop)
 *   workspace_bytes  device workspace pb_spgemm_numeric needs
 *   nbins            number of bins (all panels)
 *   npanels          number of row panels (1 unless max_tuple_bytes forces more) */
pb_status pb_plan_query(const pb_plan *plan, int64_t *flop, int64_t *c_cap, size_t *workspace_bytes,
                        int64_t *nbins, int32_t *npanels);

/*
 * Numeric phase (Alg. 2 expand, sort, compress, ConvertCSR).  Asynchronous on
 * `stream`: no host synchronisation, no allocation.  `workspace` is a device
 * buffer of at least workspace_bytes, 256-byte aligned; it is scratch and may
 * be reused after the stream reaches this call's end.  A and B must have the
 * structure the plan was made from.  C->cap must be >= nnz(C) (c_cap always
 * suffices); otherwise the device records PB_ERR_OVERFLOW and writes nothing
 * past cap.  In every case *C->nnz_dev (if set) receives nnz(C).
 * Counting run: with C->cap == 0 and all four C arrays NULL the call writes
 * only *C->nnz_dev, so a caller can size C exactly before the real call.
 * Errors: INVALID_ARG, SHAPE, WORKSPACE, CUDA.
 */
pb_status pb_spgemm_numeric(pb_handle *h, const pb_plan *plan, const pb_csc *A, const pb_csr *B,
                            pb_csr_out *C, void *workspace, size_t ws_bytes, pb_stream_t stream);

/*
 * Product from and to HOST memory (the whole method, Alg. 3 then Alg. 2, with
 * the host<->device copies overlapped with the kernels).  A and B hold host
 * pointers (pinned memory gives full copy speed); C receives C = A * B in caller
 * host buffers.  The library allocates device copies of A and B, the plan, the
 * workspace and a flop-sized device C through the handle's allocator and frees
 * them before returning.  Overlap: A's and B's value arrays and B's column
 * indices are copied on a second stream while the symbolic phase runs; the
 * numeric phase runs in row panels (cfg->min_panels, default 6 when 0) and each
 * panel's rows of C are copied back as soon as its sort has finished, while the
 * next panel computes.  Synchronous: returns when C is on the host.
 *   C->cap     entries available in C->colidx / C->val (flop always suffices);
 *              C->nnz receives nnz(C) (also when it exceeds cap)
 *   *device_status  PB_OK, or PB_ERR_OVERFLOW when nnz(C) > C->cap (C incomplete),
 *              or the device-detected error of the numeric phase.
 * Errors (returned): INVALID_ARG, SHAPE, UNSUPPORTED_DTYPE, UNSUPPORTED, OOM, CUDA.
 */
typedef struct pb_csr_host {
    int32_t nrows, ncols;
    int64_t cap;
    int64_t *rowptr;  /* host, nrows + 1 */
    int32_t *colidx;  /* host, cap */
    void *val;        /* host, cap values of the dtype's output type */
    int64_t nnz;      /* output */
} pb_csr_host;

pb_status pb_spgemm_host(pb_handle *h, const pb_csc *A, const pb_csr *B, pb_dtype dtype, const pb_config *cfg,
                         pb_csr_host *C, pb_stream_t stream, pb_status *device_status);

/* Device-side status of the last numeric call made with this plan: PB_OK or
 * the first device-detected error.  Synchronises `stream` first. */
pb_status pb_plan_status(const pb_plan *plan, pb_stream_t stream, pb_status *device_status);

/* Copy plan arrays to caller DEVICE buffers (any may be NULL), for tests and tools.
 *   F       int64 [A.ncols + 1]  exclusive prefix of per-k flop (Alg. 3)
 *   R       int64 [A.nrows + 1]  exclusive prefix of per-row flop (Sec. III-B)
 *   bin_row int32 [nbins + 1]    first row of each bin, bin_row[nbins] = A.nrows
 *   bin_off int64 [nbins + 1]    tuple offset of each bin in the workspace (padded)
 * Synchronises `stream`. */
pb_status pb_plan_export(const pb_plan *plan, int64_t *F, int64_t *R, int32_t *bin_row, int64_t *bin_off,
                         pb_stream_t stream);

/* Run only the expand phase into `workspace` (same layout numeric uses):
 * tuples of bin b occupy [bin_off[b], bin_off[b] + count_b) of the key array
 * that starts at workspace and the value array that starts at
 * workspace + pb_debug_values_offset(plan).  When pb_debug_tuple_layout(plan)
 * is 1 (4-byte values, no row above the bin capacity, not deterministic) tuple
 * t is instead the pair of uint32 {key, value bits} at workspace + 8t.  For
 * tests of the expand step. */
pb_status pb_debug_expand(pb_handle *h, const pb_plan *plan, const pb_csc *A, const pb_csr *B,
                          void *workspace, size_t ws_bytes, pb_stream_t stream);
size_t pb_debug_values_offset(const pb_plan *plan);
int32_t pb_debug_tuple_layout(const pb_plan *plan);

pb_status pb_plan_destroy(pb_plan *plan);

/* Operand validation: O(nnz(A) + nnz(B)) device checks of the preconditions the
 * compute calls trust -- colptr / rowptr start at 0, never decrease and end at nnz,
 * every row index of A lies in [0, A.nrows) and every column index of B in
 * [0, B.ncols).  Reads each array only within its declared size.  Synchronises
 * `stream`; *result receives PB_OK or PB_ERR_INVALID_ARG (pb_last_error says which
 * array is wrong).  Errors (returned): INVALID_ARG, SHAPE, CUDA.  Duplicate entries
 * inside one column or row are not checked. */
pb_status pb_validate_operands(pb_handle *h, const pb_csc *A, const pb_csr *B, pb_stream_t stream,
                               pb_status *result);

/* Measurement hooks (no counterpart in the paper; they only observe).
 * pb_set_phase_events: when events is non-NULL, every later numeric call on
 * this handle records events[0] before its first launch, events[1] after the
 * workspace reset, events[2] after the expand kernel and events[3] after the
 * sort/compress kernel, on the call's stream.  The four entries are cudaEvent_t
 * handles owned by the caller; NULL disables recording.  pb_spgemm_batch
 * records events[0] before its first launch, events[1] after its symbolic
 * kernels, events[2] after the expand kernel and events[3] after the last
 * sort launch (when the batch is not empty).
 * pb_kernel_launches: number of CUDA kernels this library has launched in the
 * process so far (all handles). */
pb_status pb_set_phase_events(pb_handle *h, void *const *events);
int64_t pb_kernel_launches(void);

/*
 * Batched products.  Running many independent products together has no
 * counterpart in the paper; every product still goes through Alg. 3, the
 * expand of Alg. 2, the bin sort of Sec. III-D and the merge of Sec. III-E.
 *
 * pb_spgemm_batch computes C[i] = A[i] * B[i] for 0 <= i < count as one pass:
 * the products are laid out back to back (rows, columns of A and A entries
 * each in one index space), bins never straddle two products, the look-back
 * that places each bin's output restarts at each product's first bin, and the
 * sort kernel writes every bin straight into its own product's C.  Symbolic
 * kernels, one expand launch and one sort launch per bin-capacity level serve
 * the whole batch with persistent grids.
 *
 * Parameters per product come from the handle's tuning table, keyed by the
 * sparsity class (log2n, dclass):
 *   log2n  = ceil(log2(max(A.nrows, 2)))
 *   dclass = bit length of round(nnz(A) / max(A.ncols, 1)), i.e. 1 for d = 1,
 *            2 for d = 2..3, 3 for 4..7, 4 for 8..15, 5 for 16..31, ...
 * An untuned class uses bin_capacity 4096, rmax_log2 11, expand_chunk 4096.
 *
 * pb_spgemm_batch is asynchronous: it allocates nothing, never synchronises
 * the host and makes no host-device copies, so a call can be captured into a
 * CUDA graph and replayed.  The products' sizes and device pointers are baked
 * into the launches; a replay recomputes everything from the arrays' current
 * contents.  The launch-parameter blocks describing the products take about
 * 160 bytes per product.
 *
 *   workspace   device buffer, 256-byte aligned, at least the size
 *               pb_spgemm_batch_query reports for these operands; scratch.
 *   C[i]        as for pb_spgemm_numeric (no counting run): exactly one of
 *               rowptr64 / rowptr32, cap >= nnz(C[i]) (the product's flop,
 *               from the query, always suffices), nnz_dev optional.
 *   device_status  DEVICE pointer to one int32 that receives, in stream
 *               order after the last kernel, PB_OK or the device-detected
 *               error of the batch: PB_ERR_OVERFLOW (a C[i] too small),
 *               PB_ERR_WORKSPACE (tuples do not fit), PB_ERR_UNSUPPORTED (a
 *               row above its product's bin capacity in a product with
 *               B.ncols > 2^22: run it with pb_spgemm_numeric),
 *               PB_ERR_TIMEOUT.
 * Rows above their product's bin capacity (hub rows, Sec. III-D) are found on
 * the device and merged in dense column tiles inside the batch (products with
 * B.ncols <= 2^22); the workspace the query reports covers their scratch.
 * Limits: count <= 2^20; the sums over the batch of A.nrows, A.ncols and
 * nnz(A) each below 2^31.
 * Errors (returned): INVALID_ARG, SHAPE, UNSUPPORTED_DTYPE, UNSUPPORTED, CUDA.
 */
typedef struct pb_batch_tune {
    int32_t log2n;         /* class key */
    int32_t dclass;        /* class key */
    int32_t bin_capacity;  /* tuples per bin sorted on chip: 2048, 4096 or 8192 */
    int32_t rmax_log2;     /* a bin spans at most 2^rmax_log2 rows (1..11) */
    int32_t expand_chunk;  /* tuples per expand work item (multiple of 32, >= 256) */
    int32_t reserved;
} pb_batch_tune;

/* Workspace for pb_spgemm_batch on these operands and, per product (host
 * arrays of count entries, either may be NULL), its flop (Alg. 3; a C
 * capacity that always suffices) and its largest per-row flop.  The workspace
 * holds the scratch of every row above 2048 tuples, so it suffices for any
 * bin capacity the tuning table may choose.
 * Synchronises `stream` once; allocates a temporary buffer through the
 * handle's allocator. */
pb_status pb_spgemm_batch_query(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, pb_dtype dtype,
                                pb_stream_t stream, size_t *workspace_bytes, int64_t *flop,
                                int64_t *max_row_flop);

pb_status pb_spgemm_batch(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, pb_csr_out *C,
                          pb_dtype dtype, void *workspace, size_t ws_bytes, pb_stream_t stream,
                          int32_t *device_status);

/* Autotuner: for every sparsity class present in the batch, times candidate
 * (bin_capacity, rmax_log2, expand_chunk) settings on that class's products
 * (CUDA events, `reps` timed runs each after one warm-up) and stores the
 * fastest in the handle's tuning table.  Synchronous.  Uses C and the
 * workspace exactly like pb_spgemm_batch (C receives the products under the
 * chosen settings); allocates a 256-byte status word through the handle's
 * allocator.  Settings whose run reports a device error are skipped. */
pb_status pb_batch_autotune(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, pb_csr_out *C,
                            pb_dtype dtype, void *workspace, size_t ws_bytes, pb_stream_t stream, int32_t reps);

/* Read / replace the tuning table.  get writes up to `cap` entries and the
 * table's size to *n; set replaces the table (entries are validated). */
pb_status pb_batch_get_tuning(const pb_handle *h, pb_batch_tune *out, int32_t cap, int32_t *n);
pb_status pb_batch_set_tuning(pb_handle *h, const pb_batch_tune *entries, int32_t n);

/*
 * Serving: a request loop with continuous batching (no counterpart in the
 * paper; each request runs the paper's method through the entry points above).
 *
 * A server owns `max_slots` slots, each a host thread with its own CUDA
 * stream.  A free slot admits a queued request as soon as the device memory it
 * needs fits the HBM budget; admitted requests run concurrently on their
 * slots' streams, so a request arriving while others are on the GPU starts
 * without waiting for them.  Among queued requests the one with the least
 * estimated work (nnz(A) times the mean row length of B) is admitted first,
 * unless the oldest queued request has already been passed over 16 times.
 * A product whose flop-sized C could never fit the budget is sized exactly by
 * a counting run first.  Operands stay where the caller put them
 * (device memory, kept alive until the request is done); the server allocates
 * plans, workspaces, intermediates and results itself with cudaMallocAsync on
 * the slot's stream (not through the handle's allocator) and counts every byte
 * against the budget.  Results stay resident, and count against the budget,
 * until pb_serve_release.
 *
 * Request kinds:
 *   PB_REQ_PRODUCT   C = A * B (A CSC, B CSR), e.g. a Markov-clustering
 *                    squaring M * M of a column-stochastic M.
 *   PB_REQ_GALERKIN  C = P^T (A P), the coarse operator of an AMG level:
 *                    A (n x n, CSC) in `A`, the prolongator P (n x nc, CSR) in
 *                    `B`.  Two products: AP = A * P (CSR), then P^T * AP with
 *                    P^T taken as the CSC view of P's CSR arrays.
 * Small requests are coalesced: a slot that admits a request of at most
 * 2^24 estimated work also takes the other queued requests that small with the
 * same dtype (16 in all at most; pb_server_set_batching changes both) and runs
 * them as one pb_spgemm_batch launch (Galerkin members: one launch for all
 * A P, one for all P^T (A P)), with flop-sized results.  A group that cannot
 * run batched runs its requests one by one.
 * A request whose need exceeds the whole budget completes with PB_ERR_BUSY.
 * No request is admitted while an admitted one waits for memory.  When every
 * admitted request is waiting for memory, the most recently admitted one is
 * preempted: its memory is released and it is queued again at the front.
 */
typedef enum pb_request_kind { PB_REQ_PRODUCT = 0, PB_REQ_GALERKIN = 1 } pb_request_kind;

typedef struct pb_request {
    int32_t kind;   /* pb_request_kind */
    int32_t dtype;  /* pb_dtype */
    pb_csc A;
    pb_csr B;
} pb_request;

typedef struct pb_server pb_server;

/* Create a server on the handle's device.  hbm_budget: bytes the server may
 * hold at once; max_slots: requests in flight at once (1..64). */
pb_status pb_server_create(pb_handle *h, size_t hbm_budget, int32_t max_slots, pb_server **s);
/* Finish every admitted and queued request, free all server memory (including
 * unreleased results) and stop the worker. */
pb_status pb_server_destroy(pb_server *s);
/* Queue a request; *req_id identifies it.  Returns PB_ERR_BUSY at once when a
 * lower bound of its need (its operands' index arrays) already exceeds the
 * budget, and argument errors as pb_spgemm_symbolic does. */
pb_status pb_serve_submit(pb_server *s, const pb_request *req, uint64_t *req_id);
/* *done = 1 once the request has finished; *result is then its status. */
pb_status pb_serve_poll(pb_server *s, uint64_t req_id, int32_t *done, pb_status *result);
/* Block until the request has finished; *result receives its status. */
pb_status pb_serve_wait(pb_server *s, uint64_t req_id, pb_status *result);
/* Device pointers of a finished request's C (int64 row pointer; C->cap = nnz(C);
 * C->nnz_dev = NULL).  Owned by the server until pb_serve_release. */
pb_status pb_serve_result(pb_server *s, uint64_t req_id, pb_csr_out *C);
/* Host-clock times of a finished request in milliseconds: queued (submit to
 * admission) and total (submit to completion seen by the worker). */
pb_status pb_serve_timing(pb_server *s, uint64_t req_id, double *queued_ms, double *total_ms);
/* Free a finished request's result and forget the request. */
pb_status pb_serve_release(pb_server *s, uint64_t req_id);
/* Counters: requests completed and preempted, bytes held now and at most. */
pb_status pb_serve_stats(pb_server *s, int64_t *completed, int64_t *preempted, size_t *bytes_in_use,
                         size_t *peak_bytes);
/* Coalescing of small requests: at most max_requests per batched launch (1
 * turns coalescing off), requests of at most max_request_work estimated work
 * (nnz(A) times the mean row length of B, per product).  Applies to later
 * admissions.  Errors: INVALID_ARG. */
pb_status pb_server_set_batching(pb_server *s, int32_t max_requests, double max_request_work);
/* Requests completed through batched launches, and those launches. */
pb_status pb_serve_batch_stats(pb_server *s, int64_t *requests, int64_t *launches);

/*
 * No-allocation entry point (the paper has no counterpart; this serves callers).
 *
 * Some callers cannot allocate device memory where they need a product: code
 * whose device memory is owned by its own manager, latency-critical loops that
 * must not enter an allocator, or callbacks that run while an allocation lock
 * is held.  pb_spgemm_noalloc computes C = A * B (symbolic and numeric) using
 * only a fixed scratch array of PB_NOALLOC_SCRATCH_BYTES bytes that the library
 * defines in device memory; every GPU that loads the library holds that array
 * until the process exits.  The call performs no cudaMalloc / cudaFree and no
 * other allocation; the caller provides A, B and C exactly as for
 * pb_spgemm_numeric (C->cap >= nnz(C); a capacity equal to the product's
 * flop count, sum over k of nnz(A(:,k)) * nnz(B(k,:)), always suffices).
 *
 *   Limit: the plan arrays take about 92*A.nrows + 12*A.ncols + 12*nnz(A)
 *   bytes and the tuples 12 (FP64) or 8 (FP32 forms) bytes each, all within
 *   PB_NOALLOC_SCRATCH_BYTES; a larger product returns PB_ERR_WORKSPACE and
 *   launches nothing further.
 *   Synchronous: it synchronises `stream` (once after the symbolic phase and
 *   once at the end) and stores the device-detected status (PB_OK,
 *   PB_ERR_OVERFLOW, ...) in *device_status.
 *   The first call on a device resolves the scratch array's device address
 *   (cudaGetSymbolAddress, with that device current) and keeps it for the
 *   life of the process; make that first call before any stream capture.
 *   Calls after a reset of the device (cudaDeviceReset) are not supported:
 *   the kept address belongs to the context the reset destroyed.
 *   *device_status uses the same mapping as pb_plan_status.
 *   All calls share the one array and it keeps the last call's contents (the
 *   call clears what it needs).  Calls whose work overlaps on the GPU, e.g.
 *   issued on two streams, race on the array: serialise them.
 * Errors: INVALID_ARG, SHAPE, UNSUPPORTED_DTYPE, UNSUPPORTED, WORKSPACE, CUDA.
 */
#define PB_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
pb_status pb_spgemm_noalloc(const pb_csc *A, const pb_csr *B, pb_dtype dtype, pb_csr_out *C, pb_stream_t stream,
                            pb_status *device_status);

#ifdef __cplusplus
}
#endif
#endif /* PB_SPGEMM_H */
