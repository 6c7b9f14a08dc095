// pb_spgemm_noalloc: the whole product (symbolic + numeric) without any
// device-memory allocation.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a product: code that owns all device memory through its own
// manager, latency-critical loops that must not enter the driver's allocator,
// or library callbacks that run while an allocation lock is held.  This entry
// point serves them: every device array it needs (the plan's arrays and the
// numeric workspace) is carved from one file-scope __device__ array of
// PB_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library holds
// until the process exits.  The caller still provides A, B and C.
//
// The host side only carves offsets into that array; it calls no cudaMalloc,
// cudaFree or other allocating routine.  Host code cannot use the array's
// symbol as a device address: on the first call on each device (with that
// device current) cudaGetSymbolAddress resolves it once and the address is
// cached.  That first call should therefore happen before any stream capture.
//
// All calls share the array and it keeps the previous call's contents; every
// region that must start at zero is cleared by the call itself.  Calls whose
// work overlaps on the GPU (e.g. on two streams) race on the array.
#include <mutex>

#include "pb_common.cuh"

namespace pb {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (resolved once).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Bump carving inside the scratch array.
struct Carve {
    char *base;
    size_t size, used;
    template <class T>
    bool take(T *&p, size_t bytes) {
        const size_t b = (bytes + 255) & ~size_t(255);
        if (b > size - used) return false;
        p = reinterpret_cast<T *>(base + used);
        used += b;
        return true;
    }
};

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((uint64_t(1) << b) < x) ++b;
    return b;
}

}  // namespace
}  // namespace pb

using namespace pb;

#define PB_NA_CUDA(call)                              \
    do {                                              \
        if ((call) != cudaSuccess) return PB_ERR_CUDA; \
    } while (0)

extern "C" pb_status pb_spgemm_noalloc(const pb_csc *A, const pb_csr *B, pb_dtype dtype, pb_csr_out *C,
                                       pb_stream_t stream_, pb_status *device_status) {
    if (!A || !B || !C || !device_status) return PB_ERR_INVALID_ARG;
    *device_status = PB_OK;
    if (dtype != PB_F64 && dtype != PB_F32 && dtype != PB_F64_F32TUPLE) return PB_ERR_UNSUPPORTED_DTYPE;
    if (A->nrows < 0 || A->ncols < 0 || B->nrows < 0 || B->ncols < 0 || A->nnz < 0 || B->nnz < 0)
        return PB_ERR_INVALID_ARG;
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) return PB_ERR_SHAPE;
    if (A->nnz > 0x7fffffffll || B->nnz > 0x7fffffffll) return PB_ERR_UNSUPPORTED;
    if (!A->colptr || !B->rowptr) return PB_ERR_INVALID_ARG;
    if ((A->nnz > 0 && (!A->rowidx || !A->val)) || (B->nnz > 0 && (!B->colidx || !B->val)))
        return PB_ERR_INVALID_ARG;
    if ((C->rowptr64 == nullptr) == (C->rowptr32 == nullptr)) return PB_ERR_INVALID_ARG;
    if (C->cap < 0 || (C->cap > 0 && (!C->colidx || !C->val))) return PB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);

    void *base = nullptr;
    PB_NA_CUDA(scratch_address(&base));
    Carve cv{static_cast<char *>(base), (size_t)PB_NOALLOC_SCRATCH_BYTES, 0};

    const int32_t m = A->nrows, k = A->ncols, n = B->ncols;
    const int64_t nnzA = A->nnz;
    const int colbits = ceil_log2((uint64_t)(n > 1 ? n : 2));
    if (colbits > 31) return PB_ERR_UNSUPPORTED;
    const int rowbits = 32 - colbits;
    const int32_t capacity = 4096, chunk = 4096;

    // ---- plan arrays (same layout as a plan made by pb_spgemm_symbolic) -----------
    SymbolicArgs a{};
    int32_t *acol = nullptr;
    int64_t *scan_tmp = nullptr;
    uint32_t *err = nullptr;
    const size_t m1 = (size_t)m + 1, m2 = (size_t)m + 2;
    const size_t scan_n = (size_t)(m > k ? m : k) + 2;
    bool ok = cv.take(a.F, 8 * ((size_t)k + 1)) && cv.take(a.R, 8 * m1) && cv.take(a.flags, 8 * m1) &&
              cv.take(a.rowinfo, 8 * (m > 0 ? (size_t)m : 1)) && cv.take(a.bin_row, 4 * m2) &&
              cv.take(a.bin_off, 8 * m2) && cv.take(a.hdr, sizeof(PlanHeader)) &&
              cv.take(scan_tmp, 8 * (size_t)scan_tmp_elems((int64_t)scan_n)) && cv.take(err, 64) &&
              cv.take(a.over_scan, 8 * m1) && cv.take(a.over_bin, 8 * m1) && cv.take(a.over_chunk_off, 8 * m1) &&
              cv.take(a.over_tuple_off, 8 * m1) && cv.take(a.ainfo, 8 * (nnzA > 0 ? (size_t)nnzA : 1));
    ok = ok && cv.take(acol, 4 * (nnzA > 0 ? (size_t)nnzA : 1)) && cv.take(a.long_cols, 4 * (k > 0 ? (size_t)k : 1)) &&
         cv.take(a.n_long, 4) && cv.take(a.aspan, 8 * (nnzA > 0 ? (size_t)nnzA : 1));
    if (!ok) return PB_ERR_WORKSPACE;  // the product needs more than the scratch array holds

    a.m = m;
    a.k = k;
    a.n = n;
    a.colptrA = A->colptr;
    a.rowidxA = A->rowidx;
    a.rowptrB = B->rowptr;
    a.colbits = colbits;
    a.rmax_log2 = rowbits < RMAX_LOG2 ? rowbits : RMAX_LOG2;
    a.capacity = capacity;
    a.heavy = capacity / 2;
    a.nnzA = nnzA;
    a.acol = acol;
    PB_NA_CUDA(cudaMemsetAsync(a.hdr, 0, sizeof(PlanHeader), s));
    PB_NA_CUDA(cudaMemsetAsync(err, 0, 64, s));
    PB_NA_CUDA(launch_symbolic(a, scan_tmp, s));
    PlanHeader hdr;
    PB_NA_CUDA(cudaMemcpyAsync(&hdr, a.hdr, sizeof(PlanHeader), cudaMemcpyDeviceToHost, s));
    PB_NA_CUDA(cudaStreamSynchronize(s));
    if (hdr.max_bin_count > 0x7fffffffull) return PB_ERR_UNSUPPORTED;
    if (hdr.max_bin_count > (unsigned long long)capacity) {
        PB_NA_CUDA(launch_symbolic_oversize(a, scan_tmp, s));
        PB_NA_CUDA(cudaMemcpyAsync(&hdr, a.hdr, sizeof(PlanHeader), cudaMemcpyDeviceToHost, s));
        PB_NA_CUDA(cudaStreamSynchronize(s));
    }

    int32_t *over_chunk_bin = nullptr;
    int over_passes = 0;
    if (hdr.n_oversize > 0) {
        over_passes = (colbits + 7) / 8;
        if (!cv.take(over_chunk_bin, 4 * (size_t)hdr.over_chunks)) return PB_ERR_WORKSPACE;
        PB_NA_CUDA(launch_over_chunk_map(a.over_chunk_off, hdr.n_oversize, over_chunk_bin, s));
    }
    const int64_t nchunks = ceil_div<int64_t>(hdr.flop, chunk);
    int32_t *chunk_e = nullptr;
    if (!cv.take(chunk_e, 4 * ((size_t)nchunks + 1))) return PB_ERR_WORKSPACE;
    PB_NA_CUDA(launch_chunk_table(a, nchunks, chunk, chunk_e, s));

    // ---- numeric workspace -----------------------------------------------------------
    const size_t tb = (dtype == PB_F64) ? 8 : 4;
    const size_t T = (size_t)hdr.tuples_padded, nb = (size_t)hdr.nbins;
    const size_t OT = (size_t)hdr.over_tuples, OC = (size_t)hdr.over_chunks, NO = (size_t)hdr.n_oversize;
    NumericArgs na{};
    char *vals = nullptr, *svals = nullptr;
    ok = cv.take(na.keys, 4 * T) && cv.take(vals, tb * T) && cv.take(na.cursor, 8 * nb) &&
         cv.take(na.status, 8 * nb) && cv.take(na.ticket, 256);
    uint32_t *hist = nullptr;
    int64_t *over_u = nullptr;
    ok = ok && cv.take(na.skeys, 4 * OT) && cv.take(svals, tb * OT) && cv.take(hist, 1024 * OC) &&
         cv.take(over_u, 8 * NO);
    if (!ok) return PB_ERR_WORKSPACE;

    na.m = m;
    na.k = k;
    na.n = n;
    na.colptrA = A->colptr;
    na.rowidxA = A->rowidx;
    na.rowptrB = B->rowptr;
    na.colidxB = B->colidx;
    na.valA = A->val;
    na.valB = B->val;
    na.F = a.F;
    na.R = a.R;
    na.ainfo = a.ainfo;
    na.acol = acol;
    na.aspan = a.aspan;
    na.bin_row = a.bin_row;
    na.bin_off = a.bin_off;
    na.chunk_e = chunk_e;
    na.flop = hdr.flop;
    na.nbins = hdr.nbins;
    na.nchunks = nchunks;
    na.chunk = chunk;
    na.colbits = colbits;
    na.capacity = capacity;
    na.vals = vals;
    na.err = err;
    na.rowptr64 = C->rowptr64;
    na.rowptr32 = C->rowptr32;
    na.colidx = C->colidx;
    na.valC = C->val;
    na.nnz_dev = C->nnz_dev;
    na.cap = C->cap;
    na.count_only = 0;
    na.cursor_stride = 1;
    na.dtype = dtype;
    int dev = 0;
    PB_NA_CUDA(cudaGetDevice(&dev));
    PB_NA_CUDA(cudaDeviceGetAttribute(&na.num_sms, cudaDevAttrMultiProcessorCount, dev));
    na.over_scan = a.over_scan;
    na.over_tuple_off = a.over_tuple_off;
    na.over_u = over_u;
    na.svals = svals;
    na.over_passes = over_passes;
    na.bin_lo = 0;  // one panel: the whole product
    na.bin_hi = hdr.nbins;
    na.tuple_base = 0;
    na.over_base = 0;

    if (m == 0) {
        if (C->rowptr64) PB_NA_CUDA(cudaMemsetAsync(C->rowptr64, 0, 8, s));
        if (C->rowptr32) PB_NA_CUDA(cudaMemsetAsync(C->rowptr32, 0, 4, s));
        if (C->nnz_dev) PB_NA_CUDA(cudaMemsetAsync(C->nnz_dev, 0, 8, s));
        PB_NA_CUDA(cudaStreamSynchronize(s));
        return PB_OK;
    }
    // regions that must start in a known state (the array keeps the last call's data)
    PB_NA_CUDA(cudaMemcpyAsync(na.cursor, a.bin_off, 8 * nb, cudaMemcpyDeviceToDevice, s));
    PB_NA_CUDA(cudaMemsetAsync(na.status, 0, 8 * nb, s));
    PB_NA_CUDA(cudaMemsetAsync(na.ticket, 0, 256, s));
    na.work = na.ticket + 32;
    PB_NA_CUDA(launch_expand(na, s));
    if (hdr.n_oversize > 0) {
        OversizeArgs o{};
        o.R = a.R;
        o.bin_row = a.bin_row;
        o.bin_off = a.bin_off;
        o.over_bin = a.over_bin;
        o.over_chunk_off = a.over_chunk_off;
        o.over_tuple_off = a.over_tuple_off;
        o.over_chunk_bin = over_chunk_bin;
        o.n_over = hdr.n_oversize;
        o.over_chunks = hdr.over_chunks;
        o.keys = na.keys;
        o.vals = vals;
        o.skeys = na.skeys;
        o.svals = svals;
        o.hist = hist;
        o.over_u = over_u;
        o.o_lo = 0;
        o.o_hi = hdr.n_oversize;
        o.c_lo = 0;
        o.c_hi = hdr.over_chunks;
        o.tuple_base = 0;
        o.over_base = 0;
        PB_NA_CUDA(launch_oversize(o, over_passes, dtype, na.num_sms, s));
    }
    PB_NA_CUDA(launch_binsort(na, s));

    uint32_t word = 0;
    PB_NA_CUDA(cudaMemcpyAsync(&word, err, 4, cudaMemcpyDeviceToHost, s));
    PB_NA_CUDA(cudaStreamSynchronize(s));
    *device_status = status_of_word(word);  // the mapping pb_plan_status uses
    return PB_OK;
}
