// Host side of the C ABI: handles, plans, argument checks, workspace layout
// and the launch sequence of the symbolic and numeric phases.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pb_common.cuh"
#include "pb_host.h"

using namespace pb;

namespace pb {
static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace pb

// A row panel: consecutive bins whose tuples fit the workspace together.
struct pb_panel {
    int64_t bin_lo, bin_hi;      // bins
    int64_t tuple_base, tuples;  // padded tuple range [tuple_base, tuple_base + tuples)
    int64_t o_lo, o_hi;          // oversize bins (indices into the oversize list)
    int64_t c_lo, c_hi;          // their work items
    int64_t over_base, over_tuples;
};

struct pb_plan {
    pb_handle *h = nullptr;
    std::vector<pb_panel> panels;
    int32_t m = 0, k = 0, n = 0;
    int64_t nnzA = 0, nnzB = 0;
    pb_dtype dtype = PB_F64;
    int32_t colbits = 1, rmax_log2 = 0, capacity = 4096;
    int64_t heavy = 0, chunk = 4096, nchunks = 0;
    PlanHeader hdr{};
    // device arrays (one arena + the chunk table)
    void *arena = nullptr;
    size_t arena_bytes = 0;
    void *chunk_mem = nullptr;
    size_t chunk_bytes = 0;
    void *apos_mem = nullptr;  // deterministic mode: run position of every A entry
    size_t apos_bytes = 0;
    int64_t *F = nullptr, *R = nullptr, *flags = nullptr, *bin_off = nullptr, *scan_tmp = nullptr;
    uint64_t *rowinfo = nullptr, *ainfo = nullptr;
    int2 *aspan = nullptr;
    int32_t *bin_row = nullptr, *chunk_e = nullptr, *acol = nullptr;
    PlanHeader *dhdr = nullptr;
    uint32_t *err = nullptr;
    int64_t *over_scan = nullptr, *over_bin = nullptr, *over_chunk_off = nullptr, *over_tuple_off = nullptr;
    void *over_map_mem = nullptr;
    size_t over_map_bytes = 0;
    int32_t *over_chunk_bin = nullptr;
    int over_passes = 0;
    int over_dense = 0, over_shift = 0;  // oversize rows merged in dense column tiles
    // 4-byte values without oversize bins or fixed run positions: tuples are
    // packed {key, value bits} pairs over the key and value regions
    int packed = 0;
    // workspace layout of the numeric phase
    size_t ws_keys = 0, ws_vals = 0, ws_cursor = 0, ws_status = 0, ws_ctrl = 0;
    size_t ws_skeys = 0, ws_svals = 0, ws_hist = 0, ws_cinfo = 0, ws_over_u = 0, ws_overp = 0, ws_overord = 0,
           ws_bytes = 0;
};

namespace {

constexpr int32_t kVersion = 1 * 10000 + 0 * 100 + 0;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bin cursors start at the bins' offsets, PB_CURSOR_STRIDE words apart.
cudaError_t reset_cursors(void *cursor, const int64_t *bin_off, size_t nb, cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    return cudaMemcpy2DAsync(cursor, 8 * (size_t)PB_CURSOR_STRIDE, bin_off, 8, 8, nb, cudaMemcpyDeviceToDevice, s);
}

void *default_alloc(size_t bytes, pb_stream_t stream, void *) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes ? bytes : 256, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void default_free(void *p, size_t, pb_stream_t stream, void *) {
    if (p) (void)cudaFreeAsync(p, reinterpret_cast<cudaStream_t>(stream));
}

pb_status fail(pb_handle *h, pb_status st, const std::string &msg) {
    if (h) h->last_error = msg;
    return st;
}

pb_status cuda_fail(pb_handle *h, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, PB_ERR_CUDA, msg);
}

#define PB_CUDA(h, call)                                         \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

int ceil_log2_u64(uint64_t x) {
    int b = 0;
    while ((uint64_t(1) << b) < x) ++b;
    return b;
}

size_t tuple_val_bytes(pb_dtype d) { return d == PB_F64 ? 8 : 4; }

bool valid_dtype(pb_dtype d) { return d == PB_F64 || d == PB_F32 || d == PB_F64_F32TUPLE; }

pb_status check_operands(pb_handle *h, const pb_csc *A, const pb_csr *B) {
    if (!A || !B) return fail(h, PB_ERR_INVALID_ARG, "A and B must not be NULL");
    if (A->nrows < 0 || A->ncols < 0 || B->nrows < 0 || B->ncols < 0 || A->nnz < 0 || B->nnz < 0)
        return fail(h, PB_ERR_INVALID_ARG, "negative dimension or nnz");
    if (A->ncols != B->nrows) return fail(h, PB_ERR_SHAPE, "A.ncols != B.nrows");
    if (A->nnz > 0x7fffffffll || B->nnz > 0x7fffffffll)
        return fail(h, PB_ERR_UNSUPPORTED, "operand nnz must fit int32 pointers");
    if (!A->colptr || !B->rowptr) return fail(h, PB_ERR_INVALID_ARG, "pointer arrays must not be NULL");
    if ((A->nnz > 0 && (!A->rowidx || !A->val)) || (B->nnz > 0 && (!B->colidx || !B->val)))
        return fail(h, PB_ERR_INVALID_ARG, "index/value arrays must not be NULL when nnz > 0");
    return PB_OK;
}

void free_plan_memory(pb_plan *p) {
    if (!p || !p->h) return;
    if (p->chunk_mem) p->h->free_fn(p->chunk_mem, p->chunk_bytes, nullptr, p->h->ctx);
    if (p->apos_mem) p->h->free_fn(p->apos_mem, p->apos_bytes, nullptr, p->h->ctx);
    p->apos_mem = nullptr;
    if (p->over_map_mem) p->h->free_fn(p->over_map_mem, p->over_map_bytes, nullptr, p->h->ctx);
    p->over_map_mem = nullptr;
    if (p->arena) p->h->free_fn(p->arena, p->arena_bytes, nullptr, p->h->ctx);
    p->chunk_mem = p->arena = nullptr;
}

}  // namespace

namespace pb {
pb_status host_fail(pb_handle *h, pb_status st, const std::string &msg) { return fail(h, st, msg); }
pb_status host_cuda_fail(pb_handle *h, cudaError_t e, const char *where) { return cuda_fail(h, e, where); }
pb_status host_check_operands(pb_handle *h, const pb_csc *A, const pb_csr *B) { return check_operands(h, A, B); }
size_t plan_device_bytes(const pb_plan *p) {
    return p ? p->arena_bytes + p->chunk_bytes + p->over_map_bytes + p->apos_bytes : 0;
}
}  // namespace pb

extern "C" {

int32_t pb_version(void) { return kVersion; }

pb_status pb_create(pb_handle **out) {
    if (!out) return PB_ERR_INVALID_ARG;
    *out = nullptr;
    pb_handle *h = new (std::nothrow) pb_handle();
    if (!h) return PB_ERR_OOM;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        (void)cudaGetLastError();
        return PB_ERR_CUDA;
    }
    h->alloc = default_alloc;
    h->free_fn = default_free;
    *out = h;
    return PB_OK;
}

pb_status pb_destroy(pb_handle *h) {
    delete h;
    return PB_OK;
}

pb_status pb_set_allocator(pb_handle *h, pb_alloc_fn alloc, pb_free_fn free_fn, void *ctx) {
    if (!h) return PB_ERR_INVALID_ARG;
    if (alloc && !free_fn) return fail(h, PB_ERR_INVALID_ARG, "free_fn required with alloc");
    h->alloc = alloc ? alloc : default_alloc;
    h->free_fn = alloc ? free_fn : default_free;
    h->ctx = alloc ? ctx : nullptr;
    return PB_OK;
}

const char *pb_last_error(const pb_handle *h) { return h ? h->last_error.c_str() : "null handle"; }

pb_status pb_spgemm_symbolic(pb_handle *h, const pb_csc *A, const pb_csr *B, pb_dtype dtype,
                             const pb_config *cfg, pb_stream_t stream_, pb_plan **out) {
    if (!h || !out) return PB_ERR_INVALID_ARG;
    *out = nullptr;
    h->last_error.clear();
    pb_status st = check_operands(h, A, B);
    if (st != PB_OK) return st;
    if (!valid_dtype(dtype)) return fail(h, PB_ERR_UNSUPPORTED_DTYPE, "unknown dtype");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);

    pb_plan *p = new (std::nothrow) pb_plan();
    if (!p) return fail(h, PB_ERR_OOM, "host allocation failed");
    p->h = h;
    p->m = A->nrows;
    p->k = A->ncols;
    p->n = B->ncols;
    p->nnzA = A->nnz;
    p->nnzB = B->nnz;
    p->dtype = dtype;
    p->colbits = ceil_log2_u64((uint64_t)(p->n > 1 ? p->n : 2));
    if (p->colbits > 31) {
        delete p;
        return fail(h, PB_ERR_UNSUPPORTED, "B.ncols too large for a 32-bit key");
    }
    int rowbits = 32 - p->colbits;
    p->rmax_log2 = rowbits < RMAX_LOG2 ? rowbits : RMAX_LOG2;
    if (cfg && cfg->bin_capacity) p->capacity = cfg->bin_capacity;
    if (p->capacity != 2048 && p->capacity != 4096 && p->capacity != 8192) {
        delete p;
        return fail(h, PB_ERR_INVALID_ARG, "bin_capacity must be 2048, 4096 or 8192");
    }
    if (cfg && cfg->sort_threads && cfg->sort_threads != p->capacity / 8) {
        delete p;
        return fail(h, PB_ERR_INVALID_ARG, "sort_threads must be 0 or bin_capacity / 8");
    }
    p->heavy = p->capacity / 2;
    if (cfg && cfg->expand_chunk) {
        if (cfg->expand_chunk < 32 || cfg->expand_chunk % 32) {
            delete p;
            return fail(h, PB_ERR_INVALID_ARG, "expand_chunk must be a positive multiple of 32");
        }
        p->chunk = cfg->expand_chunk;
    }

    // Arena of plan arrays.
    const int64_t m = p->m, k = p->k;
    const int64_t scan_n = (m > k ? m : k) + 2;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oF = take(8 * (k + 1)), oR = take(8 * (m + 1)), oFl = take(8 * (m + 1));
    const size_t oRi = take(8 * (m > 0 ? m : 1)), oBr = take(4 * (m + 2)), oBo = take(8 * (m + 2));
    const size_t oH = take(sizeof(PlanHeader)), oT = take(8 * scan_tmp_elems(scan_n)), oE = take(64);
    const size_t oOs = take(8 * (m + 1)), oOb = take(8 * (m + 1)), oOc = take(8 * (m + 1)), oOt = take(8 * (m + 1));
    const size_t oAi = take(8 * (p->nnzA > 0 ? p->nnzA : 1)), oAc = take(4 * (p->nnzA > 0 ? p->nnzA : 1));
    const size_t oAs = take(8 * (p->nnzA > 0 ? p->nnzA : 1));
    const size_t oLc = take(4 * (k > 0 ? k : 1) + 256);
    p->arena_bytes = off;
    p->arena = h->alloc(p->arena_bytes, stream_, h->ctx);
    if (!p->arena) {
        delete p;
        return fail(h, PB_ERR_OOM, "plan allocation failed");
    }
    char *base = static_cast<char *>(p->arena);
    p->F = reinterpret_cast<int64_t *>(base + oF);
    p->R = reinterpret_cast<int64_t *>(base + oR);
    p->flags = reinterpret_cast<int64_t *>(base + oFl);
    p->rowinfo = reinterpret_cast<uint64_t *>(base + oRi);
    p->bin_row = reinterpret_cast<int32_t *>(base + oBr);
    p->bin_off = reinterpret_cast<int64_t *>(base + oBo);
    p->dhdr = reinterpret_cast<PlanHeader *>(base + oH);
    p->scan_tmp = reinterpret_cast<int64_t *>(base + oT);
    p->err = reinterpret_cast<uint32_t *>(base + oE);
    p->over_scan = reinterpret_cast<int64_t *>(base + oOs);
    p->over_bin = reinterpret_cast<int64_t *>(base + oOb);
    p->over_chunk_off = reinterpret_cast<int64_t *>(base + oOc);
    p->over_tuple_off = reinterpret_cast<int64_t *>(base + oOt);
    p->ainfo = reinterpret_cast<uint64_t *>(base + oAi);
    p->acol = reinterpret_cast<int32_t *>(base + oAc);
    p->aspan = reinterpret_cast<int2 *>(base + oAs);

    auto bail = [&](pb_status code) {
        free_plan_memory(p);
        delete p;
        return code;
    };
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->dhdr, 0, sizeof(PlanHeader), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->err, 0, 64, s)) != cudaSuccess) {
        cuda_fail(h, e, "memset");
        return bail(PB_ERR_CUDA);
    }
    SymbolicArgs a{};
    a.m = p->m;
    a.k = p->k;
    a.n = p->n;
    a.colptrA = A->colptr;
    a.rowidxA = A->rowidx;
    a.rowptrB = B->rowptr;
    a.F = p->F;
    a.R = p->R;
    a.flags = p->flags;
    a.rowinfo = p->rowinfo;
    a.ainfo = p->ainfo;
    a.acol = p->acol;
    a.aspan = p->aspan;
    a.long_cols = reinterpret_cast<int32_t *>(base + oLc);
    a.n_long = reinterpret_cast<uint32_t *>(base + oLc + 4 * (k > 0 ? k : 1));
    a.nnzA = p->nnzA;
    a.bin_row = p->bin_row;
    a.bin_off = p->bin_off;
    a.hdr = p->dhdr;
    a.colbits = p->colbits;
    a.rmax_log2 = p->rmax_log2;
    a.capacity = p->capacity;
    a.heavy = p->heavy;
    a.over_scan = p->over_scan;
    a.over_bin = p->over_bin;
    a.over_chunk_off = p->over_chunk_off;
    a.over_tuple_off = p->over_tuple_off;
    if ((e = launch_symbolic(a, p->scan_tmp, s)) != cudaSuccess) {
        cuda_fail(h, e, "symbolic launch");
        return bail(PB_ERR_CUDA);
    }
    // The one synchronisation of the symbolic phase: read the sizes back.
    if ((e = cudaMemcpyAsync(&p->hdr, p->dhdr, sizeof(PlanHeader), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cuda_fail(h, e, "symbolic readback");
        return bail(PB_ERR_CUDA);
    }
    if (p->hdr.max_bin_count > 0x7fffffffull) {
        fail(h, PB_ERR_UNSUPPORTED, "a single row produces 2^31 or more tuples");
        return bail(PB_ERR_UNSUPPORTED);
    }
    if (p->hdr.max_bin_count > (unsigned long long)p->capacity) {
        // some rows exceed a bin: build their lists (a second, rarer readback)
        if ((e = launch_symbolic_oversize(a, p->scan_tmp, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&p->hdr, p->dhdr, sizeof(PlanHeader), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            cuda_fail(h, e, "oversize lists");
            return bail(PB_ERR_CUDA);
        }
    }
    // Oversize bins: work-item map for their global-memory radix sort.
    if (p->hdr.n_oversize > 0) {
        p->over_passes = (p->colbits + 7) / 8;
        // Dense column tiles when the order of the sums need not be fixed.
        const int shift = p->colbits > 8 ? p->colbits - 8 : 0;
        p->over_dense = (!(cfg && cfg->deterministic) && shift <= OVER_DENSE_MAX_SHIFT) ? 1 : 0;
        p->over_shift = shift;
        if (p->over_dense) p->over_passes = 1;  // the one partition pass leaves the tuples in scratch
        p->over_map_bytes = align256(4 * (size_t)p->hdr.over_chunks);
        p->over_map_mem = h->alloc(p->over_map_bytes, stream_, h->ctx);
        if (!p->over_map_mem) {
            fail(h, PB_ERR_OOM, "oversize map allocation failed");
            return bail(PB_ERR_OOM);
        }
        p->over_chunk_bin = static_cast<int32_t *>(p->over_map_mem);
        if ((e = launch_over_chunk_map(p->over_chunk_off, p->hdr.n_oversize, p->over_chunk_bin, s)) != cudaSuccess) {
            cuda_fail(h, e, "oversize map");
            return bail(PB_ERR_CUDA);
        }
    }
    // Expand work items (A-entry granularity) and the column of every A entry.
    p->nchunks = ceil_div<int64_t>(p->hdr.flop, p->chunk);
    p->chunk_bytes = align256(4 * ((size_t)p->nchunks + 1));
    p->chunk_mem = h->alloc(p->chunk_bytes, stream_, h->ctx);
    if (!p->chunk_mem) {
        fail(h, PB_ERR_OOM, "chunk table allocation failed");
        return bail(PB_ERR_OOM);
    }
    p->chunk_e = static_cast<int32_t *>(p->chunk_mem);
    if ((e = launch_chunk_table(a, p->nchunks, p->chunk, p->chunk_e, s)) != cudaSuccess) {
        cuda_fail(h, e, "chunk table");
        return bail(PB_ERR_CUDA);
    }
    p->packed = (tuple_val_bytes(dtype) == 4 && p->hdr.n_oversize == 0 && !(cfg && cfg->deterministic)) ? 1 : 0;
    // Deterministic mode: fixed run positions (CSC order inside each bin).
    if (cfg && cfg->deterministic && p->nnzA > 0) {
        p->apos_bytes = align256(8 * (size_t)p->nnzA);
        p->apos_mem = h->alloc(p->apos_bytes, stream_, h->ctx);
        const size_t sb = (size_t)det_scratch_bytes(p->nnzA);
        void *scratch = p->apos_mem ? h->alloc(sb, stream_, h->ctx) : nullptr;
        if (!scratch) {
            fail(h, PB_ERR_OOM, "deterministic-mode allocation failed");
            return bail(PB_ERR_OOM);
        }
        DetArgs d{p->nnzA, p->hdr.nbins, p->ainfo, p->acol, B->rowptr, p->bin_row, p->bin_off, p->R,
                  static_cast<int64_t *>(p->apos_mem)};
        e = launch_det_positions(d, scratch, h->num_sms, s);
        h->free_fn(scratch, sb, stream_, h->ctx);
        if (e != cudaSuccess) {
            cuda_fail(h, e, "deterministic positions");
            return bail(PB_ERR_CUDA);
        }
    }
    // Row panels: with a tuple budget smaller than the whole product, bins are
    // grouped into consecutive panels whose tuples fit the budget together.
    const size_t per_tuple = 4 + tuple_val_bytes(dtype);
    int64_t budget = (cfg && cfg->max_tuple_bytes > 0) ? cfg->max_tuple_bytes / (int64_t)per_tuple : 0;
    // min_panels: products of at least min_panels * 2^20 tuples are split into about that many panels
    const int64_t want = (cfg && cfg->min_panels > 1) ? cfg->min_panels : 1;
    const bool split_for_count = want > 1 && p->hdr.nbins >= want && p->hdr.tuples_padded >= (want << 20);
    if ((budget > 0 && p->hdr.tuples_padded > budget) || split_for_count) {
        const size_t nb = (size_t)p->hdr.nbins, no = (size_t)p->hdr.n_oversize;
        std::vector<int64_t> off(nb + 1), obin(no), ochunk(no + 1), otup(no + 1);
        if ((e = cudaMemcpyAsync(off.data(), p->bin_off, 8 * (nb + 1), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (no && (e = cudaMemcpyAsync(obin.data(), p->over_bin, 8 * no, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(ochunk.data(), p->over_chunk_off, 8 * (no + 1), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(otup.data(), p->over_tuple_off, 8 * (no + 1), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            cuda_fail(h, e, "panel readback");
            return bail(PB_ERR_CUDA);
        }
        // an oversize bin also needs its size again in scratch for its global sort
        std::vector<char> is_over(nb, 0);
        for (int64_t ob : obin) is_over[ob] = 1;
        if (split_for_count) {
            int64_t total = 0, largest = 0;
            for (size_t i = 0; i < nb; ++i) {
                const int64_t c = (off[i + 1] - off[i]) * (is_over[i] ? 2 : 1);
                total += c;
                largest = c > largest ? c : largest;
            }
            int64_t even = ceil_div<int64_t>(total, want);
            if (even < largest) even = largest;
            if (budget <= 0 || even < budget) budget = even;
        }
        int64_t b = 0;
        while (b < (int64_t)nb) {
            pb_panel pn{};
            pn.bin_lo = b;
            int64_t used = 0;
            while (b < (int64_t)nb) {
                const int64_t cost = (off[b + 1] - off[b]) * (is_over[b] ? 2 : 1);
                if (used + cost > budget) break;
                used += cost;
                ++b;
            }
            if (b == pn.bin_lo) {
                fail(h, PB_ERR_WORKSPACE, "max_tuple_bytes is smaller than the largest bin");
                return bail(PB_ERR_WORKSPACE);
            }
            pn.bin_hi = b;
            p->panels.push_back(pn);
        }
        for (pb_panel &pn : p->panels) {
            pn.tuple_base = off[pn.bin_lo];
            pn.tuples = off[pn.bin_hi] - off[pn.bin_lo];
            pn.o_lo = std::lower_bound(obin.begin(), obin.end(), pn.bin_lo) - obin.begin();
            pn.o_hi = std::lower_bound(obin.begin(), obin.end(), pn.bin_hi) - obin.begin();
            pn.c_lo = ochunk[pn.o_lo];
            pn.c_hi = ochunk[pn.o_hi];
            pn.over_base = otup[pn.o_lo];
            pn.over_tuples = otup[pn.o_hi] - otup[pn.o_lo];
        }
    } else {
        pb_panel pn{};
        pn.bin_lo = 0;
        pn.bin_hi = p->hdr.nbins;
        pn.tuple_base = 0;
        pn.tuples = p->hdr.tuples_padded;
        pn.o_lo = 0;
        pn.o_hi = p->hdr.n_oversize;
        pn.c_lo = 0;
        pn.c_hi = p->hdr.over_chunks;
        pn.over_base = 0;
        pn.over_tuples = p->hdr.over_tuples;
        p->panels.push_back(pn);
    }
    int64_t max_t = 0, max_ot = 0, max_oc = 0;
    for (const pb_panel &pn : p->panels) {
        max_t = std::max(max_t, pn.tuples);
        max_ot = std::max(max_ot, pn.over_tuples);
        max_oc = std::max(max_oc, pn.c_hi - pn.c_lo);
    }
    // Workspace layout of the numeric phase (sized for the largest panel).
    const size_t T = (size_t)max_t;
    const size_t nb = (size_t)p->hdr.nbins;
    size_t w = 0;
    p->ws_keys = w;
    w += align256(4 * T);
    p->ws_vals = w;
    w += align256(tuple_val_bytes(dtype) * T);
    p->ws_cursor = w;
    w += align256(8 * (size_t)PB_CURSOR_STRIDE * nb);
    p->ws_status = w;
    w += align256(8 * nb);
    p->ws_ctrl = w;
    w += 256;
    const size_t OT = (size_t)max_ot, OC = (size_t)max_oc, NO = (size_t)p->hdr.n_oversize;
    p->ws_skeys = w;
    w += align256(4 * OT);
    p->ws_svals = w;
    w += align256(tuple_val_bytes(dtype) * OT);
    p->ws_hist = w;
    w += align256(4 * 256 * OC);
    p->ws_cinfo = w;
    w += align256(sizeof(OverChunk) * OC);
    p->ws_over_u = w;
    w += align256(8 * NO);
    p->ws_overp = w;
    w += align256(8 * NO);
    p->ws_overord = w;  // dense path: row order (int32 per row) and 128 class counters
    w += p->over_dense ? align256(4 * NO) + 512 : 0;
    p->ws_bytes = w;
    *out = p;
    return PB_OK;
}

pb_status pb_plan_query(const pb_plan *p, int64_t *flop, int64_t *c_cap, size_t *workspace_bytes, int64_t *nbins,
                        int32_t *npanels) {
    if (!p) return PB_ERR_INVALID_ARG;
    if (flop) *flop = p->hdr.flop;
    if (c_cap) *c_cap = p->hdr.flop;
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    if (nbins) *nbins = p->hdr.nbins;
    if (npanels) *npanels = (int32_t)p->panels.size();
    return PB_OK;
}

static pb_status fill_numeric(pb_handle *h, const pb_plan *p, const pb_csc *A, const pb_csr *B, void *workspace,
                              size_t ws_bytes, NumericArgs &a) {
    pb_status st = check_operands(h, A, B);
    if (st != PB_OK) return st;
    if (A->nrows != p->m || A->ncols != p->k || B->ncols != p->n || A->nnz != p->nnzA || B->nnz != p->nnzB)
        return fail(h, PB_ERR_SHAPE, "operands differ from the planned structure");
    if (!workspace && p->ws_bytes) return fail(h, PB_ERR_INVALID_ARG, "workspace must not be NULL");
    if (ws_bytes < p->ws_bytes) return fail(h, PB_ERR_WORKSPACE, "workspace smaller than pb_plan_query reported");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return fail(h, PB_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    char *w = static_cast<char *>(workspace);
    a = NumericArgs{};
    a.m = p->m;
    a.k = p->k;
    a.n = p->n;
    a.colptrA = A->colptr;
    a.rowidxA = A->rowidx;
    a.rowptrB = B->rowptr;
    a.colidxB = B->colidx;
    a.valA = A->val;
    a.valB = B->val;
    a.F = p->F;
    a.R = p->R;
    a.ainfo = p->ainfo;
    a.bin_row = p->bin_row;
    a.bin_off = p->bin_off;
    a.chunk_e = p->chunk_e;
    a.acol = p->acol;
    a.aspan = p->aspan;
    a.apos = static_cast<const int64_t *>(p->apos_mem);
    a.flop = p->hdr.flop;
    a.nbins = p->hdr.nbins;
    a.nchunks = p->nchunks;
    a.chunk = p->chunk;
    a.colbits = p->colbits;
    a.capacity = p->capacity;
    a.keys = reinterpret_cast<uint32_t *>(w + p->ws_keys);
    a.cursor = reinterpret_cast<uint64_t *>(w + p->ws_cursor);
    a.cursor_stride = PB_CURSOR_STRIDE;
    a.vals = w + p->ws_vals;
    a.status = reinterpret_cast<uint64_t *>(w + p->ws_status);
    a.ticket = reinterpret_cast<uint32_t *>(w + p->ws_ctrl);
    a.work = reinterpret_cast<uint32_t *>(w + p->ws_ctrl) + 32;  // words 16, 17: oversize row tickets
    a.err = p->err;
    a.dtype = p->dtype;
    a.num_sms = h->num_sms;
    a.over_scan = p->over_scan;
    a.over_tuple_off = p->over_tuple_off;
    a.over_u = reinterpret_cast<int64_t *>(w + p->ws_over_u);
    a.skeys = reinterpret_cast<uint32_t *>(w + p->ws_skeys);
    a.svals = w + p->ws_svals;
    a.over_passes = p->over_passes;
    a.over_dense = p->over_dense;
    a.over_p = reinterpret_cast<int64_t *>(w + p->ws_overp);
    a.packed = p->packed;
    return PB_OK;
}

static OversizeArgs oversize_args(const pb_plan *p, void *workspace, const pb_panel &pn) {
    char *w = static_cast<char *>(workspace);
    OversizeArgs o{};
    o.o_lo = pn.o_lo;
    o.o_hi = pn.o_hi;
    o.c_lo = pn.c_lo;
    o.c_hi = pn.c_hi;
    o.tuple_base = pn.tuple_base;
    o.over_base = pn.over_base;
    o.R = p->R;
    o.bin_row = p->bin_row;
    o.bin_off = p->bin_off;
    o.over_bin = p->over_bin;
    o.over_chunk_off = p->over_chunk_off;
    o.over_tuple_off = p->over_tuple_off;
    o.over_chunk_bin = p->over_chunk_bin;
    o.n_over = p->hdr.n_oversize;
    o.over_chunks = p->hdr.over_chunks;
    o.keys = reinterpret_cast<uint32_t *>(w + p->ws_keys);
    o.vals = w + p->ws_vals;
    o.skeys = reinterpret_cast<uint32_t *>(w + p->ws_skeys);
    o.svals = w + p->ws_svals;
    o.hist = reinterpret_cast<uint32_t *>(w + p->ws_hist);
    o.cinfo = reinterpret_cast<OverChunk *>(w + p->ws_cinfo);
    o.over_u = reinterpret_cast<int64_t *>(w + p->ws_over_u);
    o.dense = p->over_dense;
    o.dense_shift = p->over_shift;
    o.wide = p->dtype == PB_F64_F32TUPLE ? 1 : 0;
    o.row_ticket = reinterpret_cast<uint32_t *>(w + p->ws_ctrl) + 16;  // word 0 is the sort's ticket
    o.row_order = reinterpret_cast<int32_t *>(w + p->ws_overord);
    o.order_cnt = reinterpret_cast<uint32_t *>(w + p->ws_overord + align256(4 * (size_t)p->hdr.n_oversize));
    o.over_p = reinterpret_cast<int64_t *>(w + p->ws_overp);
    return o;
}

// The numeric launch sequence; with panel_done, an event is recorded on the
// stream after each panel's sort (pb_spgemm_host copies that panel's rows of C
// back while the next panel computes).
static pb_status run_numeric(pb_handle *h, const pb_plan *p, const pb_csc *A, const pb_csr *B, pb_csr_out *C,
                             void *workspace, size_t ws_bytes, cudaStream_t s,
                             const std::vector<cudaEvent_t> *panel_done) {
    NumericArgs a;
    pb_status st = fill_numeric(h, p, A, B, workspace, ws_bytes, a);
    if (st != PB_OK) return st;
    if (C->nrows != p->m || C->ncols != p->n) return fail(h, PB_ERR_SHAPE, "C must be A.nrows x B.ncols");
    const bool count_only = C->cap == 0 && !C->colidx && !C->val && !C->rowptr64 && !C->rowptr32;
    if (!count_only && (C->rowptr64 == nullptr) == (C->rowptr32 == nullptr))
        return fail(h, PB_ERR_INVALID_ARG, "exactly one of C.rowptr64 / C.rowptr32 must be set");
    if (C->cap < 0 || (C->cap > 0 && (!C->colidx || !C->val)))
        return fail(h, PB_ERR_INVALID_ARG, "C arrays must not be NULL when cap > 0");
    a.count_only = count_only ? 1 : 0;
    a.rowptr64 = C->rowptr64;
    a.rowptr32 = C->rowptr32;
    a.colidx = C->colidx;
    a.valC = C->val;
    a.nnz_dev = C->nnz_dev;
    a.cap = C->cap;
    const size_t nb = (size_t)p->hdr.nbins;
    char *w = static_cast<char *>(workspace);
    if (h->phase_on) PB_CUDA(h, cudaEventRecord(h->phase_ev[0], s));
    PB_CUDA(h, cudaMemsetAsync(p->err, 0, 4, s));
    if (p->m == 0) {
        // no rows: C is the empty matrix with rowptr = [0]
        if (C->rowptr64) PB_CUDA(h, cudaMemsetAsync(C->rowptr64, 0, 8, s));
        if (C->rowptr32) PB_CUDA(h, cudaMemsetAsync(C->rowptr32, 0, 4, s));
        if (C->nnz_dev) PB_CUDA(h, cudaMemsetAsync(C->nnz_dev, 0, 8, s));
        return PB_OK;
    }
    PB_CUDA(h, reset_cursors(w + p->ws_cursor, p->bin_off, nb, s));
    PB_CUDA(h, cudaMemsetAsync(w + p->ws_status, 0, 8 * nb, s));  // look-back words: all panels
    if (h->phase_on) PB_CUDA(h, cudaEventRecord(h->phase_ev[1], s));
    const bool single = p->panels.size() == 1;
    for (size_t i = 0; i < p->panels.size(); ++i) {
        const pb_panel &pn = p->panels[i];
        // panels run one after another: the look-back chain continues across them
        a.bin_lo = pn.bin_lo;
        a.bin_hi = pn.bin_hi;
        a.tuple_base = pn.tuple_base;
        a.over_base = pn.over_base;
        PB_CUDA(h, cudaMemsetAsync(w + p->ws_ctrl, 0, 256, s));
        PB_CUDA(h, launch_expand(a, s));
        if (pn.o_hi > pn.o_lo)
            PB_CUDA(h, launch_oversize(oversize_args(p, workspace, pn), p->over_passes, p->dtype, h->num_sms, s));
        if (h->phase_on && single) PB_CUDA(h, cudaEventRecord(h->phase_ev[2], s));
        PB_CUDA(h, launch_binsort(a, s));
        if (pn.o_hi > pn.o_lo && p->over_dense && !count_only) {
            OversizeArgs o = oversize_args(p, workspace, pn);
            o.colidxC = C->colidx;
            o.valC = C->val;
            PB_CUDA(h, launch_oversize_emit(o, p->dtype, h->num_sms, s));
        }
        if (panel_done) PB_CUDA(h, cudaEventRecord((*panel_done)[i], s));
    }
    if (h->phase_on) {
        if (!single) PB_CUDA(h, cudaEventRecord(h->phase_ev[2], s));
        PB_CUDA(h, cudaEventRecord(h->phase_ev[3], s));
    }
    return PB_OK;
}

pb_status pb_spgemm_numeric(pb_handle *h, const pb_plan *p, const pb_csc *A, const pb_csr *B, pb_csr_out *C,
                            void *workspace, size_t ws_bytes, pb_stream_t stream_) {
    if (!h || !p || !C) return PB_ERR_INVALID_ARG;
    h->last_error.clear();
    return run_numeric(h, p, A, B, C, workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream_), nullptr);
}

// Device buffers of one pb_spgemm_host call, released on every exit path.
struct HostCall {
    pb_handle *h;
    cudaStream_t s;
    std::vector<std::pair<void *, size_t>> bufs;
    std::vector<cudaEvent_t> events;
    pb_plan *plan = nullptr;
    void *get(size_t bytes) {
        void *p = h->alloc(bytes ? bytes : 256, reinterpret_cast<pb_stream_t>(s), h->ctx);
        if (p) bufs.push_back({p, bytes ? bytes : 256});
        return p;
    }
    cudaEvent_t event() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        events.push_back(e);
        return e;
    }
    ~HostCall() {
        (void)cudaStreamSynchronize(s);
        if (h->copy_stream) (void)cudaStreamSynchronize(h->copy_stream);
        if (plan) pb_plan_destroy(plan);
        for (auto &b : bufs) h->free_fn(b.first, b.second, reinterpret_cast<pb_stream_t>(s), h->ctx);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
    }
};

pb_status pb_spgemm_host(pb_handle *h, const pb_csc *A, const pb_csr *B, pb_dtype dtype, const pb_config *cfg,
                         pb_csr_host *C, pb_stream_t stream_, pb_status *device_status) {
    if (!h || !C || !device_status) return PB_ERR_INVALID_ARG;
    h->last_error.clear();
    pb_status st = check_operands(h, A, B);
    if (st != PB_OK) return st;
    if (!valid_dtype(dtype)) return fail(h, PB_ERR_UNSUPPORTED_DTYPE, "unknown dtype");
    if (C->nrows != A->nrows || C->ncols != B->ncols) return fail(h, PB_ERR_SHAPE, "C must be A.nrows x B.ncols");
    if (!C->rowptr || C->cap < 0 || (C->cap > 0 && (!C->colidx || !C->val)))
        return fail(h, PB_ERR_INVALID_ARG, "C host arrays");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    if (!h->copy_stream) PB_CUDA(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    if (!h->small_stream) PB_CUDA(h, cudaStreamCreateWithFlags(&h->small_stream, cudaStreamNonBlocking));
    cudaStream_t sc = h->copy_stream, sr = h->small_stream;
    HostCall call{h, s};
    const size_t vin = dtype == PB_F32 ? 4 : 8, vout = vin;
    const int32_t m = A->nrows, k = A->ncols, n = B->ncols;
    // device copies of the operands; the value arrays go on the copy stream and
    // overlap with the symbolic phase, which needs only the pointer and row-index arrays
    int32_t *dcolptr = static_cast<int32_t *>(call.get(4 * ((size_t)k + 1)));
    int32_t *drowidx = static_cast<int32_t *>(call.get(4 * (size_t)A->nnz));
    void *dvalA = call.get(vin * (size_t)A->nnz);
    int32_t *drowptr = static_cast<int32_t *>(call.get(4 * ((size_t)k + 1)));
    int32_t *dcolidx = static_cast<int32_t *>(call.get(4 * (size_t)B->nnz));
    void *dvalB = call.get(vin * (size_t)B->nnz);
    if (!dcolptr || !drowidx || !dvalA || !drowptr || !dcolidx || !dvalB)
        return fail(h, PB_ERR_OOM, "operand allocation failed");
    cudaEvent_t ev_alloc = call.event(), ev_vals = call.event();
    if (!ev_alloc || !ev_vals) return fail(h, PB_ERR_CUDA, "event creation failed");
    PB_CUDA(h, cudaMemcpyAsync(dcolptr, A->colptr, 4 * ((size_t)k + 1), cudaMemcpyHostToDevice, s));
    PB_CUDA(h, cudaMemcpyAsync(drowptr, B->rowptr, 4 * ((size_t)k + 1), cudaMemcpyHostToDevice, s));
    if (A->nnz) PB_CUDA(h, cudaMemcpyAsync(drowidx, A->rowidx, 4 * (size_t)A->nnz, cudaMemcpyHostToDevice, s));
    PB_CUDA(h, cudaEventRecord(ev_alloc, s));
    PB_CUDA(h, cudaStreamWaitEvent(sc, ev_alloc, 0));
    if (A->nnz) PB_CUDA(h, cudaMemcpyAsync(dvalA, A->val, vin * (size_t)A->nnz, cudaMemcpyHostToDevice, sc));
    if (B->nnz) PB_CUDA(h, cudaMemcpyAsync(dcolidx, B->colidx, 4 * (size_t)B->nnz, cudaMemcpyHostToDevice, sc));
    if (B->nnz) PB_CUDA(h, cudaMemcpyAsync(dvalB, B->val, vin * (size_t)B->nnz, cudaMemcpyHostToDevice, sc));
    PB_CUDA(h, cudaEventRecord(ev_vals, sc));
    const pb_csc dA{m, k, A->nnz, dcolptr, drowidx, dvalA};
    const pb_csr dB{k, n, B->nnz, drowptr, dcolidx, dvalB};
    pb_config c2{};
    if (cfg) c2 = *cfg;
    if (c2.min_panels == 0) c2.min_panels = 6;
    st = pb_spgemm_symbolic(h, &dA, &dB, dtype, &c2, stream_, &call.plan);
    if (st != PB_OK) {
        call.plan = nullptr;
        return st;
    }
    const pb_plan *p = call.plan;
    const int64_t flop = p->hdr.flop;
    const int64_t cap = flop > 0 ? flop : 1;
    int64_t *drp = static_cast<int64_t *>(call.get(8 * ((size_t)m + 1)));
    int32_t *dci = static_cast<int32_t *>(call.get(4 * (size_t)cap));
    void *dva = call.get(vout * (size_t)cap);
    void *ws = call.get(p->ws_bytes);
    if (!drp || !dci || !dva || !ws) return fail(h, PB_ERR_OOM, "output or workspace allocation failed");
    std::vector<cudaEvent_t> done(p->panels.size());
    for (cudaEvent_t &e : done)
        if (!(e = call.event())) return fail(h, PB_ERR_CUDA, "event creation failed");
    PB_CUDA(h, cudaStreamWaitEvent(s, ev_vals, 0));
    pb_csr_out dC{m, n, cap, drp, nullptr, dci, dva, nullptr};
    st = run_numeric(h, p, &dA, &dB, &dC, ws, p->ws_bytes, s, &done);
    if (st != PB_OK) return st;
    // each panel's rows of C: [prefix before it, its last bin's inclusive prefix)
    const uint64_t *status = reinterpret_cast<const uint64_t *>(static_cast<char *>(ws) + p->ws_status);
    int64_t begin = 0;
    bool overflow = false;
    for (size_t i = 0; i < p->panels.size() && m > 0; ++i) {
        const pb_panel &pn = p->panels[i];
        uint64_t word = 0;
        PB_CUDA(h, cudaStreamWaitEvent(sr, done[i], 0));
        if (pn.bin_hi > pn.bin_lo) {
            PB_CUDA(h, cudaMemcpyAsync(&word, status + (pn.bin_hi - 1), 8, cudaMemcpyDeviceToHost, sr));
            PB_CUDA(h, cudaStreamSynchronize(sr));
        }
        const int64_t end = pn.bin_hi > pn.bin_lo ? (int64_t)(word & LB_VALUE_MASK) : begin;
        if (end > C->cap) overflow = true;
        if (!overflow && end > begin) {
            PB_CUDA(h, cudaStreamWaitEvent(sc, done[i], 0));
            PB_CUDA(h, cudaMemcpyAsync(C->colidx + begin, dci + begin, 4 * (size_t)(end - begin),
                                       cudaMemcpyDeviceToHost, sc));
            PB_CUDA(h, cudaMemcpyAsync(static_cast<char *>(C->val) + vout * (size_t)begin,
                                       static_cast<char *>(dva) + vout * (size_t)begin, vout * (size_t)(end - begin),
                                       cudaMemcpyDeviceToHost, sc));
        }
        begin = end;
    }
    if (!done.empty()) PB_CUDA(h, cudaStreamWaitEvent(sc, done.back(), 0));
    PB_CUDA(h, cudaMemcpyAsync(C->rowptr, drp, 8 * ((size_t)m + 1), cudaMemcpyDeviceToHost, sc));
    PB_CUDA(h, cudaStreamSynchronize(sc));
    pb_status dev = PB_OK;
    PB_CUDA(h, cudaStreamSynchronize(s));
    st = pb_plan_status(p, stream_, &dev);
    if (st != PB_OK) return st;
    C->nnz = m > 0 ? begin : 0;
    *device_status = overflow ? PB_ERR_OVERFLOW : dev;
    return PB_OK;
}

pb_status pb_validate_operands(pb_handle *h, const pb_csc *A, const pb_csr *B, pb_stream_t stream_,
                               pb_status *result) {
    if (!h || !result) return PB_ERR_INVALID_ARG;
    h->last_error.clear();
    pb_status st = check_operands(h, A, B);
    if (st != PB_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    uint32_t *bad = static_cast<uint32_t *>(h->alloc(256, stream_, h->ctx));
    if (!bad) return fail(h, PB_ERR_OOM, "validation flag");
    uint32_t word = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, 4, s);
    if (e == cudaSuccess) e = launch_validate(*A, *B, bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    h->free_fn(bad, 256, stream_, h->ctx);
    if (e != cudaSuccess) return cuda_fail(h, e, "pb_validate_operands");
    *result = word ? PB_ERR_INVALID_ARG : PB_OK;
    if (word) {
        std::string msg;
        if (word & 1u) msg += "A.colptr is not a pointer array (0 first, monotone, nnz last); ";
        if (word & 2u) msg += "B.rowptr is not a pointer array (0 first, monotone, nnz last); ";
        if (word & 4u) msg += "A.rowidx has an index outside [0, A.nrows); ";
        if (word & 8u) msg += "B.colidx has an index outside [0, B.ncols); ";
        h->last_error = msg;
    }
    return PB_OK;
}

pb_status pb_set_phase_events(pb_handle *h, void *const *events) {
    if (!h) return PB_ERR_INVALID_ARG;
    h->phase_on = events != nullptr;
    for (int i = 0; i < 4; ++i) h->phase_ev[i] = events ? static_cast<cudaEvent_t>(events[i]) : nullptr;
    if (events)
        for (int i = 0; i < 4; ++i)
            if (!h->phase_ev[i]) {
                h->phase_on = false;
                return fail(h, PB_ERR_INVALID_ARG, "all four events are required");
            }
    return PB_OK;
}

int64_t pb_kernel_launches(void) { return pb::g_launches.load(); }

pb_status pb_debug_expand(pb_handle *h, const pb_plan *p, const pb_csc *A, const pb_csr *B, void *workspace,
                          size_t ws_bytes, pb_stream_t stream_) {
    if (!h || !p) return PB_ERR_INVALID_ARG;
    NumericArgs a;
    pb_status st = fill_numeric(h, p, A, B, workspace, ws_bytes, a);
    if (st != PB_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    char *w = static_cast<char *>(workspace);
    const pb_panel &pn = p->panels.front();  // the first panel's tuples
    a.bin_lo = pn.bin_lo;
    a.bin_hi = pn.bin_hi;
    a.tuple_base = pn.tuple_base;
    a.over_base = pn.over_base;
    PB_CUDA(h, reset_cursors(w + p->ws_cursor, p->bin_off, (size_t)p->hdr.nbins, s));
    PB_CUDA(h, cudaMemsetAsync(w + p->ws_ctrl, 0, 256, s));
    PB_CUDA(h, launch_expand(a, s));
    return PB_OK;
}

size_t pb_debug_values_offset(const pb_plan *p) { return p ? p->ws_vals : 0; }

int32_t pb_debug_tuple_layout(const pb_plan *p) { return p ? p->packed : 0; }

pb_status pb_plan_status(const pb_plan *p, pb_stream_t stream_, pb_status *device_status) {
    if (!p || !device_status) return PB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    uint32_t word = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&word, p->err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p->h, e, "plan status");
    *device_status = status_of_word(word);
    return PB_OK;
}

pb_status pb_plan_export(const pb_plan *p, int64_t *F, int64_t *R, int32_t *bin_row, int64_t *bin_off,
                         pb_stream_t stream_) {
    if (!p) return PB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    pb_handle *h = p->h;
    const size_t nb = (size_t)p->hdr.nbins;
    if (F) PB_CUDA(h, cudaMemcpyAsync(F, p->F, 8 * ((size_t)p->k + 1), cudaMemcpyDeviceToDevice, s));
    if (R) PB_CUDA(h, cudaMemcpyAsync(R, p->R, 8 * ((size_t)p->m + 1), cudaMemcpyDeviceToDevice, s));
    if (bin_row) PB_CUDA(h, cudaMemcpyAsync(bin_row, p->bin_row, 4 * (nb + 1), cudaMemcpyDeviceToDevice, s));
    if (bin_off) PB_CUDA(h, cudaMemcpyAsync(bin_off, p->bin_off, 8 * (nb + 1), cudaMemcpyDeviceToDevice, s));
    PB_CUDA(h, cudaStreamSynchronize(s));
    return PB_OK;
}

pb_status pb_plan_destroy(pb_plan *p) {
    if (!p) return PB_OK;
    free_plan_memory(p);
    delete p;
    return PB_OK;
}

}  // extern "C"
