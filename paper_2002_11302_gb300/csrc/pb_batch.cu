// Batched products: C_i = A_i * B_i for many independent products in one pass
// of the method.  Each product still follows Alg. 3 (flop per column, per-row
// flop of Sec. III-B, row-range bins), the expand of Alg. 2 and the on-chip
// sort and merge of Sec. III-D/E; only the launches are shared.
//
// Layout.  The products are placed back to back in three global index spaces:
// rows (of A and C), columns of A (= rows of B) and A entries.  Each space is
// cut into tiles of BATCH_TILE elements that never straddle two products, so a
// CTA finds the product of its tile with one binary search over the products'
// first tiles.  Bins are cut per product (a product's first row always starts
// a bin) and numbered globally; the sort's look-back restarts at each
// product's first bin, so prefixes (= C offsets) are product-local and every
// bin writes straight into its own product's C.
//
// Rows above their product's bin capacity (hub rows, Sec. III-D) are listed on
// the device while the bins are cut, merged in dense column tiles after the
// expand (the single-product oversize kernels, reading the list's size from
// the device), published in their product's look-back chain by the sort and
// copied into C after it.  Their scratch follows the bins' tuples in the same
// buffer.
//
// Everything the kernels need is computed on the device: the host only packs
// the products' pointers and sizes into launch parameters, so a call makes no
// host-device copy and no host synchronisation and can be captured into a
// CUDA graph.  Grids are persistent (sized from the SM count) and read the
// actual work counts (bins, expand work items) from a device header.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pb_common.cuh"
#include "pb_host.h"

using namespace pb;

namespace {

constexpr int DESC_PER_LAUNCH = 160;  // products per descriptor-writing launch (~25 KB of parameters)
constexpr int MIN_CHUNK = 256;        // smallest expand work item (sizes the work-item table)
constexpr int NLEVELS = 3;            // bin capacities 2048, 4096, 8192: one sort launch each
constexpr int32_t MAX_COUNT = 1 << 20;
constexpr int LONG_COL = 32;
constexpr int T = 256;                // threads of the tile kernels

const int32_t kLevelCap[NLEVELS] = {2048, 4096, 8192};

int level_of(int32_t cap) {
    for (int l = 0; l < NLEVELS; ++l)
        if (kLevelCap[l] == cap) return l;
    return -1;
}

struct DescBlock {
    int32_t first, n, count;
    int32_t tiles_total[3];
    BatchDesc d[DESC_PER_LAUNCH];
    int32_t tiles[DESC_PER_LAUNCH][3];  // first tile of the product: rows, columns, entries
};
static_assert(sizeof(DescBlock) < 32000, "kernel parameter block too large");

struct LevelRows {
    int32_t row[NLEVELS + 1];  // first global row of each level; row[NLEVELS] = total rows
};

// Device arrays of one batch, carved from the caller's workspace.
struct BatchWs {
    BatchHeader *bhdr;
    uint32_t *err, *tickets, *n_long, *n_over, *row_ticket;
    BatchDesc *desc;
    BatchProd *prod;
    int32_t *tiles_m, *tiles_k, *tiles_e;
    int64_t *F, *R, *flags;
    uint64_t *rowinfo, *ainfo;
    int32_t *acol;
    int2 *aspan;
    int64_t *long_cols;
    int32_t *bin_row, *bin_prod;
    int64_t *bin_off;
    uint64_t *cursor, *status;
    int32_t *chunk_e, *chunk_prod;
    int64_t *scan_tmp;
    uint32_t *keys;
    void *vals;
    int64_t chunk_cap, tuple_cap;
    // rows above the bin capacity (oversize bins)
    int64_t *over_scan;   // [M+2] index in the oversize list of an oversize bin
    int64_t *over_count;  // [3] oversize bins, their work items (both 0 unless everything fits),
                          // offset of the work items' histograms in `keys`
    uint32_t *order_cnt;  // [128]
    int64_t *over_bin, *over_chunk_off, *over_tuple_off, *over_u, *over_p;  // [n_over_cap (+1)]
    int32_t *row_order;       // [n_over_cap]
    int32_t *over_chunk_bin;  // [ochunk_cap]
    int64_t n_over_cap, ochunk_cap;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carver {
    char *base;
    size_t off = 0;
    template <class P>
    P *take(size_t bytes) {
        off = align256(off);
        P *p = base ? reinterpret_cast<P *>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

// Fixed part of the layout (everything but the work-item table and tuples).
size_t carve_fixed(BatchWs &w, char *base, int32_t count, int64_t M, int64_t K, int64_t E) {
    Carver c{base};
    w.bhdr = c.take<BatchHeader>(sizeof(BatchHeader));
    uint32_t *ctrl = c.take<uint32_t>(256);
    w.err = ctrl;
    w.n_long = ctrl ? ctrl + 1 : nullptr;
    w.tickets = ctrl ? ctrl + 8 : nullptr;     // one per capacity level
    w.row_ticket = ctrl ? ctrl + 16 : nullptr;  // [2] oversize rows taken by the dense and copy kernels
    w.n_over = ctrl ? ctrl + 20 : nullptr;      // words 32.. hold the expand's work counter
    w.desc = c.take<BatchDesc>(sizeof(BatchDesc) * (size_t)count);
    w.prod = c.take<BatchProd>(sizeof(BatchProd) * (size_t)count);
    w.tiles_m = c.take<int32_t>(4 * ((size_t)count + 1));
    w.tiles_k = c.take<int32_t>(4 * ((size_t)count + 1));
    w.tiles_e = c.take<int32_t>(4 * ((size_t)count + 1));
    w.F = c.take<int64_t>(8 * ((size_t)K + 1));
    w.R = c.take<int64_t>(8 * ((size_t)M + 1));
    w.flags = c.take<int64_t>(8 * ((size_t)M + 1));
    w.rowinfo = c.take<uint64_t>(8 * (size_t)M);
    w.ainfo = c.take<uint64_t>(8 * (size_t)E);
    w.acol = c.take<int32_t>(4 * (size_t)E);
    w.aspan = c.take<int2>(8 * (size_t)E);
    w.long_cols = c.take<int64_t>(8 * (size_t)K);
    w.bin_row = c.take<int32_t>(4 * ((size_t)M + 2));
    w.bin_prod = c.take<int32_t>(4 * ((size_t)M + 2));
    w.bin_off = c.take<int64_t>(8 * ((size_t)M + 2));
    w.cursor = c.take<uint64_t>(8 * ((size_t)M + 1));
    w.status = c.take<uint64_t>(8 * ((size_t)M + 1));
    w.over_scan = c.take<int64_t>(8 * ((size_t)M + 2));
    w.over_count = c.take<int64_t>(24);
    w.order_cnt = c.take<uint32_t>(512);
    const int64_t scan_n = std::max<int64_t>(std::max<int64_t>(M, K), 1);
    w.scan_tmp = c.take<int64_t>(8 * (size_t)scan_tmp_elems(scan_n));
    return align256(c.off);
}

constexpr size_t kSlack = 1024;

// Oversize rows hold more than BATCH_MIN_CAPACITY tuples each, so `tuples`
// slots bound their number, and their OVER_CHUNK-tuple work items (a row of
// N > OVER_CHUNK / 2 tuples has ceil(N / OVER_CHUNK) < 2N / OVER_CHUNK).
int64_t n_over_cap_of(int64_t tuples) { return tuples / BATCH_MIN_CAPACITY + 1; }
int64_t ochunk_cap_of(int64_t tuples) { return tuples / (OVER_CHUNK / 2) + 1; }

size_t over_bytes(int64_t tuples) {
    const size_t no = (size_t)n_over_cap_of(tuples), oc = (size_t)ochunk_cap_of(tuples);
    return 5 * align256(8 * (no + 1)) + align256(4 * no) + align256(4 * oc);
}

// Bytes of the work-item table, the tuples and the oversize-row arrays for `tuples` slots.
size_t tail_bytes(int64_t tuples, int32_t count, size_t tb) {
    const int64_t chunks = tuples / MIN_CHUNK + count + 2;
    return align256(4 * ((size_t)chunks + 1)) + align256(4 * (size_t)chunks) + align256(4 * (size_t)tuples) +
           align256(tb * (size_t)tuples) + over_bytes(tuples) + kSlack;
}

// Carve the work-item table and the tuples from what the workspace has left.
void carve_tail(BatchWs &w, char *base, size_t fixed, size_t ws_bytes, int32_t count, size_t tb) {
    w.chunk_cap = 0;
    w.tuple_cap = 0;
    if (ws_bytes <= fixed + kSlack + 8 * ((size_t)count + 4)) return;
    const size_t rem = ws_bytes - fixed - kSlack - 8 * ((size_t)count + 4);
    // Per tuple slot: 4 key bytes, tb value bytes, 8/MIN_CHUNK bytes of work-item
    // table and the oversize-row arrays (44 bytes per BATCH_MIN_CAPACITY slots,
    // 4 per OVER_CHUNK / 2).  Leaving out the arrays' rounding to 256 bytes makes
    // this an upper bound, so stepping down finds the largest count that fits,
    // which is at least the count pb_spgemm_batch_query sized the workspace for.
    const double per = 4.0 + (double)tb + 8.0 / MIN_CHUNK + 44.0 / BATCH_MIN_CAPACITY + 8.0 / OVER_CHUNK;
    int64_t tuples = (int64_t)((double)rem / per);
    tuples &= ~int64_t(3);
    while (tuples > 0 && fixed + tail_bytes(tuples, count, tb) > ws_bytes) tuples -= 4;
    if (tuples <= 0) return;
    Carver c{base};
    c.off = fixed;
    const int64_t chunks = tuples / MIN_CHUNK + count + 2;
    w.chunk_e = c.take<int32_t>(4 * ((size_t)chunks + 1));
    w.chunk_prod = c.take<int32_t>(4 * (size_t)chunks);
    w.keys = c.take<uint32_t>(4 * (size_t)tuples);
    w.vals = c.take<char>(tb * (size_t)tuples);
    const size_t no = (size_t)n_over_cap_of(tuples), oc = (size_t)ochunk_cap_of(tuples);
    w.over_bin = c.take<int64_t>(8 * (no + 1));
    w.over_chunk_off = c.take<int64_t>(8 * (no + 1));
    w.over_tuple_off = c.take<int64_t>(8 * (no + 1));
    w.over_u = c.take<int64_t>(8 * (no + 1));
    w.over_p = c.take<int64_t>(8 * (no + 1));
    w.row_order = c.take<int32_t>(4 * no);
    w.over_chunk_bin = c.take<int32_t>(4 * oc);
    w.chunk_cap = chunks;
    w.tuple_cap = tuples;
    w.n_over_cap = (int64_t)no;
    w.ochunk_cap = (int64_t)oc;
}

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------

// Product owning tile t: the last p with tiles[p] <= t (tiles[0] = 0 <= t < tiles[count]).
__device__ inline int find_prod(const int32_t *__restrict__ tiles, int32_t count, int64_t t) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tiles[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ inline unsigned long long block_max_u64(unsigned long long v, unsigned long long *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(FULL, v, o);
        v = t > v ? t : v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = sh[w] > r ? sh[w] : r;
    __syncthreads();
    return r;
}

__global__ void k_bdesc(const DescBlock blk, BatchDesc *desc, BatchProd *prod, int32_t *tiles_m, int32_t *tiles_k,
                        int32_t *tiles_e) {
    const int i = threadIdx.x;
    if (i < blk.n) {
        const int q = blk.first + i;
        desc[q] = blk.d[i];
        prod[q] = BatchProd{0, 0, 0, -1, 0, 0};
        tiles_m[q] = blk.tiles[i][0];
        tiles_k[q] = blk.tiles[i][1];
        tiles_e[q] = blk.tiles[i][2];
    }
    if (i == 0 && blk.first + blk.n == blk.count) {
        tiles_m[blk.count] = blk.tiles_total[0];
        tiles_k[blk.count] = blk.tiles_total[1];
        tiles_e[blk.count] = blk.tiles_total[2];
    }
}

// Alg. 3 per product: f_k = nnz(A(:,k)) * nnz(B(k,:)) for every column (one
// thread per column), the product's flop total, and the column of each A
// entry (columns with many entries are listed for a warp-wide pass).
__global__ void __launch_bounds__(T) k_bflop(int32_t count, const BatchDesc *__restrict__ desc,
                                             const int32_t *__restrict__ tiles_k, int64_t *F, int32_t *acol,
                                             int64_t *long_cols, uint32_t *n_long, BatchProd *prod) {
    __shared__ int64_t scratch[40];
    const int64_t ntiles = tiles_k[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_k, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_k[q]) * (int64_t)BATCH_TILE;
        int64_t f = 0;
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t kk = lo + j;
            if (kk < d.k) {
                const int32_t a0 = d.colptrA[kk], a1 = d.colptrA[kk + 1];
                const int64_t fk = (int64_t)(a1 - a0) * ((int64_t)d.rowptrB[kk + 1] - d.rowptrB[kk]);
                F[d.kstart + kk] = fk;
                f += fk;
                if (a1 - a0 > LONG_COL) {
                    long_cols[atomicAdd(n_long, 1u)] = ((int64_t)q << 32) | kk;
                } else {
                    for (int32_t e = a0; e < a1; ++e) acol[d.estart + e] = (int32_t)kk;
                }
            }
        }
        const int64_t tot = block_reduce_sum<int64_t, T>(f, scratch);
        if (threadIdx.x == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long *>(&prod[q].flop), (unsigned long long)tot);
    }
}

__global__ void k_bacol_long(const BatchDesc *__restrict__ desc, const int64_t *long_cols, const uint32_t *n_long,
                             int32_t *acol) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = *n_long;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int64_t item = long_cols[i];
        const BatchDesc &d = desc[item >> 32];
        const int32_t kk = (int32_t)(item & 0xffffffffll);
        for (int32_t e = d.colptrA[kk] + lane; e < d.colptrA[kk + 1]; e += 32) acol[d.estart + e] = kk;
    }
}

// Per product: the first expand work item (work items of `chunk` tuples, as
// for a single product), the empty products' C, and the work-item total.
__global__ void __launch_bounds__(1024) k_bprod(int32_t count, const BatchDesc *__restrict__ desc, BatchProd *prod,
                                                BatchHeader *bh, uint32_t *err, int64_t chunk_cap, int32_t *chunk_e,
                                                int32_t E) {
    __shared__ int64_t scratch[40];
    int64_t carry = 0;
    for (int base = 0; base < count; base += 1024) {
        const int q = base + threadIdx.x;
        int64_t nch = 0;
        if (q < count) {
            const BatchDesc &d = desc[q];
            const int64_t f = prod[q].flop;
            nch = f > 0 ? ceil_div<int64_t>(f, d.chunk) : 0;
            if (d.m == 0) {  // no rows: C is empty with rowptr = [0]
                if (d.rowptr64) d.rowptr64[0] = 0;
                if (d.rowptr32) d.rowptr32[0] = 0;
                if (d.nnz_dev) *d.nnz_dev = 0;
            }
        }
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t, 1024>(nch, scratch, &tot);
        if (q < count) prod[q].chunk_base = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        bh->nchunks = carry;
        if (carry > chunk_cap)
            atomicOr(err, DEV_ERR_WORKSPACE);
        else
            chunk_e[carry] = E;
    }
}

// Per-row flop (Sec. III-B): every A(i,k) adds nnz(B(k,:)) to row i.
__global__ void __launch_bounds__(T) k_brow_flop(int32_t count, const BatchDesc *__restrict__ desc,
                                                 const int32_t *__restrict__ tiles_e, const int32_t *__restrict__ acol,
                                                 int64_t *R) {
    const int64_t ntiles = tiles_e[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_e, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_e[q]) * (int64_t)BATCH_TILE;
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t e = lo + j;
            if (e < d.nnzA) {
                const int32_t kk = acol[d.estart + e];
                const int64_t lb = (int64_t)d.rowptrB[kk + 1] - d.rowptrB[kk];
                if (lb)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&R[d.mstart + d.rowidxA[e]]),
                              (unsigned long long)lb);
            }
        }
    }
}

// Largest light row (r <= capacity / 2) and largest row of each product, and
// the oversize-row tuples at the smallest capacity (the workspace query's
// bound).  A row above the product's bin capacity is merged in dense tiles; a
// product whose columns are too wide for them cannot have one: the batch stops.
__global__ void __launch_bounds__(T) k_bmax(int32_t count, const BatchDesc *__restrict__ desc,
                                            const int32_t *__restrict__ tiles_m, const int64_t *__restrict__ R,
                                            BatchProd *prod, uint32_t *err) {
    __shared__ unsigned long long sh[32];
    __shared__ int64_t scratch[40];
    const int64_t ntiles = tiles_m[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_m, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_m[q]) * (int64_t)BATCH_TILE;
        const int64_t heavy = d.capacity / 2;
        unsigned long long light = 0, top = 0;
        int64_t ob = 0;
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t i = lo + j;
            if (i < d.m) {
                const int64_t g = d.mstart + i;
                const unsigned long long r = (unsigned long long)(R[g + 1] - R[g]);
                if ((int64_t)r <= heavy && r > light) light = r;
                if (r > top) top = r;
                if (r > (unsigned long long)BATCH_MIN_CAPACITY)  // scratch tuples and digit histograms
                    ob += (int64_t)((r + 3) & ~3ull) + 256 * (int64_t)ceil_div<unsigned long long>(r, OVER_CHUNK);
            }
        }
        light = block_max_u64(light, sh);
        top = block_max_u64(top, sh);
        ob = block_reduce_sum<int64_t, T>(ob, scratch);
        if (threadIdx.x == 0) {
            if (light) atomicMax(&prod[q].max_light, light);
            if (top) atomicMax(&prod[q].max_row, top);
            if (ob) atomicAdd(reinterpret_cast<unsigned long long *>(&prod[q].over_bound), (unsigned long long)ob);
            if ((int64_t)top > d.capacity && !d.over_ok) atomicOr(err, DEV_ERR_HEAVY_ROW);
        }
    }
}

// Bin starts, cut per product with its own capacity and row limit (the rule
// of the single-product symbolic phase; a product's first row starts a bin).
__global__ void __launch_bounds__(T) k_bflags(int32_t count, const BatchDesc *__restrict__ desc,
                                              const int32_t *__restrict__ tiles_m, const int64_t *__restrict__ R,
                                              const BatchProd *__restrict__ prod, int64_t *flags) {
    const int64_t ntiles = tiles_m[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_m, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_m[q]) * (int64_t)BATCH_TILE;
        const int64_t heavy = d.capacity / 2;
        const int64_t win = d.capacity - (int64_t)prod[q].max_light;  // >= capacity / 2
        const int64_t rmask = (1ll << d.rmax_log2) - 1;
        const int64_t R0 = R[d.mstart];
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t i = lo + j;
            if (i >= d.m) continue;
            const int64_t g = d.mstart + i;
            bool start = i == 0 || (i & rmask) == 0;
            if (!start)
                start = (R[g] - R0) / win != (R[g - 1] - R0) / win || R[g + 1] - R[g] > heavy ||
                        R[g] - R[g - 1] > heavy;
            flags[g] = start ? 1 : 0;
        }
    }
}

// flags holds the exclusive scan of the bin starts (flags[M] = bins).  A bin
// whose single row is above the product's capacity joins the oversize list.
__global__ void __launch_bounds__(T) k_bbin_rows(int32_t count, const BatchDesc *__restrict__ desc,
                                                 const int32_t *__restrict__ tiles_m, const int64_t *__restrict__ flags,
                                                 const int64_t *__restrict__ R, int32_t M, int32_t *bin_row,
                                                 int32_t *bin_prod, BatchProd *prod, BatchHeader *bh, LevelRows lv,
                                                 int64_t *over_scan, int64_t *over_bin, uint32_t *n_over,
                                                 int64_t n_over_cap, uint32_t *err) {
    const int64_t ntiles = tiles_m[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_m, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_m[q]) * (int64_t)BATCH_TILE;
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t i = lo + j;
            if (i >= d.m) continue;
            const int64_t g = d.mstart + i;
            const int64_t f = flags[g];
            if (flags[g + 1] != f) {
                bin_row[f] = (int32_t)g;
                bin_prod[f] = q;
                if (i == 0) prod[q].first_bin = f;
                // a row above capacity / 2 is a bin of its own (k_bflags)
                if (R[g + 1] - R[g] > d.capacity) {
                    const uint32_t o = atomicAdd(n_over, 1u);
                    if (o < n_over_cap) {
                        over_bin[o] = f;
                        over_scan[f] = o;
                    } else {
                        atomicOr(err, DEV_ERR_WORKSPACE);
                    }
                }
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t nb = flags[M];
        bin_row[nb] = M;
        bin_prod[nb] = -1;
        bh->nbins = nb;
        for (int l = 0; l <= NLEVELS; ++l) bh->level_bins[l] = flags[lv.row[l]];
    }
}

__global__ void __launch_bounds__(T) k_browinfo(int32_t count, const BatchDesc *__restrict__ desc,
                                                const int32_t *__restrict__ tiles_m, const int64_t *__restrict__ flags,
                                                const int32_t *__restrict__ bin_row, uint64_t *rowinfo) {
    const int64_t ntiles = tiles_m[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_m, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_m[q]) * (int64_t)BATCH_TILE;
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t i = lo + j;
            if (i >= d.m) continue;
            const int64_t g = d.mstart + i;
            const int64_t f = flags[g];
            const int64_t bin = (flags[g + 1] != f) ? f : f - 1;
            const uint32_t local = (uint32_t)(g - bin_row[bin]);
            rowinfo[g] = ((uint64_t)bin << 32) | (uint64_t)(local << d.colbits);
        }
    }
}

// Bin b's tuples start at round4(R[first row]) + 4b: 16-byte aligned, and
// consecutive bins never overlap (bin b holds R[row1] - R[row0] tuples and the
// next start is at least that much later).  No scan over the bins is needed.
// Cursors start at the bin offsets, look-back words at zero.
__global__ void k_bbin_off(const int64_t *__restrict__ R, const int32_t *__restrict__ bin_row, int32_t M,
                           BatchHeader *bh, int64_t tuple_cap, int64_t *bin_off, uint64_t *cursor, uint64_t *status,
                           uint32_t *err) {
    const int64_t nb = bh->nbins;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = ((R[bin_row[b]] + 3) & ~int64_t(3)) + 4 * b;
        bin_off[b] = off;
        cursor[b] = (uint64_t)off;
        status[b] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t tot = ((R[M] + 3) & ~int64_t(3)) + 4 * nb;
        bin_off[nb] = tot;
        bh->tuples = tot;
        if (tot > tuple_cap) atomicOr(err, DEV_ERR_WORKSPACE);
    }
}

// The oversize list's work items and scratch (one CTA): per oversize bin its
// first OVER_CHUNK-tuple work item and its scratch offset.  The scratch follows
// the bins' tuples in the tuple buffer and the work items' 256-entry digit
// histograms follow the scratch (in the key array); then the work item -> bin
// map.  The counts stay 0 (no oversize kernel does any work) unless
// everything fits.
__global__ void __launch_bounds__(1024) k_bover(const int64_t *__restrict__ R, const int32_t *__restrict__ bin_row,
                                                const int64_t *__restrict__ over_bin, const uint32_t *n_over,
                                                int64_t n_over_cap, int64_t ochunk_cap, int64_t tuple_cap,
                                                const BatchHeader *bh, uint32_t *err, int64_t *over_chunk_off,
                                                int64_t *over_tuple_off, int32_t *over_chunk_bin,
                                                int64_t *over_count) {
    __shared__ int64_t scratch[40];
    __shared__ int32_t fits;
    const int tid = threadIdx.x;
    const int64_t n = (*err & DEV_ERR_BATCH_FATAL) ? 0 : min((int64_t)*n_over, n_over_cap);
    const int64_t base = (bh->tuples + 3) & ~int64_t(3);
    int64_t cc = 0, tc = 0;
    for (int64_t o0 = 0; o0 < n; o0 += 1024) {
        const int64_t o = o0 + tid;
        int64_t N = 0;
        if (o < n) {
            const int64_t b = over_bin[o];
            N = R[bin_row[b + 1]] - R[bin_row[b]];
        }
        int64_t tch, ttu;
        const int64_t pc = block_exclusive_scan<int64_t, 1024>(ceil_div<int64_t>(N, OVER_CHUNK), scratch, &tch);
        const int64_t pt = block_exclusive_scan<int64_t, 1024>((N + 3) & ~int64_t(3), scratch, &ttu);
        if (o < n) {
            over_chunk_off[o] = cc + pc;
            over_tuple_off[o] = base + tc + pt;
        }
        cc += tch;
        tc += ttu;
    }
    if (tid == 0) {
        const bool ok = base + tc + 256 * cc <= tuple_cap && cc <= ochunk_cap;
        if (!ok) atomicOr(err, DEV_ERR_WORKSPACE);
        over_chunk_off[n] = cc;
        over_tuple_off[n] = base + tc;
        over_count[0] = ok ? n : 0;
        over_count[1] = ok ? cc : 0;
        over_count[2] = base + tc;
        fits = ok ? 1 : 0;
    }
    __syncthreads();
    if (!fits) return;
    for (int64_t o = tid; o < n; o += 1024)
        for (int64_t c = over_chunk_off[o]; c < over_chunk_off[o + 1]; ++c) over_chunk_bin[c] = (int32_t)o;
}

// Per A entry: its row's bin info, and the expand work items.  In product q
// the runs of its A entries tile [0, flop_q) in CSC order (entry j of column k
// owns [F_q[k] + j*lb, F_q[k] + (j+1)*lb), lb = nnz(B(k,:))); work item c of
// the product holds the entries whose run starts in [c*chunk, (c+1)*chunk).
__global__ void __launch_bounds__(T) k_bentry(int32_t count, const BatchDesc *__restrict__ desc,
                                              const int32_t *__restrict__ tiles_e, const int32_t *__restrict__ acol,
                                              const uint64_t *__restrict__ rowinfo, const int64_t *__restrict__ F,
                                              const BatchProd *__restrict__ prod, const uint32_t *err,
                                              uint64_t *ainfo, int2 *aspan, int32_t *chunk_e, int32_t *chunk_prod) {
    if (*err & DEV_ERR_BATCH_FATAL) return;
    const int64_t ntiles = tiles_e[count];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int q = find_prod(tiles_e, count, t);
        const BatchDesc &d = desc[q];
        const int64_t lo = (t - tiles_e[q]) * (int64_t)BATCH_TILE;
        const int64_t F0 = F[d.kstart];
        const int64_t cb = prod[q].chunk_base;
        const int64_t chunk = d.chunk;
        for (int j = threadIdx.x; j < BATCH_TILE; j += T) {
            const int64_t e = lo + j;
            if (e >= d.nnzA) continue;
            const int64_t eg = d.estart + e;
            ainfo[eg] = rowinfo[d.mstart + d.rowidxA[e]];
            const int32_t kk = acol[eg];
            const int64_t lb = (int64_t)d.rowptrB[kk + 1] - d.rowptrB[kk];
            aspan[eg] = make_int2(d.rowptrB[kk], (int32_t)lb);
            if (lb == 0) continue;
            const int64_t s = (F[d.kstart + kk] - F0) + (e - d.colptrA[kk]) * lb, r = s + lb;
            for (int64_t c = ceil_div<int64_t>(s, chunk); c * chunk < r; ++c) {
                chunk_e[cb + c] = (c * chunk == s) ? (int32_t)eg : (int32_t)(eg + 1);
                chunk_prod[cb + c] = q;
            }
        }
    }
}

// The batch's status word, mapped to pb_status, in stream order after the sort.
__global__ void k_bfinish(const uint32_t *err, int32_t *device_status) { *device_status = status_of_word(*err); }

unsigned grid_cap(int64_t n, int threads, int64_t cap) {
    int64_t g = ceil_div<int64_t>(n > 0 ? n : 1, threads);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((uint64_t(1) << b) < x) ++b;
    return b;
}

size_t tuple_bytes(pb_dtype d) { return d == PB_F64 ? 8 : 4; }

struct Klass {
    int32_t log2n, dclass;
};

Klass class_of(const pb_csc &A) {
    Klass c;
    c.log2n = ceil_log2((uint64_t)std::max<int32_t>(A.nrows, 2));
    const int64_t d = A.ncols > 0 ? (int64_t)std::llround((double)A.nnz / (double)A.ncols) : 0;
    int b = 0;
    while (b < 62 && (int64_t(1) << b) <= d) ++b;
    c.dclass = b;
    return c;
}

pb_batch_tune lookup(const pb_handle *h, Klass c) {
    for (const pb_batch_tune &t : h->tuning)
        if (t.log2n == c.log2n && t.dclass == c.dclass) return t;
    return pb_batch_tune{c.log2n, c.dclass, 4096, RMAX_LOG2, 4096, 0};
}

bool valid_tune(const pb_batch_tune &t) {
    return level_of(t.bin_capacity) >= 0 && t.rmax_log2 >= 1 && t.rmax_log2 <= RMAX_LOG2 &&
           t.expand_chunk >= MIN_CHUNK && t.expand_chunk % 32 == 0;
}

// Everything the host knows about a batch before launching.
struct BatchHost {
    int32_t count = 0;
    std::vector<int32_t> order;  // global position -> caller's index
    std::vector<BatchDesc> desc; // in global order
    std::vector<int32_t> tiles;  // 3 per product, global order
    int32_t tiles_total[3] = {0, 0, 0};
    int64_t M = 0, K = 0, E = 0;
    LevelRows lv{};
    int64_t level_rows[NLEVELS] = {0, 0, 0};
    bool any_over = false;  // some product may have rows above its capacity
    int over_shift = 0;     // dense tiles: the partition digit is column >> over_shift
};

pb_status prepare(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, const pb_csr_out *C, pb_dtype dtype,
                  BatchHost &bh) {
    if (count < 0 || count > MAX_COUNT) return host_fail(h, PB_ERR_INVALID_ARG, "count must be in [0, 2^20]");
    if (count > 0 && (!A || !B)) return host_fail(h, PB_ERR_INVALID_ARG, "A and B arrays must not be NULL");
    if (dtype != PB_F64 && dtype != PB_F32 && dtype != PB_F64_F32TUPLE)
        return host_fail(h, PB_ERR_UNSUPPORTED_DTYPE, "unknown dtype");
    bh.count = count;
    std::vector<pb_batch_tune> tune(count);
    std::vector<int> level(count);
    for (int32_t i = 0; i < count; ++i) {
        pb_status st = host_check_operands(h, &A[i], &B[i]);
        if (st != PB_OK) return host_fail(h, st, "product " + std::to_string(i) + ": " + h->last_error);
        if (C) {
            const pb_csr_out &c = C[i];
            if (c.nrows != A[i].nrows || c.ncols != B[i].ncols)
                return host_fail(h, PB_ERR_SHAPE, "product " + std::to_string(i) + ": C must be A.nrows x B.ncols");
            if ((c.rowptr64 == nullptr) == (c.rowptr32 == nullptr))
                return host_fail(h, PB_ERR_INVALID_ARG,
                                 "product " + std::to_string(i) + ": exactly one of C.rowptr64 / C.rowptr32");
            if (c.cap < 0 || (c.cap > 0 && (!c.colidx || !c.val)))
                return host_fail(h, PB_ERR_INVALID_ARG, "product " + std::to_string(i) + ": C arrays / cap");
        }
        tune[i] = lookup(h, class_of(A[i]));
        level[i] = level_of(tune[i].bin_capacity);
    }
    bh.order.resize(count);
    for (int32_t i = 0; i < count; ++i) bh.order[i] = i;
    std::stable_sort(bh.order.begin(), bh.order.end(), [&](int32_t a, int32_t b) { return level[a] < level[b]; });
    bh.desc.resize(count);
    bh.tiles.resize(3 * (size_t)count);
    int64_t M = 0, K = 0, E = 0, tm = 0, tk = 0, te = 0;
    int cur_level = 0;
    for (int32_t g = 0; g < count; ++g) {
        const int32_t i = bh.order[g];
        while (cur_level < level[i]) bh.lv.row[++cur_level] = (int32_t)M;
        BatchDesc &d = bh.desc[g];
        std::memset(&d, 0, sizeof(d));
        d.colptrA = A[i].colptr;
        d.rowidxA = A[i].rowidx;
        d.valA = A[i].val;
        d.rowptrB = B[i].rowptr;
        d.colidxB = B[i].colidx;
        d.valB = B[i].val;
        if (C) {
            d.rowptr64 = C[i].rowptr64;
            d.rowptr32 = C[i].rowptr32;
            d.colidxC = C[i].colidx;
            d.valC = C[i].val;
            d.nnz_dev = C[i].nnz_dev;
            d.capC = C[i].cap;
        }
        d.m = A[i].nrows;
        d.k = A[i].ncols;
        d.n = B[i].ncols;
        d.nnzA = (int32_t)A[i].nnz;
        d.mstart = (int32_t)M;
        d.kstart = (int32_t)K;
        d.estart = (int32_t)E;
        d.colbits = ceil_log2((uint64_t)std::max<int32_t>(d.n, 2));
        if (d.colbits > 31) return host_fail(h, PB_ERR_UNSUPPORTED, "B.ncols too large for a 32-bit key");
        d.rmax_log2 = std::min(tune[i].rmax_log2, 32 - d.colbits);
        d.capacity = tune[i].bin_capacity;
        d.chunk = tune[i].expand_chunk;
        d.level = level[i];
        d.over_ok = d.colbits <= 8 + OVER_DENSE_MAX_SHIFT ? 1 : 0;
        if (d.over_ok) {
            bh.any_over = true;
            bh.over_shift = std::max(bh.over_shift, d.colbits - 8);
        }
        bh.tiles[3 * (size_t)g + 0] = (int32_t)tm;
        bh.tiles[3 * (size_t)g + 1] = (int32_t)tk;
        bh.tiles[3 * (size_t)g + 2] = (int32_t)te;
        tm += ceil_div<int64_t>(d.m, BATCH_TILE);
        tk += ceil_div<int64_t>(d.k, BATCH_TILE);
        te += ceil_div<int64_t>(d.nnzA, BATCH_TILE);
        bh.level_rows[level[i]] += d.m;
        M += d.m;
        K += d.k;
        E += A[i].nnz;
        if (M >= (1ll << 31) - 2 || K >= (1ll << 31) - 2 || E >= (1ll << 31) - 2)
            return host_fail(h, PB_ERR_UNSUPPORTED, "batch rows, columns and nnz(A) must each total below 2^31");
    }
    while (cur_level < NLEVELS) bh.lv.row[++cur_level] = (int32_t)M;
    bh.M = M;
    bh.K = K;
    bh.E = E;
    bh.tiles_total[0] = (int32_t)tm;
    bh.tiles_total[1] = (int32_t)tk;
    bh.tiles_total[2] = (int32_t)te;
    return PB_OK;
}

// The symbolic kernels up to the per-product row maxima (shared by the query).
pb_status launch_front(pb_handle *h, const BatchHost &bh, const BatchWs &w, cudaStream_t s) {
    const int32_t count = bh.count;
    const int64_t cap = (int64_t)h->num_sms * 16;
    PB_CUDA_H(h, cudaMemsetAsync(w.bhdr, 0, sizeof(BatchHeader), s));
    PB_CUDA_H(h, cudaMemsetAsync(w.err, 0, 256, s));
    for (int32_t first = 0; first < count; first += DESC_PER_LAUNCH) {
        DescBlock blk;
        std::memset(&blk, 0, sizeof(blk));
        blk.first = first;
        blk.n = std::min(DESC_PER_LAUNCH, count - first);
        blk.count = count;
        for (int c = 0; c < 3; ++c) blk.tiles_total[c] = bh.tiles_total[c];
        for (int i = 0; i < blk.n; ++i) {
            blk.d[i] = bh.desc[first + i];
            for (int c = 0; c < 3; ++c) blk.tiles[i][c] = bh.tiles[3 * (size_t)(first + i) + c];
        }
        k_bdesc<<<1, DESC_PER_LAUNCH, 0, s>>>(blk, w.desc, w.prod, w.tiles_m, w.tiles_k, w.tiles_e);
        count_launches(1);
    }
    if (count == 0) return PB_OK;
    PB_CUDA_H(h, cudaGetLastError());
    // 1. Alg. 3: flop per column and per product; column of every A entry
    k_bflop<<<grid_cap(bh.tiles_total[1], 1, cap), T, 0, s>>>(count, w.desc, w.tiles_k, w.F, w.acol, w.long_cols,
                                                              w.n_long, w.prod);
    k_bacol_long<<<grid_cap(bh.K * 32, T, 4096), T, 0, s>>>(w.desc, w.long_cols, w.n_long, w.acol);
    // 2. per-row flop (Sec. III-B) and its prefix
    PB_CUDA_H(h, cudaMemsetAsync(w.R, 0, 8 * ((size_t)bh.M + 1), s));
    k_brow_flop<<<grid_cap(bh.tiles_total[2], 1, cap), T, 0, s>>>(count, w.desc, w.tiles_e, w.acol, w.R);
    count_launches(3);
    PB_CUDA_H(h, scan_i64(w.R, bh.M, w.scan_tmp, s));
    k_bmax<<<grid_cap(bh.tiles_total[0], 1, cap), T, 0, s>>>(count, w.desc, w.tiles_m, w.R, w.prod, w.err);
    count_launches(1);
    PB_CUDA_H(h, cudaGetLastError());
    return PB_OK;
}

pb_status launch_batch(pb_handle *h, const BatchHost &bh, const BatchWs &w, pb_dtype dtype, cudaStream_t s,
                       int32_t *device_status) {
    const int32_t count = bh.count;
    const int64_t cap = (int64_t)h->num_sms * 16;
    if (h->phase_on) PB_CUDA_H(h, cudaEventRecord(h->phase_ev[0], s));
    pb_status st = launch_front(h, bh, w, s);
    if (st != PB_OK) return st;
    if (count > 0) {
        // 3. F prefix (work-item boundaries), per-product work-item bases
        PB_CUDA_H(h, scan_i64(w.F, bh.K, w.scan_tmp, s));
        k_bprod<<<1, 1024, 0, s>>>(count, w.desc, w.prod, w.bhdr, w.err, w.chunk_cap, w.chunk_e, (int32_t)bh.E);
        // 4. bins (per product), their rows and products, row info
        k_bflags<<<grid_cap(bh.tiles_total[0], 1, cap), T, 0, s>>>(count, w.desc, w.tiles_m, w.R, w.prod, w.flags);
        count_launches(2);
        PB_CUDA_H(h, scan_i64(w.flags, bh.M, w.scan_tmp, s));
        k_bbin_rows<<<grid_cap(bh.tiles_total[0], 1, cap), T, 0, s>>>(
            count, w.desc, w.tiles_m, w.flags, w.R, (int32_t)bh.M, w.bin_row, w.bin_prod, w.prod, w.bhdr, bh.lv,
            w.over_scan, w.over_bin, w.n_over, w.n_over_cap, w.err);
        k_browinfo<<<grid_cap(bh.tiles_total[0], 1, cap), T, 0, s>>>(count, w.desc, w.tiles_m, w.flags, w.bin_row,
                                                                     w.rowinfo);
        k_bbin_off<<<grid_cap(bh.M, T, 4096), T, 0, s>>>(w.R, w.bin_row, (int32_t)bh.M, w.bhdr, w.tuple_cap,
                                                         w.bin_off, w.cursor, w.status, w.err);
        if (bh.any_over) {
            k_bover<<<1, 1024, 0, s>>>(w.R, w.bin_row, w.over_bin, w.n_over, w.n_over_cap, w.ochunk_cap,
                                       w.tuple_cap, w.bhdr, w.err, w.over_chunk_off, w.over_tuple_off,
                                       w.over_chunk_bin, w.over_count);
            count_launches(1);
        }
        // 5. per A entry: bin info and expand work items
        k_bentry<<<grid_cap(bh.tiles_total[2], 1, cap), T, 0, s>>>(count, w.desc, w.tiles_e, w.acol, w.rowinfo,
                                                                   w.F, w.prod, w.err, w.ainfo, w.aspan, w.chunk_e,
                                                                   w.chunk_prod);
        count_launches(4);
        PB_CUDA_H(h, cudaGetLastError());
        // numeric: expand (Alg. 2) for every product, then one sort launch per capacity level
        NumericArgs a{};
        a.ainfo = w.ainfo;
        a.acol = w.acol;
        a.aspan = w.aspan;
        a.bin_row = w.bin_row;
        a.bin_off = w.bin_off;
        a.R = w.R;
        a.chunk_e = w.chunk_e;
        a.nchunks = w.chunk_cap;  // bound: sizes the grid
        a.bin_lo = 0;
        a.bin_hi = INT64_MAX;
        a.tuple_base = 0;
        a.keys = w.keys;
        a.vals = w.vals;
        a.cursor = w.cursor;
        a.cursor_stride = 1;
        a.status = w.status;
        a.err = w.err;
        a.dtype = dtype;
        a.num_sms = h->num_sms;
        a.desc = w.desc;
        a.chunk_prod = w.chunk_prod;
        a.bin_prod = w.bin_prod;
        a.prod = w.prod;
        a.bhdr = w.bhdr;
        a.work = w.err + 32;  // the control block is zeroed at the start of the call
        a.over_scan = w.over_scan;
        a.over_u = w.over_u;
        a.over_p = w.over_p;
        a.over_passes = 1;
        a.over_dense = 1;
        OversizeArgs o{};
        o.R = w.R;
        o.bin_row = w.bin_row;
        o.bin_off = w.bin_off;
        o.over_bin = w.over_bin;
        o.over_chunk_off = w.over_chunk_off;
        o.over_tuple_off = w.over_tuple_off;
        o.over_chunk_bin = w.over_chunk_bin;
        o.n_over = w.n_over_cap;
        o.over_chunks = w.ochunk_cap;
        o.keys = w.keys;
        o.vals = w.vals;
        o.skeys = w.keys;  // the scratch follows the bins' tuples (k_bover)
        o.svals = w.vals;
        o.hist = nullptr;  // in the tuple buffer (dev_count[2])
        o.over_u = w.over_u;
        o.o_lo = 0;
        o.o_hi = w.n_over_cap;
        o.c_lo = 0;
        o.c_hi = w.ochunk_cap;
        o.dense = 1;
        o.dense_shift = bh.over_shift;
        o.wide = dtype == PB_F64_F32TUPLE ? 1 : 0;
        o.row_ticket = w.row_ticket;
        o.row_order = w.row_order;
        o.order_cnt = w.order_cnt;
        o.over_p = w.over_p;
        o.dev_count = w.over_count;
        o.desc = w.desc;
        o.bin_prod = w.bin_prod;
        if (h->phase_on) PB_CUDA_H(h, cudaEventRecord(h->phase_ev[1], s));
        PB_CUDA_H(h, launch_expand_batch(a, s));
        // rows above their capacity: one partition pass and dense tiles, before the sort publishes them
        if (bh.any_over) PB_CUDA_H(h, launch_oversize(o, 1, dtype, h->num_sms, s));
        if (h->phase_on) PB_CUDA_H(h, cudaEventRecord(h->phase_ev[2], s));
        for (int l = 0; l < NLEVELS; ++l) {
            if (bh.level_rows[l] == 0) continue;
            a.capacity = kLevelCap[l];
            a.level = l;
            a.ticket = w.tickets + l;
            a.bin_lo = 0;
            a.bin_hi = bh.level_rows[l];  // bound on the level's bins: sizes the grid
            PB_CUDA_H(h, launch_binsort_batch(a, s));
        }
        if (bh.any_over) PB_CUDA_H(h, launch_oversize_emit(o, dtype, h->num_sms, s));
        if (h->phase_on) PB_CUDA_H(h, cudaEventRecord(h->phase_ev[3], s));
    }
    k_bfinish<<<1, 1, 0, s>>>(w.err, device_status);
    count_launches(1);
    PB_CUDA_H(h, cudaGetLastError());
    return PB_OK;
}

}  // namespace

extern "C" {

pb_status pb_spgemm_batch_query(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, pb_dtype dtype,
                                pb_stream_t stream_, size_t *workspace_bytes, int64_t *flop, int64_t *max_row_flop) {
    if (!h) return PB_ERR_INVALID_ARG;
    h->last_error.clear();
    BatchHost bh;
    pb_status st = prepare(h, count, A, B, nullptr, dtype, bh);
    if (st != PB_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    BatchWs w{};
    const size_t fixed = carve_fixed(w, nullptr, count, bh.M, bh.K, bh.E);
    void *tmp = h->alloc(fixed, stream_, h->ctx);
    if (!tmp) return host_fail(h, PB_ERR_OOM, "batch query: temporary buffer");
    carve_fixed(w, static_cast<char *>(tmp), count, bh.M, bh.K, bh.E);
    std::vector<BatchProd> prod(count);
    st = launch_front(h, bh, w, s);
    cudaError_t e = cudaSuccess;
    if (st == PB_OK && count > 0)
        e = cudaMemcpyAsync(prod.data(), w.prod, sizeof(BatchProd) * (size_t)count, cudaMemcpyDeviceToHost, s);
    if (st == PB_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    h->free_fn(tmp, fixed, stream_, h->ctx);
    if (st != PB_OK) return st;
    if (e != cudaSuccess) return host_cuda_fail(h, e, "batch query");
    int64_t total = 0, over = 0;
    for (int32_t g = 0; g < count; ++g) {
        const int32_t i = bh.order[g];
        total += prod[g].flop;
        over += prod[g].over_bound;
        if (flop) flop[i] = prod[g].flop;
        if (max_row_flop) max_row_flop[i] = (int64_t)prod[g].max_row;
    }
    // the bins' tuples, then the scratch of the rows above capacity
    const int64_t tuples = ((total + 3) & ~int64_t(3)) + 4 * bh.M + 8 + over;
    if (workspace_bytes) *workspace_bytes = fixed + tail_bytes(tuples, count, tuple_bytes(dtype));
    return PB_OK;
}

pb_status pb_spgemm_batch(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, pb_csr_out *C,
                          pb_dtype dtype, void *workspace, size_t ws_bytes, pb_stream_t stream_,
                          int32_t *device_status) {
    if (!h) return PB_ERR_INVALID_ARG;
    h->last_error.clear();
    if (!device_status) return host_fail(h, PB_ERR_INVALID_ARG, "device_status must not be NULL");
    if (count > 0 && !C) return host_fail(h, PB_ERR_INVALID_ARG, "C array must not be NULL");
    if (count > 0 && (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)))
        return host_fail(h, PB_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
    BatchHost bh;
    pb_status st = prepare(h, count, A, B, C, dtype, bh);
    if (st != PB_OK) return st;
    BatchWs w{};
    char *base = static_cast<char *>(workspace);
    const size_t fixed = carve_fixed(w, nullptr, count, bh.M, bh.K, bh.E);
    if (count > 0 && ws_bytes < fixed + tail_bytes(4, count, tuple_bytes(dtype)))
        return host_fail(h, PB_ERR_WORKSPACE, "workspace smaller than pb_spgemm_batch_query reported");
    if (count > 0) {
        carve_fixed(w, base, count, bh.M, bh.K, bh.E);
        carve_tail(w, base, fixed, ws_bytes, count, tuple_bytes(dtype));
    } else {
        std::memset(&w, 0, sizeof(w));
        w.bhdr = nullptr;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    if (count == 0) {
        PB_CUDA_H(h, cudaMemsetAsync(device_status, 0, sizeof(int32_t), s));
        return PB_OK;
    }
    return launch_batch(h, bh, w, dtype, s, device_status);
}

pb_status pb_batch_get_tuning(const pb_handle *h, pb_batch_tune *out, int32_t cap, int32_t *n) {
    if (!h || !n || cap < 0 || (cap > 0 && !out)) return PB_ERR_INVALID_ARG;
    *n = (int32_t)h->tuning.size();
    for (int32_t i = 0; i < cap && i < *n; ++i) out[i] = h->tuning[i];
    return PB_OK;
}

pb_status pb_batch_set_tuning(pb_handle *h, const pb_batch_tune *entries, int32_t n) {
    if (!h || n < 0 || (n > 0 && !entries)) return PB_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i)
        if (!valid_tune(entries[i])) return host_fail(h, PB_ERR_INVALID_ARG, "invalid tuning entry " + std::to_string(i));
    h->tuning.assign(entries, entries + n);
    return PB_OK;
}

pb_status pb_batch_autotune(pb_handle *h, int32_t count, const pb_csc *A, const pb_csr *B, pb_csr_out *C,
                            pb_dtype dtype, void *workspace, size_t ws_bytes, pb_stream_t stream_, int32_t reps) {
    if (!h) return PB_ERR_INVALID_ARG;
    h->last_error.clear();
    if (reps < 1) reps = 1;
    if (count <= 0) return PB_OK;
    if (!A || !B || !C) return host_fail(h, PB_ERR_INVALID_ARG, "A, B and C arrays must not be NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    // products of each class
    std::vector<std::pair<Klass, std::vector<int32_t>>> classes;
    for (int32_t i = 0; i < count; ++i) {
        const Klass c = class_of(A[i]);
        auto it = std::find_if(classes.begin(), classes.end(), [&](const auto &x) {
            return x.first.log2n == c.log2n && x.first.dclass == c.dclass;
        });
        if (it == classes.end()) {
            classes.push_back({c, {}});
            it = classes.end() - 1;
        }
        it->second.push_back(i);
    }
    int32_t *dstatus = static_cast<int32_t *>(h->alloc(256, stream_, h->ctx));
    if (!dstatus) return host_fail(h, PB_ERR_OOM, "autotune: status word");
    cudaEvent_t ev[2] = {nullptr, nullptr};
    pb_status result = PB_OK;
    auto set_entry = [&](const pb_batch_tune &t) {
        for (pb_batch_tune &x : h->tuning)
            if (x.log2n == t.log2n && x.dclass == t.dclass) {
                x = t;
                return;
            }
        h->tuning.push_back(t);
    };
    // time one setting on a class's products; < 0 if it fails on the device
    auto time_it = [&](const std::vector<pb_csc> &a, const std::vector<pb_csr> &b, std::vector<pb_csr_out> &c,
                       double *ms) -> pb_status {
        const int32_t n = (int32_t)a.size();
        pb_status st = pb_spgemm_batch(h, n, a.data(), b.data(), c.data(), dtype, workspace, ws_bytes, stream_, dstatus);
        if (st != PB_OK) return st;
        int32_t dev = 0;
        PB_CUDA_H(h, cudaMemcpyAsync(&dev, dstatus, 4, cudaMemcpyDeviceToHost, s));
        PB_CUDA_H(h, cudaStreamSynchronize(s));
        if (dev != PB_OK) {
            *ms = -1.0;
            return PB_OK;
        }
        PB_CUDA_H(h, cudaEventRecord(ev[0], s));
        for (int r = 0; r < reps; ++r) {
            st = pb_spgemm_batch(h, n, a.data(), b.data(), c.data(), dtype, workspace, ws_bytes, stream_, dstatus);
            if (st != PB_OK) return st;
        }
        PB_CUDA_H(h, cudaEventRecord(ev[1], s));
        PB_CUDA_H(h, cudaEventSynchronize(ev[1]));
        float t = 0;
        PB_CUDA_H(h, cudaEventElapsedTime(&t, ev[0], ev[1]));
        *ms = t / reps;
        return PB_OK;
    };
    do {
        if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
            result = host_fail(h, PB_ERR_CUDA, "autotune: event creation failed");
            break;
        }
        for (auto &cls : classes) {
            std::vector<pb_csc> a;
            std::vector<pb_csr> b;
            std::vector<pb_csr_out> c;
            for (int32_t i : cls.second) {
                a.push_back(A[i]);
                b.push_back(B[i]);
                c.push_back(C[i]);
            }
            pb_batch_tune best{cls.first.log2n, cls.first.dclass, 4096, RMAX_LOG2, 4096, 0};
            double best_ms = -1;
            auto consider = [&](pb_batch_tune cand) -> pb_status {
                set_entry(cand);
                double ms = -1;
                pb_status st = time_it(a, b, c, &ms);
                if (st != PB_OK) return st;
                if (ms >= 0 && (best_ms < 0 || ms < best_ms)) {
                    best_ms = ms;
                    best = cand;
                }
                return PB_OK;
            };
            // capacity x work-item size, then the row limit of the best pair
            const int32_t chunks[3] = {1024, 4096, 16384};
            for (int l = 0; l < NLEVELS && result == PB_OK; ++l)
                for (int ci = 0; ci < 3 && result == PB_OK; ++ci)
                    result = consider({cls.first.log2n, cls.first.dclass, kLevelCap[l], RMAX_LOG2, chunks[ci], 0});
            const pb_batch_tune pair = best;
            for (int r : {8, 10})
                if (result == PB_OK) result = consider({pair.log2n, pair.dclass, pair.bin_capacity, r, pair.expand_chunk, 0});
            if (result != PB_OK) break;
            set_entry(best);
        }
        if (result != PB_OK) break;
        // leave C holding the products under the chosen settings
        result = pb_spgemm_batch(h, count, A, B, C, dtype, workspace, ws_bytes, stream_, dstatus);
        if (result == PB_OK && cudaStreamSynchronize(s) != cudaSuccess)
            result = host_fail(h, PB_ERR_CUDA, "autotune: final run");
    } while (false);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    (void)cudaStreamSynchronize(s);
    h->free_fn(dstatus, 256, stream_, h->ctx);
    return result;
}

}  // extern "C"
