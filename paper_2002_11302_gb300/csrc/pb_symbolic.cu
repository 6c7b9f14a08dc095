// Symbolic phase (Alg. 3, Sec. III-B): flop counts and row-range bins.
//
//  1. f_k = nnz(A(:,k)) * nnz(B(k,:)) and its prefix F (Alg. 3).
//  2. Per-row flop r_i = sum over A(i,k) != 0 of nnz(B(k,:)) (the per-row form
//     of Alg. 3 in Sec. III-B) and its prefix R.
//  3. Rows are cut into bins of consecutive rows (the row ranges of Fig. 4 and
//     the "variable ranges of rows" of Sec. III-D).  A bin starts at row i when
//       i is a multiple of 2^rmax_log2 (keeps the in-bin row offset small),
//       R[i] and R[i-1] fall in different windows of width T, or
//       row i or row i-1 is heavy (r > heavy threshold H).
//     Light bins therefore hold fewer than T + max_light_row tuples; T is
//     chosen as capacity - max_light_row so they fit the on-chip sort.  A
//     heavy row is a bin of its own.
//  4. Bin offsets: counts padded to a multiple of 4 tuples (16-byte aligned
//     key segments for the bulk copies of the sort phase) and prefix-summed.
#include "pb_common.cuh"

namespace pb {

namespace {

// Tiles of FT columns, one column per thread: f_k = nnz(A(:,k)) * nnz(B(k,:))
// (Alg. 3).  Then the tile's A entries, which are contiguous in CSC, one per
// thread (coalesced): the column of each entry (binary search over the
// tile's column pointers in shared memory) and the per-row flop (Sec. III-B):
// every A(i,k) adds nnz(B(k,:)) to row i.  Columns with more than LONG_COL
// entries are listed for a warp-per-column pass instead.
constexpr int FT = 256;
constexpr int LONG_COL = 8192;

__device__ inline void add_row_flop(int64_t *R, int32_t row, int64_t lb) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&R[row]), (unsigned long long)lb);
}

__global__ void __launch_bounds__(FT) k_flop_per_k(int32_t k, const int32_t *colptrA, const int32_t *rowidxA,
                                                   const int32_t *rowptrB, int64_t *F, int64_t *R, int32_t *acol,
                                                   int32_t *long_cols, uint32_t *n_long) {
    __shared__ int32_t cp[FT + 1];
    __shared__ int32_t lbs[FT];  // nnz(B(k,:)) of the tile's columns; -1 for a listed long column
    const int tid = threadIdx.x;
    const int64_t ntiles = ceil_div<int64_t>(k, FT);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t k0 = t * FT;
        const int n = (int)(k - k0 < FT ? k - k0 : FT);
        if (tid <= n) cp[tid] = colptrA[k0 + tid];
        if (tid < n) {
            const int64_t col = k0 + tid;
            const int32_t na = colptrA[col + 1] - colptrA[col];
            const int32_t lb = rowptrB[col + 1] - rowptrB[col];
            F[col] = (int64_t)na * lb;
            if (na > LONG_COL) {
                long_cols[atomicAdd(n_long, 1u)] = (int32_t)col;
                lbs[tid] = -1;
            } else {
                lbs[tid] = lb;
            }
        }
        if (tid == 0 && n == FT) cp[FT] = colptrA[k0 + FT];
        __syncthreads();
        const int32_t e1 = cp[n];
        for (int32_t e = cp[0] + tid; e < e1; e += FT) {
            int lo = 0, hi = n;  // cp[lo] <= e < cp[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (cp[mid] <= e)
                    lo = mid;
                else
                    hi = mid;
            }
            const int32_t lb = lbs[lo];
            if (lb < 0) continue;  // a long column: its warp does it
            acol[e] = (int32_t)(k0 + lo);
            if (lb) add_row_flop(R, rowidxA[e], lb);
        }
        __syncthreads();
    }
}

// One warp per listed long column: the same for each of its entries.
__global__ void k_acol_long(const int32_t *colptrA, const int32_t *rowidxA, const int32_t *rowptrB,
                            const int32_t *long_cols, const uint32_t *n_long, int64_t *R, int32_t *acol) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = *n_long;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int32_t col = long_cols[i];
        const int64_t lb = (int64_t)rowptrB[col + 1] - rowptrB[col];
        for (int32_t e = colptrA[col] + lane; e < colptrA[col + 1]; e += 32) {
            acol[e] = col;
            if (lb) add_row_flop(R, rowidxA[e], lb);
        }
    }
}

__global__ void k_max_light(int32_t m, const int64_t *R, int64_t heavy, PlanHeader *hdr) {
    __shared__ unsigned long long wmax[32];
    unsigned long long best = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = R[i + 1] - R[i];
        if (r <= heavy && (unsigned long long)r > best) best = (unsigned long long)r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_down_sync(FULL, best, o);
        best = t > best ? t : best;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = wmax[w] > best ? wmax[w] : best;
        if (best) atomicMax(&hdr->max_light_row, best);
    }
}

__device__ inline bool is_heavy(const int64_t *R, int64_t i, int64_t heavy) { return R[i + 1] - R[i] > heavy; }

__global__ void k_bin_flags(int32_t m, const int64_t *R, int64_t capacity, int64_t heavy, int32_t rmax_log2,
                            const PlanHeader *hdr, int64_t *flags) {
    const int64_t T = capacity - (int64_t)hdr->max_light_row;  // >= capacity - heavy > 0
    const int64_t rmask = (1ll << rmax_log2) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        bool start = (i == 0) || ((i & rmask) == 0);
        if (!start) {
            start = (R[i] / T) != (R[i - 1] / T) || is_heavy(R, i, heavy) || is_heavy(R, i - 1, heavy);
        }
        flags[i] = start ? 1 : 0;
    }
}

// flags now holds the exclusive scan of the start flags; flags[m] = nbins.
__global__ void k_bin_rows(int32_t m, const int64_t *scanned, int32_t *bin_row, PlanHeader *hdr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t next = (i + 1 < m) ? scanned[i + 1] : scanned[m];
        if (next != scanned[i]) bin_row[scanned[i]] = (int32_t)i;  // row i starts bin scanned[i]
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bin_row[scanned[m]] = m;
        hdr->nbins = scanned[m];
    }
}

__global__ void k_rowinfo(int32_t m, const int64_t *scanned, const int32_t *bin_row, int32_t colbits,
                          uint64_t *rowinfo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t next = (i + 1 < m) ? scanned[i + 1] : scanned[m];
        const int64_t bin = (next != scanned[i]) ? scanned[i] : scanned[i] - 1;
        const uint32_t local = (uint32_t)(i - bin_row[bin]);
        rowinfo[i] = ((uint64_t)bin << 32) | (uint64_t)(local << colbits);
    }
}

__global__ void k_bin_sizes(const int64_t *R, const int32_t *bin_row, int64_t capacity, PlanHeader *hdr,
                            int64_t *bin_off) {
    const int64_t nbins = hdr->nbins;
    unsigned long long mx = 0;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cnt = R[bin_row[b + 1]] - R[bin_row[b]];
        bin_off[b] = (cnt + 3) & ~int64_t(3);
        if ((unsigned long long)cnt > mx) mx = cnt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_down_sync(FULL, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(&hdr->max_bin_count, mx);
    }
}

__device__ inline int64_t bin_count(const int64_t *R, const int32_t *bin_row, int64_t b) {
    return R[bin_row[b + 1]] - R[bin_row[b]];
}

__global__ void k_over_flags(const int64_t *R, const int32_t *bin_row, int64_t capacity, const PlanHeader *hdr,
                             int64_t *over_scan) {
    const int64_t nbins = hdr->nbins;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x)
        over_scan[b] = bin_count(R, bin_row, b) > capacity ? 1 : 0;
}

// over_scan is now the exclusive scan of the oversize flags.
__global__ void k_over_list(const int64_t *R, const int32_t *bin_row, int64_t capacity, const PlanHeader *hdr,
                            const int64_t *over_scan, int64_t *over_bin, int64_t *over_chunk_off,
                            int64_t *over_tuple_off) {
    const int64_t nbins = hdr->nbins;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = bin_count(R, bin_row, b);
        if (n <= capacity) continue;
        const int64_t o = over_scan[b];
        over_bin[o] = b;
        over_chunk_off[o] = (n + OVER_CHUNK - 1) / OVER_CHUNK;
        over_tuple_off[o] = (n + 3) & ~int64_t(3);
    }
}


__global__ void k_finish_header(const int64_t *F, int32_t k, int32_t m, const int64_t *R, const int64_t *bin_off,
                                const int64_t *over_scan, const int64_t *over_chunk_off,
                                const int64_t *over_tuple_off, PlanHeader *hdr) {
    hdr->flop = F[k];
    hdr->tuples_padded = bin_off[hdr->nbins];
    if (R[m] != F[k]) hdr->max_bin_count = ~0ull;  // per-row counts disagree with Alg. 3: reject
    if (over_scan) {
        hdr->n_oversize = over_scan[m];
        hdr->over_chunks = over_chunk_off[m];
        hdr->over_tuples = over_tuple_off[m];
    }
}

__global__ void k_over_chunk_map(const int64_t *over_chunk_off, int64_t n_over, int32_t *over_chunk_bin) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_over; o += (int64_t)gridDim.x * blockDim.x)
        for (int64_t c = over_chunk_off[o]; c < over_chunk_off[o + 1]; ++c) over_chunk_bin[c] = (int32_t)o;
}

// Per A entry, once the bins are known:
//   ainfo[e] = rowinfo[rowidxA[e]] (bin and key high part of the entry's row);
//   expand work items at A-entry granularity.  The runs of tuples of the A
//   entries tile [0, flop) in CSC order: entry j of column k owns
//   [F[k] + j*lb, F[k] + (j+1)*lb) with lb = nnz(B(k,:)).  Work item c holds the
//   entries whose run starts in [c*chunk, (c+1)*chunk): chunk_e[c] is the first.
__device__ inline void entry_info(int64_t e, int64_t s, int32_t b0, int64_t lb, int64_t chunk, const int32_t *rowidxA,
                                  const uint64_t *rowinfo, uint64_t *ainfo, int2 *aspan, int32_t *chunk_e) {
    ainfo[e] = rowinfo[rowidxA[e]];
    aspan[e] = make_int2(b0, (int32_t)lb);
    if (lb == 0) return;
    const int64_t r = s + lb;
    for (int64_t c = ceil_div<int64_t>(s, chunk); c * chunk < r; ++c)
        chunk_e[c] = (c * chunk == s) ? (int32_t)e : (int32_t)(e + 1);
}

// One thread per A entry (coalesced), its column from the flop pass: the
// entry's run starts at F[k] + (its position in the column) * lb.
__global__ void k_entry_pass(int64_t nnzA, const int32_t *acol, const int32_t *colptrA, const int32_t *rowidxA,
                             const int32_t *rowptrB, const uint64_t *rowinfo, const int64_t *F, int64_t chunk,
                             uint64_t *ainfo, int2 *aspan, int32_t *chunk_e) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzA; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t col = acol[e];
        const int32_t b0 = rowptrB[col];
        const int64_t lb = (int64_t)rowptrB[col + 1] - b0;
        entry_info(e, F[col] + (e - colptrA[col]) * lb, b0, lb, chunk, rowidxA, rowinfo, ainfo, aspan, chunk_e);
    }
}

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }

// Grid of a grid-stride kernel: enough blocks to fill the GPU, not one per item
// (tiny blocks cost more to launch and retire than their work).
unsigned grid_for(int64_t n, int threads) {
    int64_t g = ceil_div<int64_t>(n > 0 ? n : 1, threads);
    if (g > 4096) g = 4096;
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_symbolic(const SymbolicArgs &a, int64_t *scan_tmp, cudaStream_t s) {
    cudaError_t e;
    const int T = 256;
    // 1-2. per-k flop (Alg. 3), column of every A entry, per-row flop (Sec. III-B); prefixes
    if ((e = cudaMemsetAsync(a.n_long, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.R, 0, sizeof(int64_t) * ((size_t)a.m + 1), s)) != cudaSuccess) return e;
    k_flop_per_k<<<grid_for(a.k, FT), FT, 0, s>>>(a.k, a.colptrA, a.rowidxA, a.rowptrB, a.F, a.R, a.acol,
                                                 a.long_cols, a.n_long);
    k_acol_long<<<grid_for((int64_t)a.k * 32, T), T, 0, s>>>(a.colptrA, a.rowidxA, a.rowptrB, a.long_cols, a.n_long,
                                                            a.R, a.acol);
    if ((e = scan_i64(a.F, a.k, scan_tmp, s)) != cudaSuccess) return e;
    if ((e = scan_i64(a.R, a.m, scan_tmp, s)) != cudaSuccess) return e;
    // 3. bins
    k_max_light<<<grid_for(a.m, T), T, 0, s>>>(a.m, a.R, a.heavy, a.hdr);
    k_bin_flags<<<grid_for(a.m, T), T, 0, s>>>(a.m, a.R, a.capacity, a.heavy, a.rmax_log2, a.hdr, a.flags);
    if ((e = scan_i64(a.flags, a.m, scan_tmp, s)) != cudaSuccess) return e;
    k_bin_rows<<<grid_for(a.m, T), T, 0, s>>>(a.m, a.flags, a.bin_row, a.hdr);
    k_rowinfo<<<grid_for(a.m, T), T, 0, s>>>(a.m, a.flags, a.bin_row, a.colbits, a.rowinfo);
    // 4. bin sizes and offsets.  The bin count lives on the device, so the
    //    offsets are scanned over the m-entry upper bound: entries past nbins
    //    stay zero and bin_off[nbins] receives the total.
    if ((e = cudaMemsetAsync(a.bin_off, 0, sizeof(int64_t) * ((size_t)a.m + 2), s)) != cudaSuccess) return e;
    k_bin_sizes<<<grid_for(a.m, T), T, 0, s>>>(a.R, a.bin_row, a.capacity, a.hdr, a.bin_off);
    if ((e = scan_i64(a.bin_off, a.m, scan_tmp, s)) != cudaSuccess) return e;
    k_finish_header<<<1, 1, 0, s>>>(a.F, a.k, a.m, a.R, a.bin_off, nullptr, nullptr, nullptr, a.hdr);
    count_launches(8);  // the non-scan kernels above
    return cudaGetLastError();
}

// Oversize bins (single rows above the on-chip capacity): their list, work
// items and scratch offsets.  Only needed when the header's largest bin count
// exceeds the capacity.
cudaError_t launch_symbolic_oversize(const SymbolicArgs &a, int64_t *scan_tmp, cudaStream_t s) {
    cudaError_t e;
    const int T = 256;
    const size_t mb = sizeof(int64_t) * ((size_t)a.m + 1);
    if ((e = cudaMemsetAsync(a.over_scan, 0, mb, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.over_chunk_off, 0, mb, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.over_tuple_off, 0, mb, s)) != cudaSuccess) return e;
    k_over_flags<<<grid_for(a.m, T), T, 0, s>>>(a.R, a.bin_row, a.capacity, a.hdr, a.over_scan);
    if ((e = scan_i64(a.over_scan, a.m, scan_tmp, s)) != cudaSuccess) return e;
    k_over_list<<<grid_for(a.m, T), T, 0, s>>>(a.R, a.bin_row, a.capacity, a.hdr, a.over_scan, a.over_bin,
                                                a.over_chunk_off, a.over_tuple_off);
    if ((e = scan_i64(a.over_chunk_off, a.m, scan_tmp, s)) != cudaSuccess) return e;
    if ((e = scan_i64(a.over_tuple_off, a.m, scan_tmp, s)) != cudaSuccess) return e;
    k_finish_header<<<1, 1, 0, s>>>(a.F, a.k, a.m, a.R, a.bin_off, a.over_scan, a.over_chunk_off,
                                    a.over_tuple_off, a.hdr);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_over_chunk_map(const int64_t *over_chunk_off, int64_t n_over, int32_t *over_chunk_bin,
                                  cudaStream_t s) {
    if (n_over <= 0) return cudaSuccess;
    k_over_chunk_map<<<grid_for(n_over, 256), 256, 0, s>>>(over_chunk_off, n_over, over_chunk_bin);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_chunk_table(const SymbolicArgs &a, int64_t nchunks, int64_t chunk, int32_t *chunk_e,
                               cudaStream_t s) {
    // chunk_e[nchunks] = nnzA closes the last work item
    k_set_i32<<<1, 1, 0, s>>>(chunk_e + nchunks, (int32_t)a.nnzA);
    count_launches(1);
    if (a.nnzA > 0) {
        k_entry_pass<<<grid_for(a.nnzA, 256), 256, 0, s>>>(a.nnzA, a.acol, a.colptrA, a.rowidxA, a.rowptrB,
                                                           a.rowinfo, a.F, chunk, a.ainfo, a.aspan, chunk_e);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace pb
