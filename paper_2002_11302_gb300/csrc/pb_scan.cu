// Device-wide exclusive prefix sum of int64 arrays (reduce-then-scan).
//
// Used by the symbolic phase for the per-k flop prefix (Alg. 3), the per-row
// flop prefix (Sec. III-B), the bin-start flags and the bin offsets.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int64_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Per-tile sums.
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const int64_t *x, int64_t n, int64_t *sums) {
    __shared__ int64_t scratch[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += x[i];
    }
    int64_t total = block_reduce_sum<int64_t, SCAN_THREADS>(s, scratch);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of each tile, offset by offs[tile]; the last tile also
// writes x[n] = offs[ntiles].  Items are blocked per thread for the scan.
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(int64_t *x, int64_t n, const int64_t *offs,
                                                            int64_t ntiles) {
    __shared__ int64_t scratch[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + j;
        v[j] = (i < n) ? x[i] : 0;
        s += v[j];
    }
    int64_t total;
    int64_t pre = block_exclusive_scan<int64_t, SCAN_THREADS>(s, scratch, &total);
    int64_t run = pre + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + j;
        if (i < n) x[i] = run;
        run += v[j];
    }
    if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) x[n] = (offs ? offs[blockIdx.x] : 0) + total;
}

__global__ void k_set_zero(int64_t *x) { x[0] = 0; }

}  // namespace

int64_t scan_tmp_elems(int64_t n) {
    int64_t t = 0;
    while (n > SCAN_TILE) {
        int64_t nt = ceil_div<int64_t>(n, SCAN_TILE);
        t += nt + 1;
        n = nt;
    }
    return t + 1;
}

cudaError_t scan_i64(int64_t *x, int64_t n, int64_t *tmp, cudaStream_t s) {
    if (n <= 0) {
        k_set_zero<<<1, 1, 0, s>>>(x);
        count_launches(1);
        return cudaGetLastError();
    }
    int64_t ntiles = ceil_div<int64_t>(n, SCAN_TILE);
    if (ntiles == 1) {
        k_tile_scan<<<1, SCAN_THREADS, 0, s>>>(x, n, nullptr, 1);
        count_launches(1);
        return cudaGetLastError();
    }
    if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
    k_tile_sums<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(x, n, tmp);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_i64(tmp, ntiles, tmp + ntiles + 1, s);
    if (e != cudaSuccess) return e;
    k_tile_scan<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(x, n, tmp, ntiles);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pb

// ---------------------------------------------------------------------------
// Operand validation (pb_validate_operands): reads each array only within the
// sizes the caller declared and records what is wrong in a bit mask.
// ---------------------------------------------------------------------------
namespace pb {
namespace {

__global__ void k_validate_ptr(const int32_t *ptr, int64_t n, int64_t nnz, uint32_t bit, uint32_t *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ptr[i];
        bool ok = v >= 0 && v <= nnz;
        if (i == 0) ok = ok && v == 0;
        if (i == n) ok = ok && v == nnz;
        if (i > 0) ok = ok && ptr[i - 1] <= v;
        if (!ok) atomicOr(bad, bit);
    }
}

__global__ void k_validate_idx(const int32_t *idx, int64_t nnz, int32_t bound, uint32_t bit, uint32_t *bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = idx[e];
        if (v < 0 || v >= bound) atomicOr(bad, bit);
    }
}

unsigned vgrid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_validate(const pb_csc &A, const pb_csr &B, uint32_t *bad, cudaStream_t s) {
    k_validate_ptr<<<vgrid(A.ncols + 1), 256, 0, s>>>(A.colptr, A.ncols, A.nnz, 1u, bad);
    k_validate_ptr<<<vgrid(B.nrows + 1), 256, 0, s>>>(B.rowptr, B.nrows, B.nnz, 2u, bad);
    count_launches(2);
    if (A.nnz > 0) {
        k_validate_idx<<<vgrid(A.nnz), 256, 0, s>>>(A.rowidx, A.nnz, A.nrows, 4u, bad);
        count_launches(1);
    }
    if (B.nnz > 0) {
        k_validate_idx<<<vgrid(B.nnz), 256, 0, s>>>(B.colidx, B.nnz, B.ncols, 8u, bad);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace pb
