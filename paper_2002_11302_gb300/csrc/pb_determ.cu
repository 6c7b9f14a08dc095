// Deterministic mode: fixed tuple positions for the expand phase.
//
// Alg. 2 appends each outer-product run to its bin; with atomic cursors the
// order of runs inside a bin, hence the order in which duplicates of one C entry
// are summed, varies from run to run.  Here each A entry's run gets a position
// fixed in the plan: inside every bin the runs are laid out in CSC order of A
// (ascending k).  Equal keys are merged in position order (the sort breaks key
// ties by position), so every C(i,j) is summed as sum over ascending k of
// A(i,k) B(k,j), the same order on every run.
//
// Positions: a stable LSD radix sort (8-bit digits, global memory) of the A
// entries by bin, then an exclusive scan of the run lengths nnz(B(k,:)) in that
// order.  The tuples of bins before bin b sum to R[first row of b], so entry e
// of bin b starts at bin_off[b] + scan[e] - R[first row of b].
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int DT = 512;             // threads per CTA
constexpr int DCH = 4096;           // entries per chunk
constexpr int DE = DCH / DT;        // entries per thread
constexpr int DNW = DT / 32;
constexpr int DWS = DCH / DNW;      // entries per warp in a chunk

__global__ void k_det_init(int64_t E, const uint64_t *ainfo, uint32_t *key, int32_t *val) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        key[e] = (uint32_t)(ainfo[e] >> 32);
        val[e] = (int32_t)e;
    }
}

// hist[d * nchunks + c] = entries of chunk c whose digit is d (digit-major, so
// its exclusive scan is each (digit, chunk) group's first destination).
__global__ void __launch_bounds__(DT) k_det_hist(int64_t E, int64_t nchunks, const uint32_t *key, int shift,
                                                 int64_t *hist) {
    __shared__ uint32_t h[256];
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        for (int i = threadIdx.x; i < 256; i += DT) h[i] = 0;
        __syncthreads();
        const int64_t lo = c * DCH, hi = (lo + DCH < E) ? lo + DCH : E;
        for (int64_t q = lo + threadIdx.x; q < hi; q += DT) atomicAdd(&h[(key[q] >> shift) & 255u], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += DT) hist[(int64_t)i * nchunks + c] = h[i];
        __syncthreads();
    }
}

// Stable scatter of one pass: inside a chunk, entries keep their order within
// each digit (warp multisplit with ballots, per-(digit, warp) counters).
__global__ void __launch_bounds__(DT) k_det_scatter(int64_t E, int64_t nchunks, const uint32_t *ks, const int32_t *vs,
                                                    int shift, const int64_t *off, uint32_t *kd, int32_t *vd) {
    __shared__ uint32_t wc[256 * DNW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        for (int i = threadIdx.x; i < 256 * DNW; i += DT) wc[i] = 0;
        __syncthreads();
        const int64_t lo = c * DCH;
        const int64_t len = (lo + DCH < E) ? DCH : E - lo;
        uint32_t kk[DE], lr[DE];
        int32_t vv[DE];
#pragma unroll
        for (int j = 0; j < DE; ++j) {
            const int64_t q = warp * DWS + j * 32 + lane;
            const bool valid = q < len;
            const uint32_t k = valid ? ks[lo + q] : 0u;
            vv[j] = valid ? vs[lo + q] : 0;
            const uint32_t dg = (k >> shift) & 255u;
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
                old = wc[dg * DNW + warp];
                wc[dg * DNW + warp] = old + __popc(peers);
            }
            old = __shfl_sync(FULL, old, leader);
            __syncwarp();
            lr[j] = old + __popc(peers & lanemask_lt());
            kk[j] = k;
        }
        __syncthreads();
        if (threadIdx.x < 256) {  // per digit: exclusive prefix over warps
            uint32_t run = 0;
            for (int w = 0; w < DNW; ++w) {
                const uint32_t v = wc[threadIdx.x * DNW + w];
                wc[threadIdx.x * DNW + w] = run;
                run += v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < DE; ++j) {
            const int64_t q = warp * DWS + j * 32 + lane;
            if (q < len) {
                const uint32_t dg = (kk[j] >> shift) & 255u;
                const int64_t pos = off[(int64_t)dg * nchunks + c] + wc[dg * DNW + warp] + lr[j];
                kd[pos] = kk[j];
                vd[pos] = vv[j];
            }
        }
        __syncthreads();
    }
}

// Run lengths in bin order.
__global__ void k_det_lb(int64_t E, const int32_t *sorted_e, const int32_t *acol, const int32_t *rowptrB,
                         int64_t *lbs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = acol[sorted_e[i]];
        lbs[i] = (int64_t)rowptrB[k + 1] - rowptrB[k];
    }
}

__global__ void k_det_pos(int64_t E, const int32_t *sorted_e, const uint32_t *sorted_bin, const int64_t *S,
                          const int64_t *bin_off, const int32_t *bin_row, const int64_t *R, int64_t *apos) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = sorted_bin[i];
        apos[sorted_e[i]] = bin_off[b] + S[i] - R[bin_row[b]];
    }
}

unsigned grid_cap(int64_t n, int threads, int64_t cap) {
    int64_t g = ceil_div<int64_t>(n > 0 ? n : 1, threads);
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace

int64_t det_scratch_bytes(int64_t E) {
    const int64_t nchunks = ceil_div<int64_t>(E > 0 ? E : 1, DCH);
    const int64_t scan_n = (E > 256 * nchunks ? E : 256 * nchunks) + 1;
    auto a = [](int64_t b) { return (b + 255) & ~int64_t(255); };
    return 4 * a(4 * E) + a(8 * (256 * nchunks + 1)) + a(8 * (E + 1)) + a(8 * scan_tmp_elems(scan_n));
}

cudaError_t launch_det_positions(const DetArgs &d, void *scratch, int num_sms, cudaStream_t s) {
    const int64_t E = d.E;
    if (E <= 0) return cudaSuccess;
    const int64_t nchunks = ceil_div<int64_t>(E, DCH);
    const int64_t scan_n = (E > 256 * nchunks ? E : 256 * nchunks) + 1;
    auto a = [](int64_t b) { return (b + 255) & ~int64_t(255); };
    char *w = static_cast<char *>(scratch);
    uint32_t *key[2];
    int32_t *val[2];
    key[0] = reinterpret_cast<uint32_t *>(w);
    w += a(4 * E);
    key[1] = reinterpret_cast<uint32_t *>(w);
    w += a(4 * E);
    val[0] = reinterpret_cast<int32_t *>(w);
    w += a(4 * E);
    val[1] = reinterpret_cast<int32_t *>(w);
    w += a(4 * E);
    int64_t *hist = reinterpret_cast<int64_t *>(w);
    w += a(8 * (256 * nchunks + 1));
    int64_t *lbs = reinterpret_cast<int64_t *>(w);
    w += a(8 * (E + 1));
    int64_t *tmp = reinterpret_cast<int64_t *>(w);
    (void)scan_n;
    const unsigned g = grid_cap(E, 256, 4096), gc = grid_cap(nchunks, 1, (int64_t)num_sms * 4);
    k_det_init<<<g, 256, 0, s>>>(E, d.ainfo, key[0], val[0]);
    int bits = 0;
    while ((int64_t(1) << bits) < d.nbins) ++bits;
    const int passes = (bits + 7) / 8;
    cudaError_t e;
    for (int pass = 0; pass < passes; ++pass) {
        const int src = pass & 1, dst = src ^ 1;
        k_det_hist<<<gc, DT, 0, s>>>(E, nchunks, key[src], 8 * pass, hist);
        if ((e = scan_i64(hist, 256 * nchunks, tmp, s)) != cudaSuccess) return e;
        k_det_scatter<<<gc, DT, 0, s>>>(E, nchunks, key[src], val[src], 8 * pass, hist, key[dst], val[dst]);
        count_launches(2);
    }
    const int fin = passes & 1;
    k_det_lb<<<g, 256, 0, s>>>(E, val[fin], d.acol, d.rowptrB, lbs);
    if ((e = scan_i64(lbs, E, tmp, s)) != cudaSuccess) return e;
    k_det_pos<<<g, 256, 0, s>>>(E, val[fin], key[fin], lbs, d.bin_off, d.bin_row, d.R, d.apos);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace pb
