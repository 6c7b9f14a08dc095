// Oversize bins: single heavy rows whose tuples exceed the on-chip sort capacity.
//
// The paper keeps every bin sortable in cache by using more bins or variable
// row ranges (Sec. III-D); a single row cannot be split by rows, so its tuples
// (all with in-bin row 0, key = column) are sorted here by a segmented, stable
// LSD radix sort in global memory, 8 bits per pass:
//   histogram  per chunk of CHUNK tuples, counts of each digit value;
//   offsets    per oversize bin, for every (digit, chunk) the destination of
//              the chunk's first tuple with that digit (digit-major order);
//   scatter    each chunk ranks its tuples stably (warp multisplit over the
//              digit with ballots, per-warp counters) and writes them out.
// Passes alternate between the bin's region of the tuple buffer and a scratch
// region.  Afterwards a head count gives the number of merged entries of each
// oversize bin, so the look-back chain of the sort phase never waits for the
// merge itself; the sort kernel then streams the sorted run into C.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int OT = 512;             // threads per CTA
constexpr int OE = OVER_CHUNK / OT;  // tuples per thread in a chunk
constexpr int ONW = OT / 32;
constexpr int OWS = OVER_CHUNK / ONW;  // tuples per warp in a chunk

struct ChunkRef {
    int64_t o, bin, start, len;
};

__device__ inline ChunkRef chunk_ref(const OversizeArgs &a, int64_t c) {
    ChunkRef r;
    r.o = a.over_chunk_bin[c];
    r.bin = a.over_bin[r.o];
    const int64_t N = a.R[a.bin_row[r.bin + 1]] - a.R[a.bin_row[r.bin]];
    r.start = (c - a.over_chunk_off[r.o]) * OVER_CHUNK;
    r.len = (N - r.start < OVER_CHUNK) ? N - r.start : OVER_CHUNK;
    return r;
}

template <class TV>
__device__ inline void pass_buffers(const OversizeArgs &a, int pass, const ChunkRef &r, const uint32_t *&sk,
                                    const TV *&sv, uint32_t *&dk, TV *&dv) {
    uint32_t *mk = a.keys + (a.bin_off[r.bin] - a.tuple_base);
    TV *mv = static_cast<TV *>(a.vals) + (a.bin_off[r.bin] - a.tuple_base);
    uint32_t *xk = a.skeys + (a.over_tuple_off[r.o] - a.over_base);
    TV *xv = static_cast<TV *>(a.svals) + (a.over_tuple_off[r.o] - a.over_base);
    if ((pass & 1) == 0) {
        sk = mk; sv = mv; dk = xk; dv = xv;
    } else {
        sk = xk; sv = xv; dk = mk; dv = mv;
    }
}

template <class TV>
__global__ void __launch_bounds__(OT) k_over_hist(const OversizeArgs a, int pass) {
    __shared__ uint32_t h[256];
    const int shift = 8 * pass;
    for (int64_t c = a.c_lo + blockIdx.x; c < a.c_hi; c += gridDim.x) {
        const ChunkRef r = chunk_ref(a, c);
        const uint32_t *sk;
        const TV *sv;
        uint32_t *dk;
        TV *dv;
        pass_buffers<TV>(a, pass, r, sk, sv, dk, dv);
        for (int i = threadIdx.x; i < 256; i += OT) h[i] = 0;
        __syncthreads();
        for (int64_t q = threadIdx.x; q < r.len; q += OT) atomicAdd(&h[(sk[r.start + q] >> shift) & 255u], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += OT) a.hist[(c - a.c_lo) * 256 + i] = h[i];
        __syncthreads();
    }
}

// One CTA per oversize bin: hist[c][d] becomes the destination offset (within
// the bin) of chunk c's first tuple with digit d.
__global__ void __launch_bounds__(256) k_over_offsets(const OversizeArgs a) {
    __shared__ int64_t scratch[40];
    const int d = threadIdx.x;  // one digit value per thread
    for (int64_t o = a.o_lo + blockIdx.x; o < a.o_hi; o += gridDim.x) {
        const int64_t c0 = a.over_chunk_off[o] - a.c_lo, c1 = a.over_chunk_off[o + 1] - a.c_lo;
        uint32_t run = 0;
        for (int64_t c = c0; c < c1; ++c) {
            const uint32_t v = a.hist[c * 256 + d];
            a.hist[c * 256 + d] = run;
            run += v;
        }
        int64_t total;
        const int64_t base = block_exclusive_scan<int64_t, 256>((int64_t)run, scratch, &total);
        for (int64_t c = c0; c < c1; ++c) a.hist[c * 256 + d] += (uint32_t)base;
        __syncthreads();
    }
}

template <class TV>
__global__ void __launch_bounds__(OT) k_over_scatter(const OversizeArgs a, int pass) {
    __shared__ uint32_t wc[256 * ONW];  // per (digit, warp) counts, then in-chunk offsets
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int shift = 8 * pass;
    for (int64_t c = a.c_lo + blockIdx.x; c < a.c_hi; c += gridDim.x) {
        const ChunkRef r = chunk_ref(a, c);
        const uint32_t *sk;
        const TV *sv;
        uint32_t *dk;
        TV *dv;
        pass_buffers<TV>(a, pass, r, sk, sv, dk, dv);
        for (int i = threadIdx.x; i < 256 * ONW; i += OT) wc[i] = 0;
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
                old = wc[dg * ONW + warp];
                wc[dg * ONW + warp] = old + __popc(peers);
            }
            old = __shfl_sync(FULL, old, leader);
            __syncwarp();
            lr[j] = old + __popc(peers & lanemask_lt());
            kk[j] = key;
        }
        __syncthreads();
        // per digit: exclusive prefix over warps (stable order inside the chunk)
        if (threadIdx.x < 256) {
            uint32_t run = 0;
            for (int w = 0; w < ONW; ++w) {
                const uint32_t v = wc[threadIdx.x * ONW + w];
                wc[threadIdx.x * ONW + w] = run;
                run += v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < OE; ++j) {
            const int64_t q = warp * OWS + j * 32 + lane;
            if (q < r.len) {
                const uint32_t dg = (kk[j] >> shift) & 255u;
                const int64_t pos = (int64_t)a.hist[(c - a.c_lo) * 256 + dg] + wc[dg * ONW + warp] + lr[j];
                dk[pos] = kk[j];
                dv[pos] = vv[j];
            }
        }
        __syncthreads();
    }
}

// Number of merged entries of each oversize bin = number of run heads.
__global__ void __launch_bounds__(OT) k_over_heads(const OversizeArgs a, int passes) {
    __shared__ int64_t scratch[40];
    for (int64_t c = a.c_lo + blockIdx.x; c < a.c_hi; c += gridDim.x) {
        const ChunkRef r = chunk_ref(a, c);
        const uint32_t *k = (passes & 1) ? a.skeys + (a.over_tuple_off[r.o] - a.over_base)
                                         : a.keys + (a.bin_off[r.bin] - a.tuple_base);
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

template <class TV>
cudaError_t run_oversize(const OversizeArgs &a, int passes, int num_sms, cudaStream_t s) {
    const int64_t g4 = (int64_t)num_sms * 4, g8 = (int64_t)num_sms * 8;
    const int64_t nc = a.c_hi - a.c_lo, no = a.o_hi - a.o_lo;
    const unsigned grid = (unsigned)(nc < g4 ? nc : g4);
    const unsigned ogrid = (unsigned)(no < g8 ? no : g8);
    cudaError_t e = cudaMemsetAsync(a.over_u + a.o_lo, 0, 8 * (size_t)no, s);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < passes; ++pass) {
        k_over_hist<TV><<<grid, OT, 0, s>>>(a, pass);
        k_over_offsets<<<ogrid, 256, 0, s>>>(a);
        k_over_scatter<TV><<<grid, OT, 0, s>>>(a, pass);
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

}  // namespace pb
