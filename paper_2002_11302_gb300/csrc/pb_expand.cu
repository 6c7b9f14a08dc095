// Expand phase with propagation blocking (Alg. 2 expand loop, Sec. III-C).
//
// The flop tuples are enumerated in the order of Alg. 2: column k of A (and
// row k of B), then each (rowid, aval) of A(:,k), then each (colid, bval) of
// B(k,:).  Tuple t lies in column k with F[k] <= t < F[k+1]; inside it,
// u = t - F[k] selects A entry u / nnz(B(k,:)) and B entry u % nnz(B(k,:)).
//
// Work split: the tuple range is cut into equal chunks (flop-balanced, not
// column-balanced, so hub columns of skewed inputs spread over many warps).
// A warp walks its chunk 32 tuples at a time.  For each group of 32 it loads
// the end offsets F[k+1] of the next 32 columns into the lanes once, and each
// lane finds its column with a 5-step shuffle search.
//
// Propagation blocking: tuple (i, j, a*b) goes to the bin holding row i (row
// ranges from the symbolic phase) as key = (i - first row of bin) << colbits | j
// and value a*b.  All B entries produced by one A entry share a bin, and such
// runs occupy consecutive lanes, so one lane per run reserves the whole run
// with a single atomic on the bin's cursor and the run is written to
// consecutive slots (warp-aggregated offsets; the writes of a run are
// contiguous 4-byte keys and 8-byte values).
#include "pb_common.cuh"

namespace pb {

namespace {

template <class TV, class IV>
__device__ inline TV tuple_product(IV a, IV b) {
    return static_cast<TV>(a * b);
}

template <class IV, class TV>
__global__ void __launch_bounds__(256) k_expand(const NumericArgs p) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const IV *__restrict__ valA = static_cast<const IV *>(p.valA);
    const IV *__restrict__ valB = static_cast<const IV *>(p.valB);
    TV *__restrict__ vals = static_cast<TV *>(p.vals);

    for (int64_t c = gwarp; c < p.nchunks; c += nwarps) {
        int64_t t = c * p.chunk;
        const int64_t tend = min(t + p.chunk, p.flop);
        int32_t kc = p.chunk_k[c];
        while (t < tend) {
            // Frontier: columns kc .. kc+31, one per lane.
            const int32_t kk = kc + lane;
            int64_t fend = INT64_MAX;
            int32_t a0 = 0, b0 = 0, lb = 1;
            if (kk < p.k) {
                fend = p.F[kk + 1];
                a0 = p.colptrA[kk];
                b0 = p.rowptrB[kk];
                lb = p.rowptrB[kk + 1] - b0;
            }
            int64_t fbeg = __shfl_up_sync(FULL, fend, 1);
            if (lane == 0) fbeg = p.F[kc];
            const int64_t span = min(tend, __shfl_sync(FULL, fend, 31));
            for (int64_t base = t; base < span; base += 32) {
                const int64_t tt = base + lane;
                const bool act = tt < span;  // active lanes form a prefix of the warp
                int l = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    int64_t f = __shfl_sync(FULL, fend, l + s - 1);
                    if (f <= tt) l += s;
                }
                const int64_t fk = __shfl_sync(FULL, fbeg, l);
                const int32_t A0 = __shfl_sync(FULL, a0, l);
                const int32_t B0 = __shfl_sync(FULL, b0, l);
                const int32_t LB = __shfl_sync(FULL, lb, l);
                int32_t ea = -1, eb = 0;
                if (act) {
                    const int64_t u = tt - fk;
                    int64_t ia;
                    if ((u >> 32) == 0)
                        ia = (uint32_t)u / (uint32_t)LB;
                    else
                        ia = u / LB;
                    ea = A0 + (int32_t)ia;
                    eb = B0 + (int32_t)(u - ia * LB);
                }
                // Runs of lanes sharing one A entry share one bin.
                const int32_t prev = __shfl_up_sync(FULL, ea, 1);
                const bool head = act && (lane == 0 || prev != ea);
                const uint32_t heads = __ballot_sync(FULL, head);
                const uint32_t actmask = __ballot_sync(FULL, act);
                if (act) {
                    const int32_t row = p.rowidxA[ea];
                    const IV av = valA[ea];
                    const int32_t col = p.colidxB[eb];
                    const IV bv = valB[eb];
                    const uint64_t info = p.rowinfo[row];
                    const uint32_t bin = (uint32_t)(info >> 32);
                    const uint32_t key = (uint32_t)info | (uint32_t)col;
                    const uint32_t upto = heads & (FULL >> (31 - lane));   // heads at lanes <= mine
                    const int sstart = 31 - __clz(upto);
                    const uint32_t above = heads & ~(FULL >> (31 - lane)); // heads at lanes > mine
                    const int send = above ? (__ffs(above) - 1) : (32 - __clz(actmask));
                    int64_t pos = 0;
                    if (head) {
                        const uint32_t len = (uint32_t)(send - sstart);
                        pos = p.bin_off[bin] + (int64_t)atomicAdd(&p.cursor[bin], len);
                        // a run past the bin's slots means the operands differ from the plan
                        if (pos + len > p.bin_off[bin + 1]) {
                            atomicOr(p.err, DEV_ERR_CAPACITY);
                            pos = -1;
                        }
                    }
                    pos = __shfl_sync(actmask, pos, sstart);
                    if (pos >= 0) {
                        pos += lane - sstart;
                        p.keys[pos] = key;
                        vals[pos] = tuple_product<TV, IV>(av, bv);
                    }
                }
            }
            t = span;
            kc += 32;
        }
    }
}

}  // namespace

cudaError_t launch_expand(const NumericArgs &a, cudaStream_t s) {
    if (a.flop <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (int64_t)a.num_sms * 8;
    const int64_t need = ceil_div<int64_t>(a.nchunks * 32, threads);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    switch (a.dtype) {
        case PB_F64: k_expand<double, double><<<(unsigned)blocks, threads, 0, s>>>(a); break;
        case PB_F32: k_expand<float, float><<<(unsigned)blocks, threads, 0, s>>>(a); break;
        case PB_F64_F32TUPLE: k_expand<double, float><<<(unsigned)blocks, threads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pb
