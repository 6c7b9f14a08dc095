// Sort, compress and ConvertCSR of Alg. 2, one bin per CTA pass.
//
// For each bin (a range of consecutive rows, Sec. III-A/III-D):
//   load     the bin's keys and values with two bulk global->shared copies
//            (the bin is read from DRAM exactly once: "in-cache sorting",
//            Sec. III-D, with shared memory playing the cache);
//   sort     by the packed (in-bin row, column) key (Sec. III-D).  First a
//            bucket pass on the top bits of (key - min key) with shared-memory
//            atomic counters; when every bucket is small (<= 32 tuples, the
//            common case for ER-like inputs) each bucket is finished by an
//            insertion sort.  Otherwise a stable LSD radix sort over 8-bit
//            digits (warp-level multisplit ranking with ballots) sorts the
//            whole bin.  Both give the same key order; equal keys are merged
//            next, so their order does not matter;
//   compress equal adjacent keys are summed (Sec. III-E: one pass over the
//            sorted tuples; sums accumulate in double);
//   ConvertCSR the bins are concatenated in row order: the bin's number of
//            merged entries is published and the exclusive prefix over all
//            earlier bins is found by decoupled look-back (bins are taken in
//            increasing order through a ticket counter, so every bin a CTA
//            waits for is already owned by a running CTA); then the column
//            indices, values and row pointers of the bin's rows are written.
#include "pb_common.cuh"

namespace pb {

namespace {

constexpr int RMAX = 4096;     // max rows of one bin (symbolic cuts bins at multiples of this)
constexpr int SMALL_BUCKET = 32;

template <int CAP, int THREADS, class TV>
struct SortSmem {
    static constexpr int NW = THREADS / 32;
    static constexpr int CNTN = (CAP > 256 * NW ? (CAP > RMAX ? CAP : RMAX) : (256 * NW > RMAX ? 256 * NW : RMAX));
    uint32_t kin[CAP];
    TV vin[CAP];
    uint32_t skey[CAP];
    uint16_t sidx[CAP];
    uint16_t sidx2[CAP];
    uint32_t cnt[CNTN];
    int64_t scratch[40];
    uint64_t bar;
    int64_t bin;
    int64_t prefix;
    uint32_t kmin, kmax, maxb;
    int32_t ok;
};

__device__ inline void write_rowptr(const NumericArgs &p, int64_t row, int64_t v) {
    if (p.rowptr64)
        p.rowptr64[row] = v;
    else
        p.rowptr32[row] = (int32_t)v;
}

// Exclusive scan in place of cnt[0..n) (n <= CNTN), all threads.
template <int THREADS>
__device__ inline void smem_exclusive_scan(uint32_t *cnt, int n, int64_t *scratch) {
    const int per = (n + THREADS - 1) / THREADS;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, n);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    int64_t total;
    int64_t pre = block_exclusive_scan<int64_t, THREADS>((int64_t)s, scratch, &total);
    uint32_t run = (uint32_t)pre;
    for (int i = lo; i < hi; ++i) {
        uint32_t c = cnt[i];
        cnt[i] = run;
        run += c;
    }
    __syncthreads();
}

// Decoupled look-back over bins (thread 0 only).  Returns the exclusive prefix.
__device__ inline int64_t lookback(uint64_t *status, int64_t b, uint64_t agg, uint32_t *err) {
    if (b == 0) {
        st_release_u64(&status[0], LB_PREFIX | agg);
        return 0;
    }
    st_release_u64(&status[b], LB_AGGREGATE | agg);
    uint64_t prefix = 0;
    int64_t j = b - 1;
    while (true) {
        uint64_t v;
        uint32_t spins = 0;
        while (true) {
            v = ld_acquire_u64(&status[j]);
            if (v >> LB_FLAG_SHIFT) break;
            if (++spins > SPIN_LIMIT) {
                atomicOr(err, DEV_ERR_TIMEOUT);
                v = LB_PREFIX;  // give up: treat as prefix 0 so the chain keeps moving
                break;
            }
            __nanosleep(32);
        }
        prefix += v & LB_VALUE_MASK;
        if ((v & ~LB_VALUE_MASK) == LB_PREFIX) break;
        --j;
    }
    st_release_u64(&status[b], LB_PREFIX | (prefix + agg));
    return (int64_t)prefix;
}

// Thread 0: publish this bin's merged count, find its prefix, check C's
// capacity, and let the last bin write nnz(C) and the final row pointer.
__device__ inline void publish_and_check(const NumericArgs &p, int64_t b, int64_t U, int64_t *prefix, int32_t *ok) {
    const int64_t P = lookback(p.status, b, (uint64_t)U, p.err);
    *prefix = P;
    int32_t good = p.count_only ? 0 : 1;
    if (!p.count_only && (P + U > p.cap || (p.rowptr32 && P + U > 0x7fffffffll))) {
        atomicOr(p.err, DEV_ERR_OVERFLOW);
        good = 0;
    }
    *ok = good;
    if (b == p.nbins - 1) {
        if (good) write_rowptr(p, p.m, P + U);
        if (p.nnz_dev) *p.nnz_dev = P + U;
    }
}

// An oversize bin (one row, more tuples than the on-chip capacity) was sorted
// in global memory before this kernel and its merged count is known: publish
// it at once, then stream the sorted run and write the merged entries.
template <int THREADS, class TV, class OV>
__device__ void stream_oversize_bin(const NumericArgs &p, int64_t b, int32_t row0, int32_t row1, int64_t off,
                                    int64_t N, uint32_t colmask, int64_t *scratch, int64_t *prefix, int32_t *okp) {
    const int tid = threadIdx.x;
    const int64_t o = p.over_scan[b];
    const bool in_scratch = (p.over_passes & 1) != 0;
    const uint32_t *k = in_scratch ? p.skeys + p.over_tuple_off[o] : p.keys + off;
    const TV *v = in_scratch ? static_cast<const TV *>(p.svals) + p.over_tuple_off[o]
                             : static_cast<const TV *>(p.vals) + off;
    OV *valC = static_cast<OV *>(p.valC);
    if (tid == 0) publish_and_check(p, b, p.over_u[o], prefix, okp);
    __syncthreads();
    const int64_t P = *prefix;
    const bool ok = *okp != 0;
    if (ok)
        for (int32_t r = row0 + tid; r < row1; r += THREADS) write_rowptr(p, r, r == row0 ? P : P + p.over_u[o]);
    int64_t running = 0;
    for (int64_t base = 0; base < N; base += THREADS) {
        const int64_t q = base + tid;
        const bool valid = q < N;
        const uint32_t key = valid ? k[q] : 0u;
        const bool head = valid && (q == 0 || k[q - 1] != key);
        int64_t chunk_total;
        const int64_t u = block_exclusive_scan<int64_t, THREADS>(head ? 1 : 0, scratch, &chunk_total);
        if (head && ok) {
            double acc = (double)v[q];
            for (int64_t r = q + 1; r < N && k[r] == key; ++r) acc += (double)v[r];
            p.colidx[P + running + u] = (int32_t)(key & colmask);
            valC[P + running + u] = (OV)acc;
        }
        running += chunk_total;
    }
    __syncthreads();
}

template <int CAP, int THREADS, class TV, class OV>
__global__ void __launch_bounds__(THREADS, (CAP <= 4096 ? 2 : 1)) k_binsort(const NumericArgs p) {
    using S = SortSmem<CAP, THREADS, TV>;
    constexpr int NW = THREADS / 32;
    constexpr int E = CAP / THREADS;  // items per thread
    constexpr int WS = CAP / NW;      // positions per warp in the LSD pass
    static_assert(WS % 32 == 0 && WS / 32 == E, "layout");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TV *__restrict__ gvals = static_cast<const TV *>(p.vals);
    OV *__restrict__ valC = static_cast<OV *>(p.valC);
    const uint32_t colmask = (p.colbits >= 32) ? 0xffffffffu : ((1u << p.colbits) - 1u);

    if (tid == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t phase = 0;

    while (true) {
        if (tid == 0) sm.bin = (int64_t)atomicAdd(p.ticket, 1u);
        fence_proxy_async_smem();  // earlier generic smem accesses before the next bulk copy
        __syncthreads();
        const int64_t b = sm.bin;
        if (b >= p.nbins) break;
        const int32_t row0 = p.bin_row[b], row1 = p.bin_row[b + 1];
        const int64_t off = p.bin_off[b];
        const int64_t Nfull = p.R[row1] - p.R[row0];
        if (Nfull > CAP) {
            stream_oversize_bin<THREADS, TV, OV>(p, b, row0, row1, off, Nfull, colmask, sm.scratch, &sm.prefix,
                                                 &sm.ok);
            continue;
        }
        int N = (int)Nfull;
        bool loaded = true;
        // ---- load the bin (bulk copies, 16-byte granules) -------------------
        if (N > 0) {
            const uint32_t n4 = (uint32_t)((N + 3) & ~3);
            if (tid == 0) {
                mbar_arrive_expect_tx(&sm.bar, n4 * 4u + n4 * (uint32_t)sizeof(TV));
                bulk_g2s(sm.kin, p.keys + off, n4 * 4u, &sm.bar);
                bulk_g2s(sm.vin, gvals + off, n4 * (uint32_t)sizeof(TV), &sm.bar);
            }
            loaded = mbar_wait_bounded(&sm.bar, phase);
            phase ^= 1u;
            if (!loaded) {
                if (tid == 0) atomicOr(p.err, DEV_ERR_TIMEOUT);
                N = 0;
            }
        }
        if (!__syncthreads_and(loaded)) {
            // a bulk copy may still be landing: wait for it (bounded) before the buffer is reused
            (void)mbar_wait_bounded(&sm.bar, phase ^ 1u);
            N = 0;
        }
        const int rows_b = row1 - row0;
        const uint32_t *sk = sm.skey;
        const uint16_t *si = sm.sidx;

        if (N > 0) {
            // ---- key range ----------------------------------------------------
            uint32_t kr[E];
            uint32_t lmin = 0xffffffffu, lmax = 0;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int q = tid + j * THREADS;
                kr[j] = (q < N) ? sm.kin[q] : 0u;
                if (q < N) {
                    lmin = min(lmin, kr[j]);
                    lmax = max(lmax, kr[j]);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lmin = min(lmin, __shfl_xor_sync(FULL, lmin, o));
                lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
            }
            if (tid == 0) {
                sm.kmin = 0xffffffffu;
                sm.kmax = 0;
                sm.maxb = 0;
            }
            __syncthreads();
            if (lane == 0) {
                atomicMin(&sm.kmin, lmin);
                atomicMax(&sm.kmax, lmax);
            }
            __syncthreads();
            const uint32_t kmin = sm.kmin;
            const uint32_t range = sm.kmax - kmin;
            const int rbits = range ? 32 - __clz(range) : 0;
            const int nbits = (N > 1) ? 32 - __clz((uint32_t)(N - 1)) : 0;
            const int shift = rbits > nbits ? rbits - nbits : 0;
            const int nbk = (int)(range >> shift) + 1;  // <= 2^nbits <= CAP
            // ---- bucket pass (MSD on the top bits) ------------------------------
            for (int i = tid; i < nbk; i += THREADS) sm.cnt[i] = 0;
            __syncthreads();
            uint32_t rk[E];
            uint32_t lmaxb = 0;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int q = tid + j * THREADS;
                if (q < N) {
                    rk[j] = atomicAdd(&sm.cnt[(kr[j] - kmin) >> shift], 1u);
                    lmaxb = max(lmaxb, rk[j] + 1u);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lmaxb = max(lmaxb, __shfl_xor_sync(FULL, lmaxb, o));
            if (lane == 0) atomicMax(&sm.maxb, lmaxb);
            __syncthreads();
            const bool small = sm.maxb <= SMALL_BUCKET;
            if (small) {
                smem_exclusive_scan<THREADS>(sm.cnt, nbk, sm.scratch);
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int q = tid + j * THREADS;
                    if (q < N) {
                        const uint32_t pos = sm.cnt[(kr[j] - kmin) >> shift] + rk[j];
                        sm.skey[pos] = kr[j];
                        sm.sidx[pos] = (uint16_t)q;
                    }
                }
                __syncthreads();
                for (int bk = tid; bk < nbk; bk += THREADS) {
                    const int lo = (int)sm.cnt[bk];
                    const int hi = (bk + 1 < nbk) ? (int)sm.cnt[bk + 1] : N;
                    for (int i = lo + 1; i < hi; ++i) {
                        const uint32_t kk = sm.skey[i];
                        const uint16_t xx = sm.sidx[i];
                        int jj = i - 1;
                        while (jj >= lo && sm.skey[jj] > kk) {
                            sm.skey[jj + 1] = sm.skey[jj];
                            sm.sidx[jj + 1] = sm.sidx[jj];
                            --jj;
                        }
                        sm.skey[jj + 1] = kk;
                        sm.sidx[jj + 1] = xx;
                    }
                }
                __syncthreads();
            } else {
                // ---- stable LSD radix sort, 8-bit digits ---------------------------
                uint32_t *srck = sm.kin;
                const uint16_t *srci = nullptr;  // identity on the first pass
                uint32_t *dstk = sm.skey;
                uint16_t *dsti = sm.sidx;
                const int passes_bits = rbits > 0 ? rbits : 1;
                for (int sh = 0; sh < passes_bits; sh += 8) {
                    for (int i = tid; i < 256 * NW; i += THREADS) sm.cnt[i] = 0;
                    __syncthreads();
                    uint32_t kk[E], lr[E];
                    uint16_t ii[E];
                    uint8_t dd[E];
#pragma unroll
                    for (int j = 0; j < E; ++j) {
                        const int q = warp * WS + j * 32 + lane;
                        const bool valid = q < N;
                        const uint32_t key = valid ? srck[q] : 0u;
                        const uint32_t d = ((key - kmin) >> sh) & 255u;
                        uint32_t peers = __ballot_sync(FULL, valid);
#pragma unroll
                        for (int bit = 0; bit < 8; ++bit) {
                            const bool on = (d >> bit) & 1u;
                            const uint32_t bb = __ballot_sync(FULL, on);
                            peers &= on ? bb : ~bb;
                        }
                        const int leader = valid ? (__ffs(peers) - 1) : lane;
                        uint32_t old = 0;
                        if (valid && lane == leader) {
                            old = sm.cnt[d * NW + warp];
                            sm.cnt[d * NW + warp] = old + __popc(peers);
                        }
                        old = __shfl_sync(FULL, old, leader);
                        __syncwarp();
                        lr[j] = old + __popc(peers & lanemask_lt());
                        kk[j] = key;
                        ii[j] = valid ? (srci ? srci[q] : (uint16_t)q) : 0;
                        dd[j] = (uint8_t)d;
                    }
                    __syncthreads();
                    smem_exclusive_scan<THREADS>(sm.cnt, 256 * NW, sm.scratch);
#pragma unroll
                    for (int j = 0; j < E; ++j) {
                        const int q = warp * WS + j * 32 + lane;
                        if (q < N) {
                            const uint32_t pos = sm.cnt[(uint32_t)dd[j] * NW + warp] + lr[j];
                            dstk[pos] = kk[j];
                            dsti[pos] = ii[j];
                        }
                    }
                    __syncthreads();
                    // next pass reads what this pass wrote
                    srck = dstk;
                    srci = dsti;
                    dstk = (dstk == sm.skey) ? sm.kin : sm.skey;
                    dsti = (dsti == sm.sidx) ? sm.sidx2 : sm.sidx;
                }
                sk = srck;
                si = srci;
            }
        }

        // ---- compress: count merged entries, per-row counts ----------------------
        for (int r = tid; r < rows_b; r += THREADS) sm.cnt[r] = 0;
        __syncthreads();
        int64_t local_u = 0;
        for (int q = tid; q < N; q += THREADS) {
            const uint32_t key = sk[q];
            if (q == 0 || sk[q - 1] != key) {
                ++local_u;
                atomicAdd(&sm.cnt[key >> p.colbits], 1u);
            }
        }
        const int64_t U = block_reduce_sum<int64_t, THREADS>(local_u, sm.scratch);
        if (tid == 0) publish_and_check(p, b, U, &sm.prefix, &sm.ok);
        __syncthreads();
        const int64_t P = sm.prefix;
        const bool ok = sm.ok != 0;
        // ---- row pointers of this bin's rows -----------------------------------
        smem_exclusive_scan<THREADS>(sm.cnt, rows_b, sm.scratch);
        if (ok)
            for (int r = tid; r < rows_b; r += THREADS) write_rowptr(p, row0 + r, P + sm.cnt[r]);
        // ---- merged entries in key order ---------------------------------------
        int64_t running = 0;
        for (int base = 0; base < N; base += THREADS) {
            const int q = base + tid;
            const bool valid = q < N;
            const uint32_t key = valid ? sk[q] : 0u;
            const bool head = valid && (q == 0 || sk[q - 1] != key);
            int64_t chunk_total;
            const int64_t u = block_exclusive_scan<int64_t, THREADS>(head ? 1 : 0, sm.scratch, &chunk_total);
            if (head && ok) {
                double acc = (double)sm.vin[si[q]];
                for (int r = q + 1; r < N && sk[r] == key; ++r) acc += (double)sm.vin[si[r]];
                const int64_t out = P + running + u;
                p.colidx[out] = (int32_t)(key & colmask);
                valC[out] = (OV)acc;
            }
            running += chunk_total;
        }
        __syncthreads();
    }
}

template <int CAP, int THREADS, class TV, class OV>
cudaError_t run_binsort(const NumericArgs &a, cudaStream_t s) {
    using S = SortSmem<CAP, THREADS, TV>;
    auto kern = k_binsort<CAP, THREADS, TV, OV>;
    const size_t smem = sizeof(S);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)a.num_sms * per_sm;
    if (grid > a.nbins) grid = a.nbins;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, THREADS, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <class TV, class OV>
cudaError_t dispatch_cap(const NumericArgs &a, cudaStream_t s) {
    switch (a.capacity) {
        case 2048: return run_binsort<2048, 512, TV, OV>(a, s);
        case 4096: return run_binsort<4096, 512, TV, OV>(a, s);
        case 8192: return run_binsort<8192, 512, TV, OV>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int binsort_max_capacity(int dtype) { return dtype == PB_F64 ? 8192 : 8192; }

cudaError_t launch_binsort(const NumericArgs &a, cudaStream_t s) {
    if (a.nbins <= 0) return cudaSuccess;
    switch (a.dtype) {
        case PB_F64: return dispatch_cap<double, double>(a, s);
        case PB_F32: return dispatch_cap<float, float>(a, s);
        case PB_F64_F32TUPLE: return dispatch_cap<float, double>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pb
