/*
 * CPU oracle for PB-SpGEMM -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the bench's CPU-baseline leg may
 * load this code.  It shares nothing with the CUDA library: no headers, no
 * helpers, no tables.  Everything is plain, sequential-per-row C in FP64.
 *
 * Conventions (Sec. II-A): A is m x k stored in CSC (colptr, rowidx, val),
 * B is k x n stored in CSR (rowptr, colidx, val), C = A*B is returned in CSR.
 * "flop" counts multiplications only (Sec. II-A).
 *
 * Functions and the passage each follows:
 *   pb_oracle_flop        Alg. 3 (symbolic phase): flop = sum_k nnz(A(:,k)) * nnz(B(k,:)).
 *   pb_oracle_row_flop    Sec. III-B, the per-row variant of Alg. 3: for every
 *                         A(i,k) != 0 add nnz(B(k,:)) to the count of row i.
 *   pb_oracle_expand      Alg. 2 expand loop (outer product): for every k, every
 *                         (rowid, aval) in A(:,k), every (colid, bval) in B(k,:),
 *                         emit the tuple (rowid, colid, aval*bval).
 *   pb_oracle_spgemm_*    The product itself by its plain definition
 *                         C(i,j) = sum_k A(i,k) B(k,j) over the structural
 *                         product (Sec. II-B: merging sums values with equal
 *                         (row, col); nothing is dropped), computed row by row
 *                         with a dense accumulator (the SPA of Sec. II-B,
 *                         Gustavson's algorithm).  Products of a row are added
 *                         in ascending k.  Besides C(i,j) it returns
 *                         sum_k |A(i,k) B(k,j)|, the scale of the rounding
 *                         error bound used by the parity tests.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int pb_oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of later calls (for the one-thread timing of the CPU baseline). */
void pb_oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Alg. 3: total multiplications of the outer-product formulation. */
int64_t pb_oracle_flop(int32_t k, const int32_t *colptrA, const int32_t *rowptrB) {
    int64_t flop = 0;
    for (int32_t i = 0; i < k; ++i) {
        int64_t nnzB = (int64_t)rowptrB[i + 1] - rowptrB[i];
        int64_t nnzA = (int64_t)colptrA[i + 1] - colptrA[i];
        flop += nnzB * nnzA;
    }
    return flop;
}

/* Sec. III-B per-row flop: rowflop[rowid] += nnz(B(i,:)) for every A(rowid, i). */
void pb_oracle_row_flop(int32_t m, int32_t k, const int32_t *colptrA, const int32_t *rowidxA,
                        const int32_t *rowptrB, int64_t *rowflop) {
    for (int32_t r = 0; r < m; ++r) rowflop[r] = 0;
    for (int32_t i = 0; i < k; ++i) {
        int64_t nnzB = (int64_t)rowptrB[i + 1] - rowptrB[i];
        for (int32_t e = colptrA[i]; e < colptrA[i + 1]; ++e) rowflop[rowidxA[e]] += nnzB;
    }
}

/* Alg. 2 expand: all flop tuples in loop order.  Output arrays hold flop entries. */
void pb_oracle_expand(int32_t k, const int32_t *colptrA, const int32_t *rowidxA, const double *valA,
                      const int32_t *rowptrB, const int32_t *colidxB, const double *valB,
                      int32_t *out_row, int32_t *out_col, double *out_val) {
    int64_t t = 0;
    for (int32_t i = 0; i < k; ++i) {
        for (int32_t ea = colptrA[i]; ea < colptrA[i + 1]; ++ea) {
            for (int32_t eb = rowptrB[i]; eb < rowptrB[i + 1]; ++eb) {
                out_row[t] = rowidxA[ea];
                out_col[t] = colidxB[eb];
                out_val[t] = valA[ea] * valB[eb];
                ++t;
            }
        }
    }
}

/* Row view of A: A is given by columns; Gustavson walks it by rows.  A stable
 * counting sort by row id keeps the entries of each row in ascending k.  Each
 * thread owns a block of rows and scans all of A, placing only its own rows,
 * so the scatter runs in parallel without shared writes. */
typedef struct {
    int32_t m;
    int64_t *ptr;   /* m+1 */
    int32_t *col;   /* nnz: the k of each entry */
    double *val;
} rows_of_A;

void pb_oracle_release(void *ctx) {
    rows_of_A *R = (rows_of_A *)ctx;
    if (!R) return;
    free(R->ptr); free(R->col); free(R->val); free(R);
}

void *pb_oracle_prepare(int32_t m, int32_t k, const int32_t *colptrA, const int32_t *rowidxA,
                        const double *valA) {
    int64_t nnz = colptrA[k];
    rows_of_A *R = (rows_of_A *)calloc(1, sizeof(rows_of_A));
    if (!R) return NULL;
    R->m = m;
    R->ptr = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    R->col = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    R->val = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    if (!R->ptr || !R->col || !R->val) {
        pb_oracle_release(R);
        return NULL;
    }
    for (int64_t e = 0; e < nnz; ++e) R->ptr[rowidxA[e] + 1] += 1;
    for (int32_t r = 0; r < m; ++r) R->ptr[r + 1] += R->ptr[r];
    int failed = 0;
#pragma omp parallel
    {
        int nt = 1, t = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        t = omp_get_thread_num();
#endif
        int32_t r0 = (int32_t)((int64_t)m * t / nt), r1 = (int32_t)((int64_t)m * (t + 1) / nt);
        int64_t *fill = (int64_t *)malloc(((size_t)(r1 - r0) + 1) * sizeof(int64_t));
        if (!fill) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int32_t r = r0; r < r1; ++r) fill[r - r0] = R->ptr[r];
            for (int32_t i = 0; i < k; ++i) {
                for (int32_t e = colptrA[i]; e < colptrA[i + 1]; ++e) {
                    int32_t r = rowidxA[e];
                    if (r < r0 || r >= r1) continue;
                    int64_t p = fill[r - r0]++;
                    R->col[p] = i;
                    R->val[p] = valA ? valA[e] : 0.0;
                }
            }
            free(fill);
        }
    }
    if (failed) {
        pb_oracle_release(R);
        return NULL;
    }
    return R;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Structural count of C(i,:) for each listed row.  Returns 0, or -1 on OOM. */
int pb_oracle_spgemm_count(const void *ctx, int32_t n, const int32_t *rowptrB, const int32_t *colidxB,
                           int64_t nrows_list, const int64_t *rows, int64_t *row_nnz) {
    const rows_of_A *R = (const rows_of_A *)ctx;
    int failed = 0;
#pragma omp parallel
    {
        int64_t *stamp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!stamp) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int32_t j = 0; j < n; ++j) stamp[j] = -1;
        }
        /* every thread reaches the worksharing loop, even one whose buffer failed */
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nrows_list; ++t) {
            if (!stamp) continue;
            int64_t i = rows[t];
            int64_t cnt = 0;
            for (int64_t p = R->ptr[i]; p < R->ptr[i + 1]; ++p) {
                int32_t kk = R->col[p];
                for (int32_t eb = rowptrB[kk]; eb < rowptrB[kk + 1]; ++eb) {
                    int32_t j = colidxB[eb];
                    if (stamp[j] != t) { stamp[j] = t; ++cnt; }
                }
            }
            row_nnz[t] = cnt;
        }
        free(stamp);
    }
    return failed ? -1 : 0;
}

/* Values of C(i,:) for each listed row: out_ptr[t] is where row t starts in the
 * output arrays (from pb_oracle_spgemm_count).  Columns ascending. */
int pb_oracle_spgemm_fill(const void *ctx, int32_t n, const int32_t *rowptrB, const int32_t *colidxB,
                          const double *valB, int64_t nrows_list, const int64_t *rows, const int64_t *out_ptr,
                          int32_t *out_col, double *out_val, double *out_abs) {
    const rows_of_A *R = (const rows_of_A *)ctx;
    int failed = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        double *acc_abs = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        int64_t *stamp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        int ok = acc && acc_abs && stamp;
        if (!ok) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int32_t j = 0; j < n; ++j) stamp[j] = -1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nrows_list; ++t) {
            if (!ok) continue;
            int64_t i = rows[t];
            int32_t *list = out_col + out_ptr[t];
            int64_t cnt = 0;
            for (int64_t p = R->ptr[i]; p < R->ptr[i + 1]; ++p) {
                int32_t kk = R->col[p];
                double a = R->val[p];
                for (int32_t eb = rowptrB[kk]; eb < rowptrB[kk + 1]; ++eb) {
                    int32_t j = colidxB[eb];
                    double prod = a * valB[eb];
                    if (stamp[j] != t) {
                        stamp[j] = t;
                        acc[j] = 0.0;
                        acc_abs[j] = 0.0;
                        list[cnt++] = j;
                    }
                    acc[j] += prod;
                    acc_abs[j] += fabs(prod);
                }
            }
            qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);
            for (int64_t q = 0; q < cnt; ++q) {
                out_val[out_ptr[t] + q] = acc[list[q]];
                out_abs[out_ptr[t] + q] = acc_abs[list[q]];
            }
        }
        free(acc); free(acc_abs); free(stamp);
    }
    return failed ? -1 : 0;
}
