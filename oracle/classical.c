/*
 * Oracle: classical matrix product, written as the plain definition
 *     C_ij = sum_p A_ip * B_pj                       (Section 2.1, F_C(N))
 * in FP64 (and, for pinning, in long double), row-major with leading
 * dimensions.  Loop order i-p-j, rows split across OpenMP threads, no
 * blocking, no BLAS.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of the benchmark.  Nothing on the GPU path links this.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* C (m x n) = A (m x k) * B (k x n), FP64. */
void oracle_gemm_f64(const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < m; ++i) {
        double *c = C + i * ldc;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t p = 0; p < k; ++p) {
            const double a = A[i * lda + p];
            const double *b = B + p * ldb;
            for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/* Same definition accumulated in long double (80-bit on x86, 128-bit on
 * aarch64); used to pin the FP64 oracle within the classical error bound. */
void oracle_gemm_ld(const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            long double s = 0.0L;
            for (int64_t p = 0; p < k; ++p)
                s += (long double)A[i * lda + p] * (long double)B[p * ldb + j];
            C[i * ldc + j] = (double)s;
        }
    }
}

/* Selected entries C_{rows[t], cols[t]} one by one, FP64 and long double;
 * for checking full-size products on a sample. */
void oracle_gemm_entries(const double *A, int64_t lda, const double *B, int64_t ldb,
                         int64_t k, const int64_t *rows, const int64_t *cols, int64_t count,
                         double *out_f64, double *out_ld) {
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < count; ++t) {
        const int64_t i = rows[t], j = cols[t];
        double s = 0.0;
        long double sl = 0.0L;
        for (int64_t p = 0; p < k; ++p) {
            const double a = A[i * lda + p], b = B[p * ldb + j];
            s += a * b;
            sl += (long double)a * (long double)b;
        }
        out_f64[t] = s;
        out_ld[t] = (double)sl;
    }
}
