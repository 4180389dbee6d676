/*
 * pgk_oracle.c -- CPU oracle for the parametric GEMM kernel family.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes is the plain definition of the product that the paper's
 * blocked MetaFork loop nest (Fig. "metamul", Section 2) and the generated
 * kernel0 (Fig. "cudamul", Section 2) evaluate:
 *
 *     c[p][q] += sum_z a[p][z] * b[z][q]
 *
 * written here without any blocking as C = beta*C0 + A*B, evaluated in binary64
 * (or long double for the self-check), row-major storage, loop order i-k-j.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Shared loop body: one output row i (global row index gi) of C = beta*C0 + A*B.
 * Arguments are the row pointers; the inner j loop walks a row of B. */
#define ORACLE_ROW(TA, TB)                                                    \
    do {                                                                      \
        double* crow = C + r * ldc;                                           \
        for (int64_t j = 0; j < N; ++j)                                       \
            crow[j] = (beta != 0.0) ? beta * C0[gi * ldc0 + j] : 0.0;         \
        const TA* arow = A + gi * lda;                                        \
        for (int64_t k = 0; k < K; ++k) {                                     \
            const double a = (double)arow[k];                                 \
            const TB* brow = B + k * ldb;                                     \
            for (int64_t j = 0; j < N; ++j) crow[j] += a * (double)brow[j];   \
        }                                                                     \
    } while (0)

/* C (nrows x N, ld ldc) = beta*C0 + A*B restricted to the output rows listed in
 * `rows` (all M rows when rows == NULL, then nrows must equal M).
 * A: M x K row-major FP32 (lda), B: K x N row-major FP32 (ldb), C0 fp64 (ldc0,
 * read only when beta != 0).  Returns 0, or -1 on a bad argument. */
int oracle_gemm_f32in(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                      const float* B, int64_t ldb, double beta, const double* C0,
                      int64_t ldc0, const int64_t* rows, int64_t nrows, double* C,
                      int64_t ldc, int nthreads) {
    if (M < 0 || N < 0 || K < 0 || nrows < 0) return -1;
    if (rows == NULL && nrows != M) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t gi = rows ? rows[r] : r;
        ORACLE_ROW(float, float);
    }
    (void)nthreads;
    return 0;
}

/* Same definition with binary64 operands (used for dequantised low-precision
 * operands, whose values q*scale need more than 24 significand bits). */
int oracle_gemm_f64in(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                      const double* B, int64_t ldb, double beta, const double* C0,
                      int64_t ldc0, const int64_t* rows, int64_t nrows, double* C,
                      int64_t ldc, int nthreads) {
    if (M < 0 || N < 0 || K < 0 || nrows < 0) return -1;
    if (rows == NULL && nrows != M) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t gi = rows ? rows[r] : r;
        ORACLE_ROW(double, double);
    }
    (void)nthreads;
    return 0;
}

/* Independent self-check of the two functions above on tiny inputs: the
 * textbook i-j-k dot product, accumulated in long double, no threads. */
int oracle_gemm_longdouble(int64_t M, int64_t N, int64_t K, const double* A,
                           const double* B, double* C) {
    if (M < 0 || N < 0 || K < 0) return -1;
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < N; ++j) {
            long double acc = 0.0L;
            for (int64_t k = 0; k < K; ++k)
                acc += (long double)A[i * K + k] * (long double)B[k * N + j];
            C[i * N + j] = (double)acc;
        }
    return 0;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* int32 form of the same definition, the paper's own data type (Fig.
 * "cudamul" declares int *a, *b, *c): C = beta*C0 + A*B evaluated modulo 2^32
 * and read back as two's complement.  Unsigned 32-bit arithmetic in C wraps
 * modulo 2^32 by definition, so every product and sum is taken there. */
int oracle_gemm_i32_wrap(int64_t M, int64_t N, int64_t K, const int32_t* A, int64_t lda,
                         const int32_t* B, int64_t ldb, int beta, const int32_t* C0,
                         int64_t ldc0, int32_t* C, int64_t ldc) {
    if (M < 0 || N < 0 || K < 0) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            uint32_t acc = beta ? (uint32_t)C0[i * ldc0 + j] : 0u;
            for (int64_t k = 0; k < K; ++k)
                acc += (uint32_t)A[i * lda + k] * (uint32_t)B[k * ldb + j];
            C[i * ldc + j] = (int32_t)acc;
        }
    }
    return 0;
}
