/*
 * FP64 reference GEMM for small-GEMM batches -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the oracle that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the library under
 * paper_2208_09822_gb300/.
 *
 * What it computes is the plain GEMM definition stated in Sec. I of the paper
 * ("C = alpha*A*B + beta*C", C is MxN, A is MxK, B is KxN) with the
 * transposition naming and column-major convention of the note under
 * Table I (first letter = A, "T" = the stored matrix is transposed):
 *
 *   C[i,j] = alpha * sum_{k<K} opA(i,k) * opB(k,j) + beta * C0[i,j]
 *   opA(i,k) = transA ? A[k + i*lda] : A[i + k*lda]
 *   opB(k,j) = transB ? B[j + k*ldb] : B[k + j*ldb]
 *
 * Every element is promoted to double; the sum runs k = 0,1,...,K-1.  alpha
 * and beta arrive already rounded to the instance's type by the caller.
 * Following the reference-BLAS convention (the paper is silent): beta == 0
 * means C0 is never read, and alpha == 0 or K == 0 skips the sum.
 *
 * The result goes to a separate double array, tight MxN column-major, so no
 * rounding back to the storage type happens here.
 *
 * Plant a mistake for the pin tests by compiling with -DORACLE_MUTANT=n
 * (see the switch in oracle_elem); the default build has none.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

static double load_elem(const void *base, int is_f64, int64_t idx)
{
    if (is_f64)
        return ((const double *)base)[idx];
    return (double)((const float *)base)[idx];
}

static double oracle_elem(int i, int j, int K, int lda, int ldb, int transA,
                          int transB, double alpha, double beta,
                          const void *A, const void *B, const void *C0,
                          int ldc, int is_f64)
{
    double sum = 0.0;
    double out;
    int k;
    if (alpha != 0.0) {
        for (k = 0; k < K; ++k) {
            int64_t ia = transA ? (int64_t)k + (int64_t)i * lda
                                : (int64_t)i + (int64_t)k * lda;
            int64_t ib = transB ? (int64_t)j + (int64_t)k * ldb
                                : (int64_t)k + (int64_t)j * ldb;
#if ORACLE_MUTANT == 1 /* transposed A operand */
            ia = transA ? (int64_t)i + (int64_t)k * lda
                        : (int64_t)k + (int64_t)i * lda;
#endif
#if ORACLE_MUTANT == 2 /* off-by-one in the k range (dropped last term) */
            if (k == K - 1)
                break;
#endif
            sum += load_elem(A, is_f64, ia) * load_elem(B, is_f64, ib);
        }
    }
    out = alpha * sum;
#if ORACLE_MUTANT == 3 /* wrong sign on the beta term */
    if (beta != 0.0)
        out -= beta * load_elem(C0, is_f64, (int64_t)i + (int64_t)j * ldc);
#elif ORACLE_MUTANT == 4 /* beta term read even when beta == 0 */
    out += beta * load_elem(C0, is_f64, (int64_t)i + (int64_t)j * ldc);
#else
    if (beta != 0.0)
        out += beta * load_elem(C0, is_f64, (int64_t)i + (int64_t)j * ldc);
#endif
    return out;
}

/*
 * Compute every instance of a batch.  Arrays are indexed by instance; the
 * matrices of instance t live at element offsets offA[t], offB[t], offC[t]
 * of the pools Apool, Bpool, Cpool (float or double, per is_f64).  The
 * result of instance t is written tight (leading dimension M) at Out +
 * offOut[t].  Returns 0, or -1 on a negative size.
 */
int oracle_gemm_batch(int64_t count, int is_f64,
                      const int32_t *M, const int32_t *N, const int32_t *K,
                      const int32_t *lda, const int32_t *ldb,
                      const int32_t *ldc, const uint8_t *transA,
                      const uint8_t *transB, const double *alpha,
                      const double *beta, const void *Apool,
                      const int64_t *offA, const void *Bpool,
                      const int64_t *offB, const void *Cpool,
                      const int64_t *offC, double *Out,
                      const int64_t *offOut, int nthreads)
{
    int64_t t;
    int bad = 0;
    size_t esz = is_f64 ? sizeof(double) : sizeof(float);
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (t = 0; t < count; ++t)
        if (M[t] < 0 || N[t] < 0 || K[t] < 0)
            bad = 1;
    if (bad)
        return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (t = 0; t < count; ++t) {
        const char *A = (const char *)Apool + offA[t] * esz;
        const char *B = (const char *)Bpool + offB[t] * esz;
        const char *C0 = (const char *)Cpool + offC[t] * esz;
        double *o = Out + offOut[t];
        int i, j;
        for (j = 0; j < N[t]; ++j)
            for (i = 0; i < M[t]; ++i)
                o[(int64_t)i + (int64_t)j * M[t]] = oracle_elem(
                    i, j, K[t], lda[t], ldb[t], transA[t], transB[t],
                    alpha[t], beta[t], A, B, C0, ldc[t], (int)is_f64);
    }
    return 0;
}

/* Number of threads an OpenMP region of this build uses (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
