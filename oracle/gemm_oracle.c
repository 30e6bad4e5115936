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
 * (1-4: see the switch in oracle_elem; 5-7: oracle_cgemm_batch); the default
 * build has none.
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

/* Number of threads an OpenMP region of the compiled oracle uses (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Complex GEMM (CGEMM / ZGEMM; Table I rows 3-4 and the type list of Sec. III-A,
 * which name single- and double-precision complex matrix multiplication with
 * the same four cases NN, NT, TN, TT and no conjugation):
 *
 *   C[i,j] = alpha * sum_{k<K} opA(i,k) * opB(k,j) + beta * C0[i,j]
 *
 * with complex alpha, beta and entries.  An element is a (real, imaginary)
 * pair stored next to each other -- 2 floats (is_c64 == 0) or 2 doubles --
 * and leading dimensions and offsets count elements.  Each complex product
 * is the textbook one, (a+bi)(c+di) = (ac - bd) + (ad + bc)i: four real
 * multiplies and four real additions per multiply-add, the 8 flops that
 * Eq. 2 counts.  Everything is promoted to double and the sum runs k
 * ascending.  beta == 0 (both parts) means C0 is never read; alpha == 0 (both
 * parts) or K == 0 skips the sum.  alpha and beta arrive as (re, im) pairs,
 * already rounded to the instance's component type.  The result of instance
 * t goes tight (leading dimension M) to Out as (re, im) double pairs starting
 * at pair offOut[t].
 *
 * Planted mistakes (pin tests only): 5 conjugates A, 6 drops the imaginary
 * part of alpha, 7 flips the sign of beta's imaginary part.
 */
static void load_cplx(const void *base, int is_c64, int64_t idx, double *re, double *im)
{
    if (is_c64) {
        *re = ((const double *)base)[2 * idx];
        *im = ((const double *)base)[2 * idx + 1];
    } else {
        *re = (double)((const float *)base)[2 * idx];
        *im = (double)((const float *)base)[2 * idx + 1];
    }
}

int oracle_cgemm_batch(int64_t count, int is_c64,
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
    size_t esz = is_c64 ? 2 * sizeof(double) : 2 * sizeof(float);
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
        double *o = Out + 2 * offOut[t];
        double ar = alpha[2 * t], ai = alpha[2 * t + 1];
        double br = beta[2 * t], bi = beta[2 * t + 1];
        int i, j, k;
#if ORACLE_MUTANT == 6
        ai = 0.0;
#endif
#if ORACLE_MUTANT == 7
        bi = -bi;
#endif
        for (j = 0; j < N[t]; ++j) {
            for (i = 0; i < M[t]; ++i) {
                double sr = 0.0, si = 0.0, outr, outi;
                if (ar != 0.0 || ai != 0.0) {
                    for (k = 0; k < K[t]; ++k) {
                        int64_t ia = transA[t] ? (int64_t)k + (int64_t)i * lda[t]
                                               : (int64_t)i + (int64_t)k * lda[t];
                        int64_t ib = transB[t] ? (int64_t)j + (int64_t)k * ldb[t]
                                               : (int64_t)k + (int64_t)j * ldb[t];
                        double xr, xi, yr, yi;
                        load_cplx(A, is_c64, ia, &xr, &xi);
                        load_cplx(B, is_c64, ib, &yr, &yi);
#if ORACLE_MUTANT == 5
                        xi = -xi;
#endif
                        sr += xr * yr - xi * yi;
                        si += xr * yi + xi * yr;
                    }
                }
                outr = ar * sr - ai * si;
                outi = ar * si + ai * sr;
                if (br != 0.0 || bi != 0.0) {
                    double cr, ci;
                    load_cplx(C0, is_c64, (int64_t)i + (int64_t)j * ldc[t], &cr, &ci);
                    outr += br * cr - bi * ci;
                    outi += br * ci + bi * cr;
                }
                o[2 * ((int64_t)i + (int64_t)j * M[t])] = outr;
                o[2 * ((int64_t)i + (int64_t)j * M[t]) + 1] = outi;
            }
        }
    }
    return 0;
}
