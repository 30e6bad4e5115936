/*
 * iaat.h -- C ABI of the GB300 small-GEMM library (after IAAT, arXiv
 * 2208.09822).
 *
 * Operation (Sec. I of the paper):  C = alpha * op(A) * op(B) + beta * C
 *   C is M x N, op(A) is M x K, op(B) is K x N.
 *   op(X) = X (IAAT_OP_N) or X^T (IAAT_OP_T).  The case names NN/NT/TN/TT give
 *   A's op first, B's second (note under Table I).
 *   Storage is column-major (note under Table I): element (i, j) of a stored
 *   matrix X with leading dimension ldx is X[i + j * ldx].  The stored A is
 *   M x K (op N) or K x M (op T); the stored B is K x N (op N) or N x K (op T).
 *
 * Domain (Sec. I and Sec. VI): cbrt(M*N*K) <= 80, or <= 32 for the TN case.
 *   It is checked in integer form, M*N*K <= 512000 (TN: <= 32768); larger
 *   problems are refused with IAAT_ERR_NOT_SMALL and never computed.
 *
 * Argument rules (reference-BLAS xGEMM conventions; the paper is silent):
 *   M, N, K >= 0;  lda >= max(1, transA ? K : M);  ldb >= max(1, transB ? N : K);
 *   ldc >= max(1, M).  M == 0 or N == 0: nothing is done.  alpha == 0 or
 *   K == 0: C = beta * C and A, B are not read.  beta == 0: C is not read, so
 *   NaN or Inf already in C does not reach the result.  Elements of C outside
 *   its M x N part (the ld padding) are never written.  Pointers must be
 *   aligned to the element size: 4 bytes (FP32), 8 (FP64 and complex float),
 *   16 (complex double); otherwise IAAT_ERR_MISALIGNED.
 *   A, B and C of one call or one plan must not overlap in written memory.
 *
 * Memory and execution:
 *   Every A, B, C pointer is a DEVICE pointer owned by the caller.  All work
 *   is enqueued on the caller's stream (a cudaStream_t passed as void*, NULL
 *   for the legacy default stream) and returns without waiting for the GPU.
 *   No exception crosses this ABI; every entry point returns a status, and
 *   iaat_last_error() gives a message for the calling thread's last failure.
 *   On any error status nothing has been enqueued.
 *
 * The library reads, as 16-byte-aligned blocks, the aligned 16-byte granules
 * that contain the elements of A, B and C it needs; bytes of those granules
 * outside the matrices are read but never used or written (a granule never
 * crosses a page, so this cannot fault).
 */
#ifndef IAAT_H
#define IAAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { IAAT_OP_N = 0, IAAT_OP_T = 1 } iaat_op_t;

/* Element types.  IAAT_C32 / IAAT_C64 are the complex types of Table I
 * (CGEMM / ZGEMM): an element is a (real, imaginary) pair stored next to each
 * other, 2 floats (8 bytes) or 2 doubles (16 bytes); leading dimensions count
 * elements.  Complex batches are planned with iaat_plan_create_complex. */
typedef enum { IAAT_F32 = 0, IAAT_F64 = 1, IAAT_C32 = 2, IAAT_C64 = 3 } iaat_dtype_t;

/* Arithmetic used for an FP32 plan (FP64 plans accept only the default).
 * DEFAULT: FP32 FFMA on the CUDA cores (FP64: DFMA).
 * 3XBF16:  tcgen05 tensor cores, X = Xh + Xl with Xh = bf16(X), Xl =
 *          bf16(X - Xh); Ah*Bh + Ah*Bl + Al*Bh accumulated in FP32.
 * TF32:    tcgen05 kind::tf32 on round-to-nearest TF32 inputs, FP32 accumulate.
 * FP16:    tcgen05 kind::f16 on FP16-rounded inputs, FP32 accumulate.
 * 6XBF16:  tcgen05 tensor cores, X = Xh + Xm + Xl (three BF16 terms, each
 *          the rounding of what the previous ones leave); the six products
 *          of order up to two (mm, lh, hl, mh, hm, hh) accumulated in FP32,
 *          for FFMA-like accuracy per instance also at tiny K. */
typedef enum {
    IAAT_PREC_DEFAULT = 0,
    IAAT_PREC_3XBF16 = 1,
    IAAT_PREC_TF32 = 2,
    IAAT_PREC_FP16 = 3,
    IAAT_PREC_6XBF16 = 4
} iaat_precision_t;

typedef enum {
    IAAT_OK = 0,
    IAAT_ERR_INVALID_VALUE = 1,   /* bad size, leading dimension, pointer or enum */
    IAAT_ERR_NOT_SMALL = 2,       /* outside the small-GEMM domain */
    IAAT_ERR_MISALIGNED = 3,      /* pointer not aligned to its element size */
    IAAT_ERR_UNSUPPORTED = 4,     /* combination not built (e.g. FP64 + 3XBF16) */
    IAAT_ERR_CUDA = 5,            /* a CUDA runtime call failed */
    IAAT_ERR_DEVICE_TIMEOUT = 6,  /* a kernel gave up waiting and stopped early */
    IAAT_ERR_OOM = 7              /* device or host allocation failed */
} iaat_status_t;

/* One GEMM instance of a grouped call.  alpha and beta are rounded to the
 * plan's type.  transA / transB take iaat_op_t values. */
typedef struct {
    int32_t M, N, K;
    int32_t lda, ldb, ldc;
    int32_t transA, transB;
    double alpha, beta;
    const void *A;
    const void *B;
    void *C;
} iaat_gemm_desc_t;

/* One complex GEMM instance (CGEMM / ZGEMM, Table I rows 3-4):
 *   C = alpha * op(A) * op(B) + beta * C  with complex alpha, beta, A, B, C,
 * op = N or T as above (the paper's four cases; no conjugate transpose).
 * Same sizes, leading dimensions, domain and argument rules as the real
 * GEMM; alpha == 0 and beta == 0 mean both parts zero.  alpha and beta are
 * rounded to the component type of the plan.  Each complex multiply-add is
 * four real multiply-adds on the FP32 / FP64 pipes, so a plan's flops count
 * 8*M*N*K per instance (Eq. 2). */
typedef struct {
    int32_t M, N, K;
    int32_t lda, ldb, ldc;
    int32_t transA, transB;
    double alpha_re, alpha_im;
    double beta_re, beta_im;
    const void *A;
    const void *B;
    void *C;
} iaat_cgemm_desc_t;

typedef struct iaat_plan_s *iaat_plan_t;

/* Optional knobs of iaat_plan_create (pass NULL for the tuned defaults).
 * Zero in any field means "use the tuned default". */
typedef struct {
    int32_t ctas_per_sm;       /* persistent CTAs per SM (the kernel uses 1) */
    int32_t max_group_tasks;   /* tasks in one pipeline stage (<= 32) */
    int32_t force_variant;     /* 0: tiler's choice; k > 0: register-tile variant k-1 */
    int32_t inject_fault;      /* testing only: 1 = corrupt the first stage's task
                                  count so the kernel must detect it, give up and
                                  report IAAT_ERR_DEVICE_TIMEOUT via iaat_plan_check */
    int32_t route_k_below;     /* tensor-core plans only: instances with K below this
                                  value run on the FP32 CUDA-core kernel instead, in
                                  the same iaat_gemm_grouped call (a second launch on
                                  the same stream).  The split's dropped low-low term
                                  is not averaged out at tiny K; with 8, every
                                  instance meets FP32-like accuracy.  0: no routing */
    int32_t kernel;            /* FP32 plans: 0 = default, 1 = the stage-program kernels
                                  (one producer warp per SM fills pipeline stages that
                                  all compute warps share), 2 = the stream kernels (the
                                  CUDA-core warp-stream kernel, in which every warp
                                  streams its own warp tasks, and the tensor-core
                                  pack-stream kernel, in which four warp groups with a
                                  producer warp each stream dense 128-row packs),
                                  3 = the warp-tile tensor-core kernel (tensor-core
                                  precisions only: every warp stages, converts and
                                  multiplies its own blocks of at most 32 x 32, op(A)
                                  from tensor memory; the CUDA-core part of a routed
                                  plan then takes the default), 4 = the warp-direct
                                  CUDA-core kernel (FP32 or FP64 plans of the default
                                  precision: every warp runs its own blocks of at most
                                  32 rows straight from global memory, no staging
                                  pipeline; for batches of tiny instances).  Complex
                                  plans always run stage programs, FP64 plans stage
                                  programs unless 4 is asked for */
    int32_t route_mnk_below;   /* tensor-core plans only: instances with M*N*K below
                                  this value also run on the FP32 CUDA-core kernel
                                  (the same second launch as route_k_below); the
                                  tensor cores then take only the instances large
                                  enough to fill their tiles.  0: no size routing */
    int32_t route_kernel;      /* routed tensor-core plans: the kernel family of the
                                  CUDA-core part (values as for kernel: 1, 2 or 4);
                                  0: the main plan's family when that is 1 or 2,
                                  else the default */
} iaat_plan_options_t;

/* Statistics of a plan (iaat_plan_info). */
typedef struct {
    int64_t instances;         /* descriptors passed in */
    int64_t active;            /* instances that need work */
    int64_t tasks;             /* work pieces after splitting */
    int64_t groups;            /* pipeline stages */
    int64_t blocks;            /* warp blocks over all tasks (tensor-core plans: MMA
                                  packs, plus the warp blocks of routed instances) */
    int64_t flops;             /* sum of 2*M*N*K over active instances (Eq. 1);
                                  complex plans 8*M*N*K (Eq. 2) */
    int64_t algorithmic_bytes; /* A, B, C written, C read when beta != 0 */
    int64_t plan_bytes;        /* device bytes the plan holds (descriptors) */
    int32_t grid;              /* CTAs of each launch */
    int32_t kernels;           /* kernels one iaat_gemm_grouped launches (2 when a
                                  tensor-core plan routes small-K instances) */
    int32_t dtype, precision;
    int32_t kernel_family;     /* the kernels the plan runs: 1 stage programs, 2 stream
                                  (warp-stream / pack-stream), 3 warp-tile, 4 warp-direct;
                                  for a routed plan, its tensor-core part's */
    int32_t reserved;
} iaat_plan_info_t;

/* Single small GEMM, FP32 / FP64 (BLAS sgemm/dgemm argument order, Sec. I).
 * Device pointers; asynchronous on `stream`.  The instance's tasks travel in
 * the kernel's parameter block, at most 32 per launch, so the call allocates
 * nothing and shares no device state with other calls (an instance cut into
 * more pieces, such as 512000 x 1 x 1, takes several launches in a row on
 * `stream`); a device-side time-out is reported by iaat_plan_check(NULL,
 * stream).  For the paper's "same size repeatedly" use (Sec. VII), a plan
 * (iaat_plan_create) keeps the tiling and descriptors on the device and
 * replays them. */
iaat_status_t iaat_sgemm(int transA, int transB, int M, int N, int K,
                         float alpha, const float *A, int lda,
                         const float *B, int ldb, float beta, float *C,
                         int ldc, void *stream);
iaat_status_t iaat_dgemm(int transA, int transB, int M, int N, int K,
                         double alpha, const double *A, int lda,
                         const double *B, int ldb, double beta, double *C,
                         int ldc, void *stream);

/* Single small complex GEMM, CGEMM (complex float) / ZGEMM (complex double),
 * Table I rows 3-4: the operation, cases and argument rules of
 * iaat_cgemm_desc_t with one instance.  alpha and beta point to (re, im)
 * pairs in host memory, read during the call; A, B, C are device pointers
 * aligned to 8 (CGEMM) or 16 (ZGEMM) bytes.  Asynchronous on `stream`, no
 * allocation: the call plans on the host and copies the instance's scalars
 * and stage programs into one fixed device scratch array of 512 KB (a
 * file-scope __device__ array every GPU loading this library holds), then
 * launches the complex kernel, its C cut into pieces of about 16 x 16
 * (ZGEMM) or 32 x 32 (CGEMM) that run on separate SMs.  Calls reuse that
 * scratch, so calls that overlap on the GPU (other streams or threads) race:
 * order them on one stream.  A device time-out is reported by
 * iaat_plan_check(NULL, stream).  Batches: iaat_plan_create_complex. */
iaat_status_t iaat_cgemm(int transA, int transB, int M, int N, int K,
                         const float *alpha, const void *A, int lda,
                         const void *B, int ldb, const float *beta, void *C,
                         int ldc, void *stream);
iaat_status_t iaat_zgemm(int transA, int transB, int M, int N, int K,
                         const double *alpha, const void *A, int lda,
                         const void *B, int ldb, const double *beta, void *C,
                         int ldc, void *stream);

/* Allocation-free grouped GEMM.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory after start-up
 * -- for example a serving process that reserves all GPU memory at launch and
 * treats any later cudaMalloc as a failure, because cudaMalloc/cudaFree
 * synchronise the device and can fail under memory pressure.
 *
 * Same arguments and results as iaat_plan_create + iaat_gemm_grouped with the
 * default precision, but nothing is allocated on the device or the heap: the
 * plan is built in static host arrays, copied with cudaMemcpyAsync on
 * `stream` into one fixed device scratch array of about 545 KB (a file-scope
 * __device__ array that every GPU loading this library holds until the
 * process exits), and the CUDA-core grouped kernel runs from there.
 * Limits: at most 8192 tasks per call (an instance is one task, or a few
 * column pieces when its operands do not fit one pipeline stage); larger
 * batches return IAAT_ERR_INVALID_VALUE and enqueue nothing.
 * The first call on a device looks up the scratch array's device address
 * (and reads the tuning cache).  The call cannot be captured in a CUDA
 * graph: it copies each call's plan from host arrays that the next call
 * reuses, so on a capturing stream it returns IAAT_ERR_UNSUPPORTED and
 * enqueues nothing.  Every call reuses the same scratch array and the kernel
 * reads it while it runs, so calls that overlap on the GPU (other streams,
 * other threads) race and give wrong results: order them on one stream.  A
 * device time-out is reported by iaat_plan_check(NULL, stream). */
iaat_status_t iaat_gemm_grouped_noalloc(const iaat_gemm_desc_t *descs, int64_t count,
                                        iaat_dtype_t dtype, void *stream);

/* Build a plan for `count` instances (host array `descs`, device pointers
 * inside): validates every instance (the first failure's index is in
 * iaat_last_error), tiles each one into warp blocks (run-time stage,
 * Sec. V-A), groups the pieces into pipeline stages, orders them for the
 * persistent schedule and copies the descriptors to the device (synchronous;
 * uses the current CUDA device).  The plan keeps the pointers: re-plan when
 * they change.  `opts` may be NULL.  dtype IAAT_F32 or IAAT_F64 (complex
 * dtypes: iaat_plan_create_complex; here IAAT_ERR_INVALID_VALUE).
 * A default tensor-core plan (opts NULL or kernel 0, on the stage programs)
 * sends the instances a pipeline stage cannot hold whole to the warp-tile
 * kernel, which stages K in pieces, when they carry at least a quarter of the
 * batch's bytes; one iaat_gemm_grouped then launches both (iaat_plan_info:
 * kernels).  On the stage programs alone (kernel 1) such
 * instances are cut into row / column pieces, and one whose row of A and
 * column of B do not fit a stage (e.g. 1 x 1 x 20000) is rejected with
 * IAAT_ERR_UNSUPPORTED. */
iaat_status_t iaat_plan_create(const iaat_gemm_desc_t *descs, int64_t count,
                               iaat_dtype_t dtype, iaat_precision_t precision,
                               const iaat_plan_options_t *opts,
                               iaat_plan_t *out);

/* Build a plan for `count` complex instances, dtype IAAT_C32 (CGEMM) or
 * IAAT_C64 (ZGEMM): the same validation, tiling into warp blocks of the
 * complex register-tile family, stage programs and persistent schedule as
 * iaat_plan_create (which refuses complex dtypes), plus a device table of
 * each instance's alpha and beta that the plan owns.  The complex kernel runs
 * on the CUDA cores (FFMA / DFMA) only.  Run it with iaat_gemm_grouped;
 * check, inspect and free it like any plan.  `opts` may be NULL (its
 * force_variant picks from the complex family, 1..5). */
iaat_status_t iaat_plan_create_complex(const iaat_cgemm_desc_t *descs, int64_t count,
                                       iaat_dtype_t dtype,
                                       const iaat_plan_options_t *opts,
                                       iaat_plan_t *out);

/* Enqueue one execution of the plan (the kernel executing plan, Sec. V-B) on
 * `stream`: one persistent kernel launch, no host synchronisation and no
 * allocation, so it can be captured in a CUDA graph. */
iaat_status_t iaat_gemm_grouped(iaat_plan_t plan, void *stream);

/* Synchronise `stream`, then report (and clear) a device-side error of the
 * plan's kernels: IAAT_ERR_DEVICE_TIMEOUT if a bounded wait gave up or a
 * malformed plan record was refused.  plan == NULL checks the error words of
 * the single calls and of the allocation-free entry point; both are read and
 * cleared, and the first error is returned.  Sec. V-B runs a plan's kernels;
 * this is the host's view of how that run ended. */
iaat_status_t iaat_plan_check(iaat_plan_t plan, void *stream);

iaat_status_t iaat_plan_info(iaat_plan_t plan, iaat_plan_info_t *info);

/* Free the plan's device memory (synchronises the device first).  The
 * counterpart of building the kernel executing plan (Sec. V-B): a plan can
 * be replayed any number of times until it is destroyed. */
iaat_status_t iaat_plan_destroy(iaat_plan_t plan);

/* Install-time tuning (Sec. III-A and Sec. IV: the kernels are tuned once
 * for the hardware they run on).  Times the register-tile variants on the
 * current GPU for (dtype, precision), the stage size on an uneven batch and,
 * for FP32, the kernel family default plans run (FFMA: stage programs,
 * stream or warp-direct; tensor cores: stage programs, stream or warp-tile;
 * another family only when at least 3% faster than the stage programs),
 * and writes the per-variant cost scales, stage sizes and families as JSON to
 * `cache_path` (NULL: the path in IAAT_TUNE_CACHE, else no file), together
 * with the GPU's name, SM count, driver and runtime versions.  Later
 * processes read the cache named by IAAT_TUNE_CACHE and ignore it when any
 * of those differ from the current GPU's.  Synchronous; allocates its own
 * test matrices. */
iaat_status_t iaat_autotune(iaat_dtype_t dtype, iaat_precision_t precision,
                            const char *cache_path);

/* Measure the FP32 FFMA (IAAT_F32) or FP64 DFMA (IAAT_F64) pipe throughput
 * of the current GPU in GFLOP/s (2 flops per FMA), the compute roof of the
 * CUDA-core paths.  Synchronous; allocates a small scratch buffer. */
iaat_status_t iaat_fma_peak(iaat_dtype_t dtype, double *gflops);

/* The pack step of a conventional GEMM, for ablation only (the GPU analogue
 * of Fig. 3, the share of the time a traditional GEMM spends packing; the
 * library's own paths never pack).  iaat_pack_create validates the instances
 * like iaat_plan_create (FP32 or FP64), allocates a device workspace and
 * writes to the caller's host array `packed` (count entries) descriptors of
 * the same GEMMs on packed operands: op(A) as a tight column-major M x K
 * matrix and op(B) as a tight K x N one in the workspace, transA = transB = N,
 * lda = max(1, M), ldb = max(1, K); C, ldc, alpha and beta unchanged
 * (instances that read neither A nor B get NULL there).  *bytes_moved (may be
 * NULL) receives the pack kernel's algorithmic bytes per run: op(A) and op(B)
 * of every packed instance read once and written once.  iaat_pack_run
 * enqueues the copy (one kernel) on `stream`; plan the packed descriptors with
 * iaat_plan_create.  iaat_pack_destroy synchronises the device and frees the
 * workspace, which the packed descriptors point into. */
typedef struct iaat_pack_s *iaat_pack_t;
iaat_status_t iaat_pack_create(const iaat_gemm_desc_t *descs, int64_t count,
                               iaat_dtype_t dtype, iaat_gemm_desc_t *packed,
                               int64_t *bytes_moved, iaat_pack_t *out);
iaat_status_t iaat_pack_run(iaat_pack_t pack, void *stream);
iaat_status_t iaat_pack_destroy(iaat_pack_t pack);

/* Host-only view of the run-time tiler (no GPU needed).  Tiles one M x N
 * (x K) instance of the given type and case with the library's register-tile
 * variants (all four dtypes; complex ones with the complex family) and
 * writes up to `cap` blocks as (row0, col0, rows, cols) quadruples to
 * `blocks`.  This is the per-instance choice; inside a plan, an instance too
 * large for the staging ring to hold one per consumer warp is given smaller
 * tiles (more warp blocks), and large instances are first cut into pieces.  Returns the number of blocks (may exceed `cap`),
 * or -1 on bad arguments. */
int64_t iaat_tile(iaat_dtype_t dtype, int transA, int transB, int M, int N,
                  int K, int32_t *blocks, int64_t cap);

/* Host-only exact-cover tiler under the paper's memops objective (Sec. V-A,
 * "Minimal Memops"): tile an M x N C into row strips whose heights are the
 * `nheights` entries of `heights`, each strip cut into blocks of widths
 * 1..max_width[h] of that height, minimising sum(m_i + n_i).  Writes up to
 * `cap` quadruples to `blocks`; returns the block count, or -1 when no exact
 * cover exists or the arguments are bad.  `*sum_out` receives sum(m_i+n_i). */
int64_t iaat_tile_exact(int M, int N, const int32_t *heights,
                        const int32_t *max_width, int nheights,
                        int32_t *blocks, int64_t cap, int64_t *sum_out);

/* Version string of the library. */
const char *iaat_version(void);

/* Message for the calling thread's last failing call ("" if none): which
 * instance broke which rule of Sec. I's domain or of the BLAS argument
 * rules, or which CUDA call failed.  Thread-local; valid until the thread's
 * next failing call. */
const char *iaat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IAAT_H */
