/*
 * tsvd.h -- C ABI of the GB300 (sm_103a) mixed precision Gram-matrix thin SVD.
 *
 * Method: Algorithm 1 of Carson, Ma, Shao, "Mixed precision thin SVD
 * algorithms based on the Gram matrix" (arXiv 2603.11953).  For a full-rank
 * tall-and-skinny A (m >= n), with working precision u and higher precision
 * u_h:
 *   1. M_h = A^T A formed in the higher precision          (Alg. 1 lines 1-2)
 *   2. M_h = V_h Sigma_h^2 V_h^T in the higher precision   (Alg. 1 line 3): by
 *      default (n <= 256) a pivoted Cholesky M_h = R^T R followed by a
 *      one-sided Jacobi SVD of R^T (the factor-then-SVD structure of Alg. 2,
 *      all in the higher precision); two-sided Jacobi on M_h (Sec. 2.1) on
 *      request (tsvd_opts.eig_variant); Algorithm 2 as written on request
 *   3. Sigma, V rounded to working precision               (Alg. 1 lines 4-5)
 *   4. U = A (V Sigma^{-1}) in working precision           (Alg. 1 line 6)
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major.  A has m rows, n columns, leading dimension
 *     lda >= m (elements).  All A/G/sigma/V/U pointers are DEVICE pointers
 *     owned by the caller; the library never frees them.
 *   - Work is enqueued on the handle's stream and is asynchronous.  Argument
 *     errors are detected on the host and returned immediately (nothing is
 *     enqueued).  Numeric outcomes (non-finite input, rank deficiency, Jacobi
 *     non-convergence) are only known on the device: they are written to the
 *     optional tsvd_info (device or pinned host memory) and can be fetched
 *     with tsvd_sync_status().
 *   - sigma is sorted descending; each column of V is signed so that its
 *     largest-magnitude entry is positive (lowest row index wins ties); the
 *     columns of U follow V.
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 *   - There is no CPU fallback: every step runs in the library's CUDA kernels.
 *   - The handle grows device workspace on demand (cudaMalloc); the first call
 *     at a given size allocates, later calls of the same or smaller size do
 *     not.
 */
#ifndef TSVD_H
#define TSVD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TSVD_API __attribute__((visibility("default")))
#else
#define TSVD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsvd_ctx* tsvd_handle;

/* Precision tags.  working in {TSVD_FP32, TSVD_FP64}; higher in {TSVD_FP64,
 * TSVD_DD}.  TSVD_DD is a double-double (hi, lo) pair (u_h ~ 2^-104). */
typedef enum { TSVD_FP32 = 0, TSVD_FP64 = 1, TSVD_DD = 2 } tsvd_prec;

typedef enum {
    TSVD_OK = 0,
    TSVD_ERR_ARG = 1,            /* bad size, null pointer, bad tag */
    TSVD_ERR_ALIGN = 2,          /* the input must be TMA-loadable (16-byte aligned A, lda a
                                    multiple of 4): the fixed-scale and row-sharded Grams only;
                                    every other path accepts any alignment */
    TSVD_ERR_NONFINITE = 3,      /* A contains Inf or NaN */
    TSVD_ERR_NOT_FULL_RANK = 4,  /* some eigenvalue of M_h is <= 0 */
    TSVD_ERR_NO_CONVERGENCE = 5, /* Jacobi hit max_sweeps */
    TSVD_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
    TSVD_ERR_UNSUPPORTED = 7,    /* size / precision combination not built */
    TSVD_ERR_CUDA = 8,           /* a CUDA runtime call failed */
    TSVD_ERR_ALLOC = 9           /* workspace allocation failed */
} tsvd_status;

/* Options; a zero field selects the default. */
typedef struct {
    int slices;            /* Ozaki digit count k (default 7: 55 bits per entry) */
    int chunk_rows;        /* rows per exact INT chunk (default 128; must be 128) */
    int split_k;           /* CTAs over m for the Gram (default: from m and the SM count) */
    double jacobi_tol;     /* skip test |m_pq| <= tol*sqrt(m_pp m_qq) (default n * 2^-53; n * 2^-104
                              for the double-double n x n stage of FP64 working precision) */
    int max_sweeps;        /* Jacobi sweep limit (default 40) */
    int eig_variant;       /* 0 = default (2 for n <= 256, else 1); 1 = two-sided
                              Jacobi on M_h (Sec. 2.1); 2 = pivoted Cholesky of M_h
                              + one-sided Jacobi on R^T over a thread-block cluster,
                              both in FP64 (n <= 256);
                              3 = Algorithm 2 as the paper writes it: plain FP64
                              Cholesky M_h = R_h^T R_h, R = RN_32(R_h), SVD of R in
                              FP32 by one-sided Jacobi (skip threshold n 2^-24 unless
                              jacobi_tol is set); FP32 working, n <= 64; accuracy
                              O(u) kappa(B) + O(u_h) kappa(B)^2 (Remark 2) */
    int autotune;          /* 1: the first tsvd_gram / tsvd_solve of a shape (m, n, working,
                              TMA-loadable input) times the Gram with split_k = one CTA per
                              SM, half, twice and three times that, and for an FP32 U
                              (n <= 64) the tensor-core and the CUDA-core U kernel, keeps
                              the fastest for the handle's later calls of that shape
                              (tsvd_autotune_choice).  Synchronises the stream once per
                              shape; not while the stream is being captured, and not when
                              split_k, u_variant, fixed_scale or gram_variant is set.
                              Results stay within every bound stated here. */
    long long timeout_cycles; /* limit, in GPU clock cycles, of each steady-state mbarrier
                                 wait of the tcgen05 Gram kernel and of the cluster Jacobi
                                 (0 = default, 2^31, about a second); a wait that runs out
                                 makes the call report TSVD_ERR_TIMEOUT (outputs undefined).
                                 Waits for copies and MMAs already in flight before a kernel
                                 exits keep the default. */
    int gram_variant;      /* 0 = Ozaki-BF16 Gram on tcgen05/TMEM (mma.sync when the
                              input cannot be TMA-loaded; FP64 input through exact
                              23-bit pieces), 1 = plain FP64 Gram (the comparison
                              form; no double-double), 2 = Ozaki-BF16 Gram on
                              mma.sync (comparison; FP32 input only) */
    int timing;            /* k >= 1: record per-stage CUDA events of the last k calls
                              (k <= TSVD_MAX_TIMED; tsvd_last_stage_ms, tsvd_stage_ms_mean) */
    int u_variant;         /* 0 = U = A W on tcgen05 in a 3-term TF32 split when the input
                              can be TMA-loaded (FP32, n <= 64), else CUDA cores;
                              1 = CUDA-core FP32 kernel */
    int fixed_scale;       /* 1: the FP32 Gram first finds every column's exponent over the
                              whole of A (one extra read of A) and digits every entry against
                              it: the Gram is then bitwise the same for any split over CTAs
                              and any order of the rows, and equals the row-sharded Gram of
                              tsvd_gram_partial / tsvd_gram_finish.  FP32 working, n <= 64,
                              A 16-byte aligned and lda a multiple of 4 (else
                              TSVD_ERR_ALIGN).  0 (default): running per-CTA scales (one
                              read of A; bitwise reproducible run to run for a given split) */
} tsvd_opts;

/* Per-call numeric report (written asynchronously by the device). */
typedef struct {
    int status;       /* tsvd_status of the numeric part */
    int sweeps;       /* Jacobi sweeps performed (eig_variant 2 may end with one first-order step
                         in place of a last sweep, when the remaining pairs allow it; not counted) */
    double off_norm;  /* max_{p<q} |m_pq| / sqrt(m_pp m_qq) at exit */
    double kappa_B;   /* estimate of kappa(B) = (lambda_max / lambda_min)^(1/2) of the
                         column-scaled Gram C = D^-1 M_h D^-1 (A = B D, Sec. 3; the
                         kappa(B) of Theorem 1), from FP32 power and inverse
                         iterations on the pivoted Cholesky factor of C (an
                         under-estimate, typically within a few per cent); +Inf when
                         M_h is not positive definite; 0 where not computed (the
                         two-sided n x n stage, the double-double stage, batches,
                         n > 64) */
} tsvd_info;

/* Create a handle bound to `device` and `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  opts may be NULL.  Returns TSVD_ERR_ARG for a null
 * h or a bad option, TSVD_ERR_CUDA if the device cannot be selected. */
TSVD_API tsvd_status tsvd_create(tsvd_handle* h, int device, void* stream, const tsvd_opts* opts);

/* Release the handle and its workspace (synchronises its stream). */
TSVD_API tsvd_status tsvd_destroy(tsvd_handle h);

/* Human-readable name of a status code (static storage; never NULL). */
TSVD_API const char* tsvd_status_string(tsvd_status s);

/* Alg. 1 lines 1-2 (eq. (ATA)): G = A^T A in the higher precision.
 *   A: device, m x n, lda >= m, type per `working` (FP32 or FP64).
 *   G: device FP64, n x n column-major, ldg >= n, both triangles written.
 *      higher == TSVD_DD additionally writes the low parts of the
 *      double-double result at G + ldg*n (another n x n block, same ldg).
 * Built for FP32 working precision: n <= 64 in one tensor-core pass; 64 < n
 * <= 256 as one pass per pair of 32-column blocks (A 16-byte aligned and lda
 * a multiple of 4, so that the tiles can be TMA-loaded).  FP64 working
 * precision, n <= 64: each column scaled by a power of two and cut into four
 * exact 23-bit fixed-point FP32 pieces (an m x 4n FP32 copy in the handle's
 * workspace), whose block-pair Grams run on the same tensor-core kernel and
 * are summed in double-double: |G - A^T A|_ij <= 2^-88 m 2^(e_i + e_j), with
 * 2^e_j the least power of two above max_r |a_rj|.  gram_variant 1 gives the
 * plain FP64 Gram instead (no double-double form).
 * Errors: TSVD_ERR_ARG (m < 1, n < 1, lda < m, ldg < n, null pointer, bad
 * tag), TSVD_ERR_UNSUPPORTED (n > 256 or a combination not built). */
TSVD_API tsvd_status tsvd_gram(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                      tsvd_prec working, tsvd_prec higher, double* G, int64_t ldg);

/* Alg. 1 lines 3-5 on a given symmetric positive definite M_h (Sec. 2.1,
 * two-sided Jacobi in FP64; column scaling D = sqrt(diag M) drives the
 * stopping test of A = B D, Sec. 3):
 *   M: device FP64 n x n column-major (ldm >= n), read only.
 *   lambda: device FP64 [n] eigenvalues, descending.   V: device FP64 n x n
 *   (ldv >= n), sign-normalised eigenvectors.  info: optional.
 * Errors: TSVD_ERR_ARG, TSVD_ERR_UNSUPPORTED (n > 256). */
TSVD_API tsvd_status tsvd_eig(tsvd_handle h, const double* M, int64_t n, int64_t ldm, double* lambda,
                     double* V, int64_t ldv, tsvd_info* info);

/* Algorithm 1 end to end for one matrix.
 *   A: device, m x n (m >= n), lda >= m, type per `working`.
 *   sigma: device [n], working type, descending.
 *   V: device n x n working type, ldv >= n.
 *   U: device m x n working type, ldu >= m, or NULL to skip line 6.
 *   info: NULL, or device / pinned-host tsvd_info written at the end.
 * higher must be TSVD_FP64 for FP32 working.  FP64 working (n <= 64): the
 * double-double Gram of tsvd_gram, then with higher = TSVD_DD a double-double
 * pivoted Cholesky and one-sided Jacobi (Alg. 2 form, one CTA), with higher =
 * TSVD_FP64 the FP64 n x n stage on the Gram's high part; U in FP64.
 * Errors: TSVD_ERR_ARG (m < n, n < 1, lda < m, ldv < n, ldu < m with U,
 * null required pointer, bad tag), TSVD_ERR_UNSUPPORTED (n > 256, FP32 with
 * higher = TSVD_DD, FP64 with n > 64, or TSVD_DD with gram_variant 1). */
TSVD_API tsvd_status tsvd_solve(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                       tsvd_prec working, tsvd_prec higher, void* sigma, void* V, int64_t ldv,
                       void* U, int64_t ldu, tsvd_info* info);

/* Many independent instances of Alg. 1 (ragged m and n, n <= 64, FP32 working,
 * FP64 higher) in one call.  All pointer arrays (A[count], sigma[count],
 * V[count], U[count]) and size arrays (m, n, lda, ldv, ldu) are HOST arrays of
 * device pointers / sizes; U (the array) may be NULL, or any U[i] may be NULL,
 * to skip U for that instance.  info: NULL or `count` entries (device or
 * pinned host), each with that instance's status.
 * The batch runs in a fixed number of launches whatever the count: Gram work
 * items of at most 16384 rows (tensor-core Gram through per-instance tensor
 * maps when A[i] is 16-byte aligned and lda[i] % 4 == 0, else the CUDA-core
 * Ozaki kernel; gram_variant 2 forces the latter), one combine, one CTA per
 * instance for a FP64 pivoted Cholesky + one-sided Jacobi and the finish, and
 * U over all instances' row tiles.  gram_variant 1 (the plain FP64 form)
 * solves the instances one after another instead.  The handle's status
 * (tsvd_sync_status) is the most severe of the instances'.
 * Errors: TSVD_ERR_ARG for any bad instance (nothing is enqueued),
 * TSVD_ERR_UNSUPPORTED for n > 64 or another precision pair. */
TSVD_API tsvd_status tsvd_batch_solve(tsvd_handle h, int32_t count, const void* const* A, const int64_t* m,
                             const int64_t* n, const int64_t* lda, tsvd_prec working,
                             tsvd_prec higher, void* const* sigma, void* const* V,
                             const int64_t* ldv, void* const* U, const int64_t* ldu,
                             tsvd_info* info);

/* Synchronise the handle's stream and return the numeric status of the last
 * call (TSVD_OK, TSVD_ERR_NONFINITE, TSVD_ERR_NOT_FULL_RANK,
 * TSVD_ERR_NO_CONVERGENCE) or TSVD_ERR_CUDA. */
TSVD_API tsvd_status tsvd_sync_status(tsvd_handle h);

/* The autotuner's choice for a shape (opts.autotune): split_k (0 = one CTA per SM),
 * u_variant, and the measured milliseconds of the chosen Gram and U (u_ms = 0 when U was
 * not tuned); any of u_variant, gram_ms, u_ms may be NULL.  TSVD_ERR_ARG when the handle
 * has not tuned that shape. */
TSVD_API tsvd_status tsvd_autotune_choice(tsvd_handle h, int64_t m, int64_t n, tsvd_prec working, int32_t* split_k,
                                          int32_t* u_variant, float* gram_ms, float* u_ms);

/* Per-stage device times of the last tsvd_solve or tsvd_solve_gram (requires
 * opts.timing >= 1): ms[0] Gram (split + MMA + combine; 0 for tsvd_solve_gram,
 * whose caller formed G), ms[1] eigensolver (scaling, Jacobi, sort, cast),
 * ms[2] compute U, ms[3] total.  Synchronises the stream.
 * These are the components of the paper's time breakdown (Sec. 4.1.2). */
TSVD_API tsvd_status tsvd_last_stage_ms(tsvd_handle h, float ms[4]);

/* Mean per-stage device times (same layout as tsvd_last_stage_ms) over the
 * last `last` timed calls (1 <= last <= min(calls so far, opts.timing)).
 * Synchronises on the recorded events only.  TSVD_ERR_ARG otherwise. */
#define TSVD_MAX_TIMED 1024
TSVD_API tsvd_status tsvd_stage_ms_mean(tsvd_handle h, int last, float ms[4]);

/* ---- Row-sharded Gram (Sec. 4.2.1: the rows of A are distributed over the
 * processes, each computes its part of A^T A, and one global sum combines them).
 * Per rank, with A_r its block of rows (FP32, n <= 64, device pointers):
 *   1. tsvd_gram_colexp(A_r) -> E (n int32): E_j = the least e with max |a_rj| < 2^e
 *      over the rank's rows (INT32 -1048576 for an all-zero column).
 *   2. all-reduce E with MAX over the ranks (E must bound the whole column).
 *   3. tsvd_gram_partial(A_r, E) -> limbs (4 x n x n int64): the rank's part of
 *      A^T A as an exact integer in units 2^(E_i + E_j - 63), split into four
 *      32-bit limbs (value = sum_k limbs[k][i][j] 2^(32k)).
 *   4. all-reduce the limbs with SUM over the ranks (integer sums: exact in any
 *      order, no overflow for up to 2^31 ranks).
 *   5. tsvd_gram_finish(limbs, E) -> G (and its double-double low part): one
 *      rounding of the exact sum.
 *   6. tsvd_solve_gram(G, A_r) on every rank: the n x n stage (the same on every
 *      rank) and the rank's rows of U.
 * The Gram is bitwise the same for every partition of the rows over ranks and
 * CTAs and every order of the rows, and equals tsvd_gram with fixed_scale = 1 on
 * the whole A.  The accuracy is that of tsvd_gram (2^-50 (|A|^T|A|) per entry). */

/* Step 1.  A: m x n FP32 (m >= 0), lda >= max(m, 1).  E: device int32[n].
 * Errors: TSVD_ERR_ARG, TSVD_ERR_UNSUPPORTED (FP64 working or n > 64).  Inf or
 * NaN in A: TSVD_ERR_NONFINITE via tsvd_sync_status. */
TSVD_API tsvd_status tsvd_gram_colexp(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                                      tsvd_prec working, int32_t* E);

/* Step 3.  A as for step 1, 16-byte aligned with lda a multiple of 4 (else
 * TSVD_ERR_ALIGN); E: device, the column exponents over ALL ranks (an entry at
 * or above 2^E_j gives TSVD_ERR_ARG via tsvd_sync_status); limbs: device int64
 * [4][n][n] (limb k of entry (i, j) at limbs[k n^2 + i + j n]). */
TSVD_API tsvd_status tsvd_gram_partial(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                                       tsvd_prec working, const int32_t* E, int64_t* limbs);

/* Step 5.  limbs, E: device, as above (summed over the ranks).  G: device FP64
 * n x n (ldg >= n), both triangles; higher == TSVD_DD also writes the low parts
 * at G + ldg * n.  Errors: TSVD_ERR_ARG, TSVD_ERR_UNSUPPORTED (n > 64). */
TSVD_API tsvd_status tsvd_gram_finish(tsvd_handle h, const int64_t* limbs, const int32_t* E, int64_t n,
                                      tsvd_prec higher, double* G, int64_t ldg);

/* Alg. 1 lines 3-6 on a given M_h = G (device FP64 n x n, ldg >= n): the n x n
 * stage (as tsvd_solve: eig_variant, tolerances, kappa_B), sigma and V in
 * working precision, and U = A W for the given rows of A (m >= 0 rows, lda >=
 * max(m, 1); U NULL to skip).  FP32 working, FP64 higher, n <= 256.
 * Arguments and errors otherwise as tsvd_solve. */
TSVD_API tsvd_status tsvd_solve_gram(tsvd_handle h, const double* G, int64_t ldg, const void* A, int64_t m,
                                     int64_t n, int64_t lda, tsvd_prec working, tsvd_prec higher, void* sigma,
                                     void* V, int64_t ldv, void* U, int64_t ldu, tsvd_info* info);

/* The mixed precision Cholesky QR algorithm (Sec. 3.1; Theorem 3): A = Q R with
 *   1. M_h = A^T A at the higher precision (tsvd_gram's kernels),
 *   2. M_h = R^T R, the plain Cholesky factorization in FP64,
 *   3. Q from the linear systems Q R = A at the working precision: each row of Q
 *      by forward substitution in FP32 against RN_32(R).
 * With u_h = 2^-53 <= u^2, ||Q^T Q - I|| = O(u) kappa(B) (Theorem 3).
 *   A: device m x n FP32 (m >= n), lda >= m.  Q: device m x n FP32, ldq >= m,
 *   or NULL (R only).  R: device FP64 n x n upper triangular (zeros below the
 *   diagonal), ldr >= n, or NULL.  info: NULL or device / pinned-host tsvd_info.
 * FP32 working, FP64 higher, n <= 64.  Errors: TSVD_ERR_ARG, TSVD_ERR_UNSUPPORTED;
 * numeric (via info / tsvd_sync_status): TSVD_ERR_NOT_FULL_RANK at a non-positive
 * Cholesky pivot, TSVD_ERR_NONFINITE. */
TSVD_API tsvd_status tsvd_cholqr(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda, tsvd_prec working,
                                 tsvd_prec higher, void* Q, int64_t ldq, double* R, int64_t ldr, tsvd_info* info);

/* Size of the one device array that tsvd_gram_static works in (16 MiB). */
#define TSVD_GRAM_STATIC_SCRATCH_BYTES ((size_t)16 << 20)

/* The Gram matrix of tsvd_gram without any allocation.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc
 * (services that reserve all device memory up front and forbid allocation
 * on the request path, plug-ins that must not own device memory, code that
 * may not risk the implicit synchronisation of cudaMalloc / cudaFree).  It
 * needs no handle and allocates nothing: its split-K partials and status
 * block live in one fixed device array of TSVD_GRAM_STATIC_SCRATCH_BYTES
 * that every GPU which loads this part of the library holds until exit.
 *   A, m, n, lda, working, higher, G, ldg: as for tsvd_gram (working must be
 *     TSVD_FP32, n <= 64).  Input TMA can load (16-byte aligned A, lda a
 *     multiple of 4) runs the tcgen05 Gram of tsvd_gram with the same split-K
 *     plan: bitwise the result of tsvd_gram with default options.  Other
 *     input runs the mma.sync Ozaki Gram (tsvd_gram's kernel for it), whose
 *     split-K may be capped by the array: the same error bound, the bits may
 *     differ.
 *   info: NULL or a device / pinned-host tsvd_info.  There is no handle and
 *     so no tsvd_sync_status: info is the only place a data-dependent outcome
 *     (TSVD_ERR_NONFINITE for Inf or NaN in A; G is then undefined) is
 *     reported; with info NULL it is not visible.
 *   stream: a cudaStream_t (NULL = the legacy default stream); the work runs
 *     on the calling thread's current device.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it with the
 *   device's current context (a new context, e.g. after cudaDeviceReset, is
 *   looked up again); make that first call before any stream capture.
 *   Every call reuses the same array and leaves its contents behind (the
 *   status block is cleared at the start of each call); calls that overlap
 *   on the GPU, e.g. on two streams at once, race on it.
 * Errors: TSVD_ERR_ARG as tsvd_gram; TSVD_ERR_UNSUPPORTED when the partials
 * would not fit the array, i.e. m > 32768 * floor((16 MiB - 512) /
 * (16 NP^2 + 4 NP)) with NP = 64 for TMA-loadable input and NP = n rounded
 * up to 16, 32, 48 or 64 otherwise (m > 8,323,072 at NP = 64), or for FP64
 * working / n > 64; TSVD_ERR_CUDA if the runtime fails. */
TSVD_API tsvd_status tsvd_gram_static(const void* A, int64_t m, int64_t n, int64_t lda,
                                      tsvd_prec working, tsvd_prec higher, double* G, int64_t ldg,
                                      tsvd_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TSVD_H */
