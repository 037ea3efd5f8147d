// internal.cuh -- declarations shared by the CUDA translation units of libtsvd.
// (Nothing here is shared with the CPU oracle.)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsvd.h"

namespace tsvd {

// Device-side report; layout identical to tsvd_info so it can be copied out.
struct DevInfo {
    int flags;        // FLAG_* bits, turned into a tsvd_status by finalize_info
    int sweeps;
    double off_norm;
    double kappa;
};
static_assert(sizeof(DevInfo) == sizeof(tsvd_info), "DevInfo must mirror tsvd_info");

enum : int {
    FLAG_NONFINITE = 1,
    FLAG_NOT_FULL_RANK = 2,
    FLAG_NO_CONVERGENCE = 4,
    FLAG_TIMEOUT = 8,
    FLAG_BAD_SCALE = 16,  // a given column exponent does not bound its column
};

// Limit, in GPU clock cycles, of the steady-state bounded waits of the
// pipelined kernels for a tsvd_opts.timeout_cycles value (0 = the default,
// about a second of GPU clock).  Waits that drain copies and MMAs already in
// flight before a kernel exits keep the default whatever the option.
constexpr long long WAIT_CYCLES_DEFAULT = 1ll << 31;
inline long long wait_limit_of(long long opt) { return opt > 0 ? opt : WAIT_CYCLES_DEFAULT; }

// A second stream and two events of a handle: small independent kernels fork
// off the main stream and join it again (capturable in a CUDA graph).
struct EigSide {
    cudaStream_t stream;
    cudaEvent_t fork, join;
};

// Exact 128-bit integer helpers of the Gram combines (device only).
__device__ __forceinline__ int msb_u128(unsigned __int128 v) {
    const unsigned long long hi = (unsigned long long)(v >> 64);
    if (hi) return 127 - __clzll((long long)hi);
    return 63 - __clzll((long long)(unsigned long long)v);
}

// Round v * 2^scale to the nearest double (ties to even); rounded_int gets
// the exact integer value of the result in units of 2^scale.
__device__ __forceinline__ double round_i128(__int128 v, int scale, __int128& rounded_int) {
    if (v == 0) { rounded_int = 0; return 0.0; }
    const bool neg = v < 0;
    unsigned __int128 mag = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const int msb = msb_u128(mag);
    unsigned long long mant;
    int sh = 0;
    if (msb <= 52) {
        mant = (unsigned long long)mag;
    } else {
        sh = msb - 52;
        mant = (unsigned long long)(mag >> sh);
        const unsigned __int128 rem = mag - ((unsigned __int128)mant << sh);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) ++mant;  // mant may become 2^53: still exact
    }
    const __int128 r = (__int128)((unsigned __int128)mant << sh);
    rounded_int = neg ? -r : r;
    const double d = ldexp((double)mant, sh + scale);
    return neg ? -d : d;
}

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)h2 << 64) | (unsigned __int128)l2);
}


// Sentinel exponent of an all-zero column (no digits, nothing accumulated).
constexpr int EXP_EMPTY = -(1 << 20);

// ---------------------------------------------------------------- Gram (Alg. 1 l.1-2)
// Ozaki split into k = 7 signed digits (|q| <= 128, exact in bf16) relative
// to a running per-column power-of-two scale; every digit-pair block is an
// exact integer sum over a 128-row chunk (BF16 MMA, FP32 accumulate, all
// partial sums below 2^22) folded into two int64 fixed-point accumulators.
constexpr int GRAM_KC = 128;           // rows per exact chunk
constexpr int GRAM_DIGITS = 7;         // k
constexpr int GRAM_MAX_ROWS_PER_CTA = 32768;  // keeps the int64 accumulators in range

struct GramPlan {
    int NP;            // padded n (16, 32, 48 or 64)
    int P;             // CTAs over m (split-K)
    int64_t rows_per_cta;
    long long wait_cycles = 0;  // limit of the tensor-core Gram's steady-state waits (0 = default)
    const int* E_fixed = nullptr;  // tensor-core Gram: fixed column exponents (device, 64 ints) or null
};
GramPlan gram_plan(int64_t m, int n, int sm_count, int split_k_opt);
size_t gram_partials_bytes(const GramPlan& p);

// part: workspace of gram_partials_bytes(plan) bytes.
cudaError_t launch_gram_ozaki(const void* A, int working, int64_t m, int n, int64_t lda,
                              const GramPlan& plan, void* part, DevInfo* info, cudaStream_t s);
// tcgen05 / TMEM / TMA version of the same Gram (FP32, n <= 64, 16-byte
// aligned columns).  Writes partials in the layout of launch_gram_ozaki with
// NP = 64; plan from gram_tc_plan.
bool gram_tc_ok(const void* A, int working, int n, int64_t lda);
GramPlan gram_tc_plan(int64_t m, int n, int sm_count, int split_k_opt);
// Two 32-column groups (c1, c2) of a wider A as the 64 virtual columns (n > 64).
cudaError_t launch_gram_tc2(const void* A, int64_t m, int n, int64_t lda, int c1, int c2, const GramPlan& plan,
                            void* part, DevInfo* info, cudaStream_t s);
cudaError_t launch_gram_tc(const void* A, int64_t m, int n, int64_t lda, const GramPlan& plan, void* part,
                           DevInfo* info, cudaStream_t s);
// Row-partitioned Gram (gram_sharded.cu).  launch_colexp: E[j] = the least e with
// max_r |a_rj| < 2^e (EXP_EMPTY for a zero column; FP32, n <= 64; colmax_ws: n
// unsigned).  With plan.E_fixed = E the tensor-core Gram's partials are exact
// integers in units 2^(E_i + E_j - 63); launch_gram_limbs sums them exactly into
// four 32-bit limbs per entry (limbs: 4 n x n int64), launch_gram_finish rounds a
// (possibly rank-summed) limb array to G (and G_lo).
cudaError_t launch_colexp(const float* A, int64_t m, int n, int64_t lda, unsigned* colmax_ws, int* E, DevInfo* info,
                          int sm_count, cudaStream_t s);
cudaError_t launch_gram_limbs(const GramPlan& plan, const void* part, int n, const int* E, long long* limbs,
                              cudaStream_t s);
cudaError_t launch_gram_finish(const long long* limbs, int n, const int* E, double* G, double* G_lo, int64_t ldg,
                               cudaStream_t s);

// Combine the partials into G (n x n FP64, both triangles) and optionally the
// double-double low parts G_lo (may be null).
cudaError_t launch_gram_combine(const GramPlan& plan, const void* part, int n, double* G,
                                double* G_lo, int64_t ldg, cudaStream_t s);
// The 64 x 64 partials of a two-group launch into G: local column l maps to
// (l < 32 ? c1 + l : c2 + l - 32) (dropped when >= n); wmask bit 0 writes the
// first group's diagonal tile, bit 1 the second's, bit 2 the cross tile.
cudaError_t launch_gram_combine2(const GramPlan& plan, const void* part, int n, int c1, int c2, int wmask, double* G,
                                 double* G_lo, int64_t ldg, cudaStream_t s);

// Plain all-FP64 Gram (the comparison form): DFMA over m, fixed-order combine.
size_t gram_plain_partials_bytes(int64_t m, int n, int sm_count);
cudaError_t launch_gram_plain(const void* A, int working, int64_t m, int n, int64_t lda,
                              int sm_count, void* part, double* G, int64_t ldg, DevInfo* info,
                              cudaStream_t s);

// Double-double Gram of an FP64 A (working FP64): exact 23-bit fixed-point
// pieces (four per entry, column-scaled by powers of two) into an m x 4NB FP32
// matrix in `extra` (fp64_extra_bytes), whose 32-column block pairs
// (fp64_pair_needed) go through the tensor-core Gram into the 4NB x 4NB
// double-double G3 (fp64_g3); launch_fp64_fold sums the pieces into G, G_lo.
int fp64_block_cols(int n);
int64_t fp64_split_ld(int64_t m);
size_t fp64_extra_bytes(int64_t m, int n);
bool fp64_pair_needed(int n, int b1, int b2);
const float* fp64_split_matrix(const void* extra);
double* fp64_g3(void* extra, int64_t m, int n, double** g3lo);
cudaError_t launch_fp64_split(const double* A, int64_t m, int n, int64_t lda, void* extra, DevInfo* info,
                              cudaStream_t s);
cudaError_t launch_fp64_fold(void* extra, int64_t m, int n, double* G, double* G_lo, int64_t ldg, cudaStream_t s);

// ---------------------------------------------------------------- eigen stage (Alg. 1 l.3-5)
// Two-sided Jacobi in FP64 on M (n x n, read from M/ldm), one CTA.
// scratch: 2*n*n doubles (used when n > 64).  Writes unsorted lambda and V
// (n x n, ld n) into lam_ws / V_ws.
cudaError_t launch_jacobi(const double* M, int n, int64_t ldm, double tol, int max_sweeps,
                          double* scratch, double* lam_ws, double* V_ws, DevInfo* info,
                          cudaStream_t s);

// Preconditioned one-sided Jacobi in FP64 (pivoted Cholesky, then one-sided
// Jacobi on R^T over a thread-block cluster), n <= 64.  scratch: at least
// n*n doubles + 256 ints.  Writes unsorted lambda and V like launch_jacobi,
// and the kappa(B) estimate into info->kappa (on side->stream when given,
// joined back into s before returning).  wait_cycles: tsvd_opts.timeout_cycles.
cudaError_t launch_eig_onesided(const double* M, int n, int64_t ldm, double tol, int max_sweeps,
                                void* scratch, double* lam_ws, double* V_ws, DevInfo* info,
                                cudaStream_t s, const EigSide* side = nullptr, long long wait_cycles = 0);

// Cholesky of M (FP64, one CTA) into X = R^T (n x n, ld n, rows in pivot order) and
// perm (position -> original index); pivot = false is the plain factorization (perm =
// identity).  A non-positive pivot flags rank deficiency.  n <= 64 in shared memory;
// 64 < n <= 256 needs gm_scratch (2 n^2 doubles) for the Schur complement and R.
cudaError_t launch_cholesky(const double* M, int n, int64_t ldm, double* X, int* perm, DevInfo* info, bool pivot,
                            cudaStream_t s, double* gm_scratch = nullptr);

// Algorithm 2 (n <= 64): the plain FP64 Cholesky M = R^T R, R cast to FP32, and
// the SVD of that R by a one-CTA one-sided Jacobi in FP32 (tol: the scaled skip
// threshold, e.g. n 2^-24).  Writes unsorted lambda = sigma^2 and V (FP64 copies
// of the FP32 results) like launch_jacobi.  scratch as launch_eig_onesided.
cudaError_t launch_eig_alg2(const double* M, int n, int64_t ldm, float tol, int max_sweeps, void* scratch,
                            double* lam_ws, double* V_ws, DevInfo* info, cudaStream_t s);

// Cholesky QR, step 3 (cholqr.cu): Q from Q R = A by FP32 forward substitution per row
// against RN_32(R), X = R^T (FP64, ld n, plain Cholesky); also R into the caller's
// R (FP64, ldr; skipped when null).  FP32, n <= 64.
cudaError_t launch_cholqr_q(const float* A, int64_t m, int n, int64_t lda, const double* X, float* Q, int64_t ldq,
                            double* R, int64_t ldr, int sm_count, cudaStream_t s);

// Double-double eigen stage for FP64 working (n <= 64, one CTA): pivoted
// Cholesky of M = G + G_lo in double-double, then a one-sided Jacobi SVD of
// R^T in double-double.  scratch: unused.  Writes unsorted lambda (rounded to
// FP64) and V like launch_jacobi.
cudaError_t launch_eig_dd(const double* M, const double* M_lo, int n, int64_t ldm, double tol, int max_sweeps,
                          double* lam_ws, double* V_ws, DevInfo* info, cudaStream_t s);

// Eigensolver variants (tsvd_opts.eig_variant).
enum : int { EIG_DEFAULT = 0, EIG_TWO_SIDED = 1, EIG_ONE_SIDED = 2, EIG_ALG2 = 3 };

// Sort descending, sign rule, sigma = sqrt(lambda), round to working.
// working: 0 FP32, 1 FP64.  Outputs (any may be null):
//   sigma_w [n], V_w (ldv), W_w = RN(V_w / sigma_w) (ld n) in working type;
//   lam_sorted [n], V_sorted (ld_vs) in FP64.  sigma_n < uh sigma_1 flags rank deficiency.
cudaError_t launch_finish(const double* lam_ws, const double* V_ws, int n, int working,
                          void* sigma_w, void* V_w, int64_t ldv, void* W_w, double* lam_sorted,
                          double* V_sorted, int64_t ld_vs, DevInfo* info, cudaStream_t s,
                          double uh = 1.1102230246251565e-16);

// ---------------------------------------------------------------- U (Alg. 1 l.6)
cudaError_t launch_compute_u(const void* A, int working, int64_t m, int n, int64_t lda,
                             const void* W, void* U, int64_t ldu, cudaStream_t s);
// Streaming FP32 U kernel (bulk-copy pipeline, packed FMA); requires
// compute_u_v2_ok(): FP32, n <= 64, 16-byte aligned columns, m % 4 == 0.
bool compute_u_v2_ok(const void* A, int working, int64_t m, int n, int64_t lda, const void* U, int64_t ldu);
// tcgen05 U (3-term TF32 split): FP32, n <= 64, TMA-loadable A.
bool compute_u_tc_ok(const void* A, int working, int64_t m, int n, int64_t lda);
cudaError_t launch_compute_u_tc(const float* A, int64_t m, int n, int64_t lda, const float* W, float* U,
                                int64_t ldu, int sm_count, DevInfo* info, cudaStream_t s);
cudaError_t launch_compute_u_v2(const float* A, int64_t m, int n, int64_t lda, const float* W, float* U,
                                int64_t ldu, int sm_count, DevInfo* info, cudaStream_t s);

// ---------------------------------------------------------------- batched instances (n <= 64, FP32)
// One descriptor per instance, in device memory.  Workspace pointers (G, lam,
// Vh, W) are the instance's own; sigma, V, U are the caller's (U may be null).
constexpr size_t BATCH_SLOT = 64 * 64;  // int64 entries per Gram partial slot (hi or lo)
constexpr int BATCH_ROWS = 16384;       // rows per Gram work item (a multiple of GRAM_KC)
// rows per U work item: 256 threads x 4 rows, spread over ceil(n / 16) column groups
__host__ __device__ inline int batch_u_rows(int n) { return n <= 16 ? 1024 : n <= 32 ? 512 : 256; }
struct BatchInst {
    const float* A;
    int64_t m, lda;
    int n, NP;
    int slot0, nslots;  // Gram partial slots of this instance
    int halves;         // 2: each slot holds two diagonal 32 x 32 tiles to add (packed rows)
    double* G;          // n x n, ld n
    double* lam;        // n
    double* Vh;         // n x n, ld n
    float* W;           // n x n, ld n
    float* sigma;
    float* V;
    int64_t ldv;
    float* U;
    int64_t ldu;
    int64_t utile0;     // first U work item of this instance (prefix over instances)
};
struct BatchGramItem {
    int inst, slot;
    int64_t r0, r1;
};
// Tensor-core items: one CTA streams rows [r0, r1) (r0 a multiple of 64, at most
// 2^15 rows) of one instance through its tensor map (tc_tmap_bytes() bytes,
// 64-byte aligned, in device memory; made by make_tc_batch_tmap on the host).
// With tmap2 (n <= 32; tmap and tmap2 map rows 0.. and 64.. of the instance with
// 32-column boxes) the CTA takes two 64-row blocks per step as the two column
// groups, and the instance's partial is the sum of the two diagonal tiles.
struct TcBatchItem {
    const void* tmap;
    const void* tmap2;
    int64_t r0, r1;
    int n, slot, inst, pad;
};
bool gram_tc_batch_ok(const void* A, int64_t lda);
size_t tc_tmap_bytes();
cudaError_t make_tc_batch_tmap(void* map, const float* A, int64_t m, int n, int64_t lda, int box_cols);
cudaError_t launch_gram_tc_batch(const TcBatchItem* items, int nitems, void* part, int total_slots, DevInfo* infos,
                                 cudaStream_t s, long long wait_cycles = 0);
size_t gram_batch_partials_bytes(int total_slots);
// One launch for the items of one padded width NP (16, 32, 48 or 64).
cudaError_t launch_gram_batch(const BatchInst* inst, const BatchGramItem* items, int nitems, int NP, bool vec,
                              void* part, int total_slots, DevInfo* infos, int grid, cudaStream_t s);
cudaError_t launch_gram_combine_batch(const BatchInst* inst, int count, const void* part, int total_slots,
                                      cudaStream_t s);
// One CTA per instance: FP64 pivoted Cholesky + one-sided Jacobi, then sort /
// sign / sigma / W; U over all instances' row tiles (utile total); statuses
// into infos[i] and, ORed, into agg (then finalised).
cudaError_t launch_eig_batch(const BatchInst* inst, int count, double tol, int max_sweeps, DevInfo* infos,
                             cudaStream_t s);
cudaError_t launch_finish_batch(const BatchInst* inst, int count, DevInfo* infos, cudaStream_t s);
cudaError_t launch_u_batch(const BatchInst* inst, int count, int64_t utiles, int grid, cudaStream_t s);
cudaError_t launch_finalize_batch(DevInfo* infos, int count, DevInfo* agg, cudaStream_t s);

// flags -> tsvd_status in info->flags (overwritten by the status code).
cudaError_t launch_finalize_info(DevInfo* info, cudaStream_t s);

}  // namespace tsvd
