// eig_onesided.cu -- the n x n eigen stage by a preconditioned one-sided
// Jacobi in FP64 (Alg. 1 line 3 with the one-sided Jacobi SVD option of
// Sec. 2.1; the factor-then-SVD structure of Algorithm 2, here entirely in
// the higher precision).
//
//   1. Pivoted Cholesky of M_h in FP64: P M_h P^T = R^T R, the pivot being
//      the largest remaining diagonal entry (scale-invariant, so the
//      grading D of A = B D costs no accuracy).  A non-positive pivot marks
//      rank deficiency (TSVD_ERR_NOT_FULL_RANK).
//   2. One-sided Jacobi on X = R^T: X <- X J over column pairs until every
//      pair satisfies |x_p^T x_q| <= tol ||x_p|| ||x_q|| (the scaled test).
//      Then X X^T = P M_h P^T is unchanged and the columns of X are
//      orthogonal, so lambda_j = ||x_j||^2 and the eigenvectors of M_h are
//      v_j = P^T x_j / ||x_j||.  The rotation of a pair is the two-sided
//      Jacobi rotation of its 2 x 2 Gram [||x_p||^2, g; g, ||x_q||^2]
//      (Rutishauser's formulas), so this is two-sided Jacobi on X^T X
//      without forming it and without accumulating V.
//   3. The pairs are scheduled by the round-robin ("circle") tournament over
//      a thread-block cluster.
//
// GB300 sets the shape of step 3.  Its FP64 pipe takes one instruction of a
// warp per ~64 cycles (independent or not, whatever the number of active
// lanes) and about one per 19 cycles from a whole SM; FP32 is ~60x faster.
// So (i) the pairs are spread over the 16 SMs of a (non-portable) cluster,
// two per SM, two warps per pair (one row per lane), and a warp issues only
// the FP64 instructions that carry the result: 1 for its part of x_p^T x_q,
// 1 for the norm difference, 4 for the rotation of its rows, and either the 6
// of the orthogonality correction or the 3 of the norm updates; (ii) the
// reduction of the dot product (exact 64-bit fixed point), the angle and the
// scaled test (FP32) run on the integer and FP32 pipes; (iii) a column that
// leaves an SM is written straight from registers into the neighbour's shared
// memory by st.async, into a ring of receive buffers whose slot of every
// column follows from the step count in closed form, each store completing a
// transaction on the neighbour's mbarrier: no copy, no fence, no shared map
// and no cluster-wide barrier within a sweep.
//
// The rotation angle and (c0, s0) are computed in FP32 while the applied
// rotation is made orthogonal to FP64 precision by one correction factor:
// an inexact angle only leaves a residual g * O(2^-24) on a pair,
// which later sweeps remove, whereas a non-orthogonal rotation would change
// the singular values.  Squared norms are updated within a sweep by the exact
// quadratic form of the rotation, recomputed at the start of every sweep and
// whenever a norm drops below 1/16 of its previous value; the stopping test
// of the final, rotation-free sweep therefore uses exact norms.
//
// kappa_kernel estimates kappa(B) = kappa(C)^(1/2), C = D^-1 M_h D^-1 (the
// column-scaled Gram of A = B D), from the Cholesky factor: the rows of X
// scaled by 1/d form a Cholesky factor L of P C P^T, and FP32 power and
// inverse iterations on L L^T give its extreme eigenvalues.  It runs on a
// second stream beside the Jacobi.
#include <climits>

#include <cooperative_groups.h>

#include "internal.cuh"
#include "tma_util.cuh"

namespace cg = cooperative_groups;

namespace tsvd {
namespace {

// ---------------------------------------------------------------- pivoted Cholesky
// One CTA.  M (n x n, ldm) -> X = R^T (n x n, ld n, lower triangular, rows in pivot
// order) and perm (pivot position -> original index).  The trailing Schur complement
// is kept by original index and only its lower triangle (row index >= column index,
// original order) is stored and updated: half the FP64 work of a full update, and no
// rows or columns are swapped.  The remaining indices are a bit mask; their ascending
// list turns the triangle into contiguous work for the warps.  pivot = 0 takes the
// lowest remaining index instead (the plain Cholesky factorization M_h = R_h^T R_h that
// Algorithm 2 names); it fails, like the pivoted one, at a non-positive diagonal.
__device__ __forceinline__ double chol_S(const double* sa, int n, int x, int y) {
    return x >= y ? sa[x + (size_t)y * n] : sa[y + (size_t)x * n];
}
// Conversions by integer bit operations (the FP64 pipe is the scarce resource):
// double -> float truncates the significand and flushes values outside the normal
// float range to 0 / +-max (only angles and heuristics use it); float -> double is
// exact for normal floats and gives 0 for subnormal ones.
__device__ __forceinline__ float os_to_float(double x) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned sgn = (unsigned)((unsigned long long)b >> 63) << 31;
    if (ex < -126) return __uint_as_float(sgn);
    if (ex > 127) return __uint_as_float(sgn | 0x7f7fffffu);
    return __uint_as_float(sgn | ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff));
}
__device__ __forceinline__ double os_to_double(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned ex = (b >> 23) & 0xff;
    if (ex == 0) return 0.0;
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(ex + 896) << 52) |
                                 ((unsigned long long)(b & 0x7fffff) << 29);
    return __longlong_as_double((long long)d);
}
// 1 / sqrt(d) for a positive normal d: d = dm 4^k with dm in [1, 4) by an exponent shift,
// y0 = rsqrtf(dm) (FP32), one Newton step with its second-order term in FP64,
// y = y0 (1 + e/2 + 3e^2/8) with e = 1 - dm y0^2 (|e| ~ 2^-23, error O(e^3)), then 2^-k.
__device__ __forceinline__ double chol_rsqrt(double d) {
    const long long b = __double_as_longlong(d);
    const int k = (int)(((b >> 52) & 0x7ff) - 1023) >> 1;  // floor(exponent / 2)
    const double dm = __longlong_as_double(b - ((long long)(2 * k) << 52));
    const double y0 = os_to_double(rsqrtf(os_to_float(dm)));  // dm in [1, 4): both conversions exact-range
    const double e = fma(-dm * y0, y0, 1.0);
    const double y = y0 * fma(e, fma(e, 0.375, 0.5), 1.0);
    return __longlong_as_double(__double_as_longlong(y) - ((long long)k << 52));
}

// n <= 64: one CTA of 16 warps with a look-ahead.  Warp 0 (the panel) runs the dependent
// chain of each step one step ahead of the others: 1 / r_kk, row k of R from the pivot
// column, the remaining diagonal D -= R_k^2, the next pivot, and that pivot's column brought
// up to date (the other warps' update of the previous step has been applied to S; this
// step's term the panel subtracts itself), and only then publishes row k.  Warps 1-15 apply
// each published step's update S(a, b) -= R_k[a] R_k[b] to the strictly lower triangle of the
// remaining indices, one entry per thread (a flat index table spreads the triangle evenly).
// The two sides meet on mbarriers (row k published; every bulk warp done with step k), waited
// on with a suspend-time hint and a bound.  Every value is computed by the same operations as
// in a plain right-looking factorization.
constexpr int CHL_THREADS = 512, CHL_BULK_WARPS = CHL_THREADS / 32 - 1;

// pivot: the largest remaining diagonal, lowest original index on ties (keys: 0 for a
// negative value, else the bit pattern's high word + 1 and its low word; non-negative doubles
// order like their patterns), or the lowest remaining index without pivoting.  Whole warp.
__device__ __forceinline__ int chol_pick(const double* D, int n, unsigned long long rem, int pivot, int lane) {
    if (!pivot) return __ffsll((long long)rem) - 1;
    unsigned khi = 0u, klo = 0u;
    int bo = n;
    for (int o = lane; o < n; o += 32) {
        if (!((rem >> o) & 1ull)) continue;
        const long long dd = __double_as_longlong(D[o]);
        const unsigned h = dd < 0 ? 0u : (unsigned)(dd >> 32) + 1u, l = dd < 0 ? 0u : (unsigned)dd;
        if (bo == n || h > khi || (h == khi && l > klo)) { khi = h; klo = l; bo = o; }
    }
    const unsigned mh = __reduce_max_sync(0xffffffffu, khi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, khi == mh ? klo : 0u);
    return (int)__reduce_min_sync(0xffffffffu, (khi == mh && klo == ml) ? (unsigned)bo : (unsigned)n);
}

__global__ void __launch_bounds__(CHL_THREADS, 1)
    chol_piv_kernel(const double* __restrict__ M, int n, int64_t ldm, double* __restrict__ X,
                    int* __restrict__ perm_out, DevInfo* info, int pivot) {
    extern __shared__ double sa[];    // [n][n] Schur complement, strictly lower triangle by original index
    double* Rr = sa + (size_t)n * n;  // [n][n]: row k of R by original column index
    __shared__ double s_D[64];        // diagonal of the Schur complement (the panel's)
    __shared__ double s_pcol[64];     // the current pivot's column, up to date
    __shared__ unsigned short s_tab[2016];  // flat index ia (ia - 1) / 2 + jb -> ia | jb << 8
    __shared__ int s_list[2][64];     // per step (mod 2): remaining indices without its pivot, ascending
    __shared__ int s_rc[2];
    __shared__ int s_perm[64];
    __shared__ uint64_t s_rowbar[2];  // per step (mod 2): row k of R published (one arrival)
    __shared__ uint64_t s_bulkbar[2]; // per step (mod 2): every bulk warp applied step k
    __shared__ int s_stop;            // the panel is done (or gave up); steps >= s_kend are not rows
    __shared__ int s_kend;
    __shared__ unsigned long long s_rem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int idx = tid; idx < n * n; idx += CHL_THREADS) {
        const int r = idx % n, c = idx / n;
        sa[idx] = r >= c ? M[r + (size_t)c * ldm] : 0.0;
        Rr[idx] = 0.0;
    }
    for (int t = tid; t < 2016; t += CHL_THREADS) {
        int ia = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
        while (ia * (ia - 1) / 2 > t) --ia;
        while ((ia + 1) * ia / 2 <= t) ++ia;
        s_tab[t] = (unsigned short)(ia | ((t - ia * (ia - 1) / 2) << 8));
    }
    if (tid < n) s_D[tid] = M[tid + (size_t)tid * ldm];
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) { mbar_init(&s_rowbar[i], 1); mbar_init(&s_bulkbar[i], CHL_BULK_WARPS); }
        mbar_fence_init();
        s_stop = 0;
        s_kend = n;
    }
    __syncthreads();
    if (warp == 0) {
        // ---------------- panel
        unsigned long long rem = n == 64 ? ~0ull : ((1ull << n) - 1ull);
        int ok = chol_pick(s_D, n, rem, pivot, lane);
        for (int o = lane; o < n; o += 32) s_pcol[o] = chol_S(sa, n, o, ok);
        __syncwarp();
        bool deficient = false, timeout = false;
        int k = 0;
        while (k < n) {
            // d > 0 (finite) decided on the bit pattern
            const double d = s_D[ok];
            const long long db = __double_as_longlong(d);
            if (!(db > 0 && db < 0x7ff0000000000000ll)) { deficient = true; break; }
            const unsigned long long rn = rem & ~(1ull << ok);
            const double rinv = chol_rsqrt(d);
            double* rk = Rr + (size_t)k * n;
            for (int o = lane; o < n; o += 32) {
                if (o == ok) rk[o] = d * rinv;
                else if ((rn >> o) & 1ull) {
                    const double r = s_pcol[o] * rinv;
                    rk[o] = r;
                    s_D[o] = fma(-r, r, s_D[o]);
                    s_list[k & 1][__popcll(rn & ((1ull << o) - 1ull))] = o;
                }
            }
            if (lane == 0) { s_perm[k] = ok; s_rc[k & 1] = __popcll(rn); }
            rem = rn;
            __syncwarp();
            int nok = -1;
            if (rem != 0ull) {
                nok = chol_pick(s_D, n, rem, pivot, lane);
                // the next pivot's column: in S once the bulk warps finished step k - 1, minus
                // this step's term (S itself gets it from them after row k is published)
                if (k >= 1 && !mbar_wait_susp(&s_bulkbar[(k - 1) & 1], ((k - 1) >> 1) & 1)) timeout = true;
                const double rkn = rk[nok];
                for (int o = lane; o < n; o += 32)
                    if (((rem >> o) & 1ull) && o != nok) s_pcol[o] = fma(-rk[o], rkn, chol_S(sa, n, o, nok));
            }
            // publish row k, its list and count
            __threadfence_block();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_rowbar[k & 1]);
            ++k;
            if (timeout || rem == 0ull) break;
            ok = nok;
        }
        if (lane == 0) {
            s_kend = k;
            s_rem = rem;
            if (deficient) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
            if (timeout) atomicOr(&info->flags, FLAG_TIMEOUT);
            *reinterpret_cast<volatile int*>(&s_stop) = 1;
            __threadfence_block();
            mbar_arrive(&s_rowbar[k & 1]);  // wakes the bulk warps waiting for step k: none follows
        }
    } else {
        // ---------------- bulk: the update of every published step
        const int btid = tid - 32;
        for (int k = 0;; ++k) {
            if (!mbar_wait_susp(&s_rowbar[k & 1], (k >> 1) & 1)) {
                if (lane == 0) atomicOr(&info->flags, FLAG_TIMEOUT);
                break;
            }
            if (*reinterpret_cast<volatile int*>(&s_stop) && k >= *reinterpret_cast<volatile int*>(&s_kend)) break;
            const int rc = s_rc[k & 1];
            const int* list = s_list[k & 1];
            const double* rk = Rr + (size_t)k * n;
            const int T = rc * (rc - 1) / 2;
            for (int t = btid; t < T; t += CHL_THREADS - 32) {
                const unsigned e = s_tab[t];
                const int a = list[e & 0xffu], b = list[e >> 8];
                double* sp = sa + a + (size_t)b * n;
                *sp = fma(-rk[a], rk[b], *sp);
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_bulkbar[k & 1]);
        }
    }
    __syncthreads();
    // X = R^T with rows in pivot order: X[pos][c] = R[c][perm[pos]] for pos >= c.  Past a
    // rank deficiency the remaining positions take the remaining indices in ascending order.
    const int kend = s_kend;
    if (tid == 0) {
        const unsigned long long rem = s_rem;
        int pos = kend;
        for (int o = 0; o < n; ++o)
            if ((rem >> o) & 1ull) s_perm[pos++] = o;
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += CHL_THREADS) {
        const int pos = idx % n, c = idx / n;
        X[idx] = (pos >= c && c < kend) ? Rr[(size_t)c * n + s_perm[pos]] : 0.0;
    }
    for (int i = tid; i < n; i += CHL_THREADS) perm_out[i] = s_perm[i];
}

// 64 < n <= 256: the same factorization with the Schur complement S (lower triangle by original
// index) and the rows of R in global scratch (2 n^2 doubles, L2-resident), one CTA of 1024
// threads.  Thread o < n owns index o for the pivot search and the ascending list of the
// remaining indices, which a ballot per warp and the warps' counts build without a serial pass.
__global__ void __launch_bounds__(1024, 1)
    chol_piv_gm_kernel(const double* __restrict__ M, int n, int64_t ldm, double* __restrict__ S,
                       double* __restrict__ Rr, double* __restrict__ X, int* __restrict__ perm_out, DevInfo* info,
                       int pivot) {
    __shared__ int s_list[256];
    __shared__ int s_perm[256];
    __shared__ unsigned char s_rem[256];
    __shared__ long long s_key[32];
    __shared__ int s_idx[32];
    __shared__ int s_cnt[8];
    __shared__ int s_ok;
    __shared__ double s_rinv;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int idx = tid; idx < n * n; idx += nt) {
        const int r = idx % n, c = idx / n;
        S[idx] = r >= c ? M[r + (size_t)c * ldm] : 0.0;
        Rr[idx] = 0.0;
    }
    for (int i = tid; i < 256; i += nt) s_rem[i] = i < n ? 1 : 0;
    __syncthreads();
    bool deficient = false;
    int kend = n;
    for (int k = 0; k < n; ++k) {
        // pivot: the largest remaining diagonal, lowest original index on ties (non-negative doubles
        // order like their bit patterns; every negative value sorts below them); without
        // pivoting the remaining indices are k..n-1 in order
        if (pivot) {
            long long key = LLONG_MIN;
            int bo = n;
            if (tid < n && s_rem[tid]) {
                const long long dd = __double_as_longlong(S[tid + (size_t)tid * n]);
                key = dd < 0 ? LLONG_MIN + 1 : dd;
                bo = tid;
            }
            for (int off = 16; off > 0; off >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, key, off);
                const int oo = __shfl_xor_sync(0xffffffffu, bo, off);
                if (ob > key || (ob == key && oo < bo)) { key = ob; bo = oo; }
            }
            if (lane == 0) { s_key[warp] = key; s_idx[warp] = bo; }
            __syncthreads();
            if (warp == 0) {
                key = lane < nw ? s_key[lane] : LLONG_MIN;
                bo = lane < nw ? s_idx[lane] : n;
                for (int off = 16; off > 0; off >>= 1) {
                    const long long ob = __shfl_xor_sync(0xffffffffu, key, off);
                    const int oo = __shfl_xor_sync(0xffffffffu, bo, off);
                    if (ob > key || (ob == key && oo < bo)) { key = ob; bo = oo; }
                }
                if (lane == 0) s_ok = bo;
            }
            __syncthreads();
        }
        const int ok = pivot ? s_ok : k;
        const double d = S[ok + (size_t)ok * n];
        // d > 0 (finite) decided on the bit pattern, and 1 / r_kk only by the warps that use it
        // (the SM's FP64 pipe is shared by all 32 warps)
        const long long db = __double_as_longlong(d);
        if (!(db > 0 && db < 0x7ff0000000000000ll)) { deficient = true; kend = k; break; }
        // 1 / r_kk by one thread, the row k of R over the remaining indices and their ascending
        // list (without ok) after the barrier
        if (tid == 0) s_rinv = chol_rsqrt(d);
        const bool keep = tid < n && s_rem[tid] && tid != ok;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0 && warp < 8) s_cnt[warp] = __popc(bal);
        __syncthreads();
        if (tid < n) {
            const double rinv = s_rinv;
            if (tid == ok) Rr[(size_t)k * n + tid] = d * rinv;
            else if (keep) Rr[(size_t)k * n + tid] = chol_S(S, n, tid, ok) * rinv;
        }
        if (keep) {
            int pos = __popc(bal & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) pos += s_cnt[w];
            s_list[pos] = tid;
        }
        if (tid == 0) { s_perm[k] = ok; s_rem[ok] = 0; }
        __syncthreads();
        // trailing update S(a, b) -= R[k][a] R[k][b] over the remaining lower triangle: the warps
        // take its columns b (round robin), the lanes its rows a >= b
        const int rc = n - 1 - k;
        const double* rk = Rr + (size_t)k * n;
        for (int jb = warp; jb < rc; jb += nw) {
            const int b = s_list[jb];
            const double rb = rk[b];
            for (int ia = jb + lane; ia < rc; ia += 32) {
                const int a = s_list[ia];
                S[a + (size_t)b * n] -= rk[a] * rb;
            }
        }
        __syncthreads();
    }
    // X = R^T with rows in pivot order; past a rank deficiency the remaining positions take the
    // remaining indices in ascending order
    if (tid == 0) {
        int pos = kend;
        for (int o = 0; o < n; ++o)
            if (s_rem[o]) s_perm[pos++] = o;
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
        const int pos = idx % n, c = idx / n;
        X[idx] = (pos >= c && c < kend) ? Rr[(size_t)c * n + s_perm[pos]] : 0.0;
    }
    for (int i = tid; i < n; i += nt) perm_out[i] = s_perm[i];
    if (tid == 0 && deficient) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
}

// ---------------------------------------------------------------- cluster one-sided Jacobi
constexpr int OS_MAXRING = 18;  // receive buffers per side: 2P + 2 for P <= 8
constexpr int OS_MAXP = 8;   // pairs per CTA (n <= 256 on 16 CTAs: two warps each)

struct OsParams {
    const double* X;  // n x n (ld n): columns to orthogonalise (X = R^T)
    const int* perm;
    int n;            // true size
    int np;           // padded column count (multiple of 4 * clusterSize)
    int P;            // pairs per CTA (2 <= P <= OS_MAXP)
    double tol;
    int max_sweeps;
    long long wait_limit;
    double* lam;      // [n]  ||x_j||^2
    double* V;        // n x n, column j = P^T x_j / ||x_j||
    DevInfo* info;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ uint32_t os_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int os_hi(double x) { return __double2hiint(x); }
__device__ __forceinline__ uint32_t os_mapa(const void* local, int rank) {
    uint32_t raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(os_smem(local)), "r"(rank));
    return raddr;
}
// bounded wait with cluster-scope acquire
__device__ __forceinline__ bool os_wait(const uint64_t* bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(os_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}
// st.async into another CTA's shared memory: the write completes an 8-byte transaction on that
// CTA's mbarrier (no release fence on the sender; the receiver's acquire sees the data)
__device__ __forceinline__ void os_st_async(uint32_t raddr, double v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
                 "l"(__double_as_longlong(v)), "r"(rbar)
                 : "memory");
}
// one arrival on this CTA's mbarrier that expects `bytes` more for the phase
__device__ __forceinline__ void os_arm(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(os_smem(bar)), "r"(bytes) : "memory");
}
// X 2^k (X unsigned), rounded to nearest even, as a double (normal range assumed)
__device__ __forceinline__ double os_u64_to_double(unsigned long long X, int k, bool neg) {
    if (X == 0ull) return 0.0;
    const int lz = __clzll((long long)X);
    const unsigned long long a = X << lz;
    unsigned long long m = a >> 11;
    const unsigned long long rest = a & 0x7ffull;
    if (rest > 0x400ull || (rest == 0x400ull && (m & 1ull))) ++m;
    int e = 63 - lz + k;  // exponent of the leading bit
    if (m >> 53) { m >>= 1; ++e; }
    return __longlong_as_double((long long)((neg ? (1ull << 63) : 0ull) | ((unsigned long long)(e + 1023) << 52) |
                                            (m & 0xfffffffffffffull)));
}
// x as a signed fixed-point integer in units 2^(S - 62), truncated toward zero; requires |x| < 2^S
// (then the magnitude stays below 2^62)
__device__ __forceinline__ long long os_to_fixed(double x, int S) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;
    const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);  // x = mant 2^(ex - 1075)
    const int sh = ex - 1075 - (S - 62);
    const long long v = sh >= 0 ? (long long)(mant << sh) : (sh <= -64 ? 0ll : (long long)(mant >> (-sh)));
    return (b >> 63) ? -v : v;
}
// Column slots of a CTA: top[u] and bot[u] (u < P) hold the two columns of pair u.  A
// slot maps to one of the CTA's buffers: 2P local ones (the initial columns), then a ring
// of D buffers for columns arriving from the left neighbour and one for columns from the
// right.  In the circle tournament, per step, the top row moves right and the bottom row
// left: top[P-1] leaves to the right neighbour's top[0], bot[0] to the left neighbour's
// bot[P-1]; the first CTA keeps top[0] and moves bot[0] to top[1], the last moves top[P-1]
// to bot[P-1].  A received column stays at most 2P steps in a CTA (the last CTA passes it
// through its top and its bottom row).  A neighbour stores into ring slot K mod D at step K
// only after it has received this CTA's column of step K - 1, which was sent after this
// CTA's barrier of step K - 2: so a ring of D = 2P + 2 buffers per side keeps every store
// causally after the last read of the column it overwrites.
//
// os_buf gives the buffer of a slot at step K in closed form (ring = K mod D): a column
// that entered the CTA from a neighbour sits in the ring slot of the step it arrived,
// which is a fixed number of steps back along its path through the CTA; before any
// arrival the slot still holds an initial column.  A single-CTA cluster only rotates its
// 2P - 1 moving columns round the circle.
__device__ __forceinline__ int os_wrap(int v, int D) { return v < 0 ? v + D : v; }
__device__ __forceinline__ int os_buf(int c, int C, int P, int D, int K, int ring, int u, bool top) {
    if (C == 1) {
        if (top && u == 0) return 0;
        const int L = 2 * P - 1;
        const int x = top ? u - 1 : 2 * P - 2 - u;  // position on the circle
        const int y = ((x - K) % L + L) % L;         // where its column started
        return y <= P - 2 ? y + 1 : 3 * P - 2 - y;
    }
    const int RL0 = 2 * P, RR0 = 2 * P + D;
    if (top) {
        if (c > 0) return K > u ? RL0 + os_wrap(ring - u - 1, D) : u - K;
        if (u == 0) return 0;
        if (K < u) return u - K;  // first CTA: top[u] came from bot[0] u steps back
        return K - u > P - 1 ? RR0 + os_wrap(ring - u - P, D) : P + K - u;
    }
    if (c < C - 1) return K > P - 1 - u ? RR0 + os_wrap(ring - P + u, D) : P + u + K;
    // last CTA: bot[u] came from top[P-1] P - u steps back
    if (K <= P - 1 - u) return P + u + K;
    if (K < 2 * P - u) return 2 * P - 1 - K - u;
    return RL0 + os_wrap(ring - 2 * P + u, D);
}
__device__ __forceinline__ void os_pair_bar(int a) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + a) : "memory");
}

// Two warps per pair (half h holds rows 32 h .. 32 h + 31, one per lane): GB300's FP64 pipe
// takes one instruction of a warp per ~64 cycles, independent or not, and about one per 19
// cycles from the whole SM, so the FP64 work of a step is spread over the pair's two warps.
// Per step a warp issues 1 FP64 instruction for its part of g = x_p^T x_q, 1 for a_qq - a_pp
// and 4 for the rotation of its rows; half 0 also the 6 of the orthogonality correction,
// half 1 the 3 of the norm updates (they exchange their results through shared memory at a
// 64-thread barrier).  The reduction of g is an exact sum of 64-bit fixed-point integers
// (units 2^(S - 62), 2^S above 4 ||x_p|| ||x_q|| from the exponents of the norms) on the
// integer pipes, over the lanes and then the two halves, and the angle is FP32.  A leaving
// column is written from registers with st.async into the neighbour's ring buffer, each
// 8-byte store completing a transaction on the neighbour's mbarrier, which its owner arms
// (one arrival expecting a column's bytes) for every use.
// RPL rows per lane and half: columns of 64 RPL rows (n <= 64 RPL); lane l of half h holds rows
// 32 h + l + 64 i, i < RPL.
template <int RPL>
__global__ void __launch_bounds__(64 * OS_MAXP, 1) onesided_jacobi_kernel(OsParams prm) {
    constexpr int ROWS = 64 * RPL, LD = ROWS + 2;  // a column: its rows, squared norm, id (integer bits)
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int c = (int)cluster.block_rank();
    const int n = prm.n, np = prm.np, P = prm.P;
    const int D = 2 * P + 2;  // receive ring depth per side
    extern __shared__ __align__(16) double sm[];
    double* bufs = sm;  // [2P + 2D][LD]
    const int RL0 = 2 * P, RR0 = 2 * P + D;
    __shared__ uint64_t rbar[2][OS_MAXRING];  // [0]: from the left, [1]: from the right
    __shared__ long long s_g[OS_MAXP][2];     // per pair: each half's part of g (fixed point)
    __shared__ double s_rot2[OS_MAXP][2];     // per pair: the applied (cs, sn)
    __shared__ double s_nrm[OS_MAXP][2];      // per pair: the updated squared norms
    __shared__ double s_rc[OS_MAXP][2][2];    // per pair: recomputed squared norms, by column and half
    __shared__ int s_rcf[OS_MAXP];            // per pair: which norms are recomputed
    __shared__ int s_rot;
    __shared__ int s_cnt[2];                // used in CTA 0: per-sweep cluster totals
    __shared__ int s_total;
    __shared__ int s_lmax;                  // this CTA's largest scaled |g| of the sweep (float bits)
    __shared__ int s_mx[2];                 // used in CTA 0: per-sweep cluster maxima (float bits)
    __shared__ int s_mx_total;
    __shared__ int s_fail[2];               // used in CTA 0: failed pairs of a convergence check
    __shared__ int s_fail_total;
    __shared__ int s_napp[2];               // used in CTA 0: columns outside the first-order range
    __shared__ int s_napp_total;
    __shared__ double s_coef[2 * OS_MAXP][2 * OS_MAXP * 16];  // first-order angles E(local u, column v)
    __shared__ int s_colofs[2 * OS_MAXP * 16];   // check: offset of each column of the cluster
    __shared__ int s_timeout;
    __shared__ float s_off[16];             // per warp: the largest scaled |g| left in the sweep
    __shared__ float s_off_cta;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = (int)(blockDim.x >> 5);  // 2P
    const int a = warp >> 1, h = warp & 1;      // this warp's pair and half
    const int row = 32 * h + lane;
    const int N = np - 1;
    const double tol2 = prm.tol * prm.tol;
    const int T2 = (int)((__double_as_longlong(tol2) >> 52) & 0x7ff) - 1023;  // tol^2 in [2^T2, 2^(T2+1))
    const unsigned colbytes = (unsigned)(sizeof(double) * LD);

    if (tid == 0) {
        for (int s = 0; s < 2; ++s)
            for (int r = 0; r < D; ++r) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(os_smem(&rbar[s][r])));
            }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the first use of every ring slot expects one column
        for (int s = 0; s < 2; ++s)
            for (int r = 0; r < D; ++r) os_arm(&rbar[s][r], colbytes);
        s_cnt[0] = s_cnt[1] = 0;
        s_mx[0] = s_mx[1] = 0;
        s_fail[0] = s_fail[1] = 0;
        s_napp[0] = s_napp[1] = 0;
        s_timeout = 0;
    }
    // initial placement: local top u <- column cP+u, bottom u <- column np-1-cP-u
    for (int u = warp; u < 2 * P; u += nwarps) {
        const int col = (u < P) ? c * P + u : np - 1 - c * P - (u - P);
        double* b = bufs + (size_t)u * LD;
        double s2 = 0.0;
        for (int r = lane; r < ROWS; r += 32) {
            const double v = (col < n && r < n) ? prm.X[r + (size_t)col * n] : 0.0;
            b[r] = v;
            s2 = fma(v, v, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) { b[ROWS] = s2; b[ROWS + 1] = __longlong_as_double((long long)col); }
    }
    cluster.sync();

    int sweep = 0;
    bool converged = false;
    int K = 0;               // global step counter
    float best_off = 0.0f;
    float sweep_mx = 0.0f;  // the largest scaled |g| met in the sweep
    int checks = 0;
    bool timed_out = false;
    int ring = 0;            // K mod D
    unsigned phase = 0u;     // (K / D) mod 2
    while (sweep < prm.max_sweeps) {
        ++sweep;
        if (tid == 0) { s_rot = 0; s_lmax = 0; }
        best_off = 0.0f;
        sweep_mx = 0.0f;
        // exact squared norms at the start of the sweep
        for (int u = warp; u < 2 * P; u += nwarps) {
            double* b = bufs + (size_t)(u < P ? os_buf(c, C, P, D, K, ring, u, true)
                                              : os_buf(c, C, P, D, K, ring, u - P, false)) * LD;
            double s2 = 0.0;
#pragma unroll
            for (int i = 0; i < 2 * RPL; ++i) s2 = fma(b[lane + 32 * i], b[lane + 32 * i], s2);
            s2 = warp_sum(s2);
            if (lane == 0) b[ROWS] = s2;
        }
        __syncthreads();
        int bt = os_buf(c, C, P, D, K, ring, a, true), bb = os_buf(c, C, P, D, K, ring, a, false);
        for (int k = 0; k < N; ++k, ++K) {
            double* xp = bufs + (size_t)bt * LD;
            double* xq = bufs + (size_t)bb * LD;
            double pr[RPL], qr[RPL];
#pragma unroll
            for (int i = 0; i < RPL; ++i) { pr[i] = xp[row + 64 * i]; qr[i] = xq[row + 64 * i]; }
            const double app = xp[ROWS], aqq = xq[ROWS];
            const long long idp = __double_as_longlong(xp[ROWS + 1]), idq = __double_as_longlong(xq[ROWS + 1]);
            // g = x_p^T x_q: one FP64 product per lane, summed exactly as 64-bit fixed-point
            // integers in units 2^(S - 62), with 2^S >= 4 (a_pp a_qq)^(1/2) >= 4 sum |x_p x_q|
            const int ea = (int)((__double_as_longlong(app) >> 52) & 0x7ff) - 1023;
            const int eb = (int)((__double_as_longlong(aqq) >> 52) & 0x7ff) - 1023;
            const int S = ((ea + eb + 3) >> 1) + 2;
            long long G = 0;
#pragma unroll
            for (int i = 0; i < RPL; ++i) G += os_to_fixed(pr[i] * qr[i], S);
            const double dpq = aqq - app;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) G += __shfl_xor_sync(0xffffffffu, G, o);
            if (lane == 0) s_g[a][h] = G;
            os_pair_bar(a);
            G = s_g[a][0] + s_g[a][1];
            const double g = os_u64_to_double((unsigned long long)(G < 0 ? -G : G), S - 62, G < 0);
            // both halves take every decision below from the same values, so they agree.
            // Column ids are integer bit patterns; positive doubles have positive patterns.
            const bool live = idp < n && idq < n && __double_as_longlong(app) > 0 && __double_as_longlong(aqq) > 0;
            // the scaled test |g| > tol sqrt(a_pp a_qq), decided on the exponents when they are
            // clearly on one side: with normal g, a_pp, a_qq, g^2 / (a_pp a_qq) lies in
            // (2^(d-2), 2^(d+2)) for d = 2 e_g - e_p - e_q, and tol^2 in [2^T, 2^(T+1)); exactly in
            // FP64 otherwise.  The FP32 ratio only feeds the sweep statistics.
            bool rot = false;
            if (live && G != 0) {
                const int bg = (os_hi(g) >> 20) & 0x7ff, ba = ea + 1023, bb = eb + 1023;
                const int d = 2 * bg - ba - bb;
                const bool normal = bg > 0 && ba > 0 && bb > 0 && bg < 0x7ff && ba < 0x7ff && bb < 0x7ff;
                if (normal && d >= T2 + 3) rot = true;
                else if (!normal || d >= T2 - 1) rot = g * g > tol2 * (app * aqq);
                const float gf = fabsf(os_to_float(g)), af = os_to_float(app), bf = os_to_float(aqq);
                const bool in_range =
                    af > 1e-30f && af < 1e30f && bf > 1e-30f && bf < 1e30f && gf > 1e-30f && gf < 1e30f;
                const float rr = in_range ? gf * rsqrtf(af) * rsqrtf(bf) : 0.0f;
                if (!rot) best_off = fmaxf(best_off, rr);
                sweep_mx = fmaxf(sweep_mx, in_range ? rr : (rot ? 1.0f : 0.0f));
            }
            double nr[RPL], mr[RPL];
#pragma unroll
            for (int i = 0; i < RPL; ++i) { nr[i] = pr[i]; mr[i] = qr[i]; }
            double np2 = app, nq2 = aqq;
            if (rot) {
                // Rutishauser's t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)), zeta = (a_qq - a_pp)/2g,
                // sgn(0) = +1, in FP32 from ratios <= 1 (its accuracy only sets how far g is
                // reduced; a_qq - a_pp comes from FP64: for clustered sigma the difference of two
                // FP32 roundings would be noise); c0 = 1/sqrt(1 + t^2), s0 = t c0; the applied
                // rotation is (c0, s0) scaled to unit length in FP64.
                // Taken by half angles: tan 2theta = |2g| / |a_qq - a_pp|, theta in [0, pi/4];
                // cos 2theta and sin 2theta from the ratio (<= 1) of the smaller to the larger,
                // then c0 = (1 + cos 2theta) / (2 (1 + cos 2theta))^(1/2) = cos theta and
                // |s0| = sin 2theta / (2 (1 + cos 2theta))^(1/2) = sin theta (1 + cos 2theta >= 1:
                // no cancellation); t = tan theta = sin 2theta / (1 + cos 2theta).
                const float df = os_to_float(dpq);
                const float hf = 2.0f * os_to_float(g);
                const float adf = fabsf(df), ahf = fabsf(hf);
                const float sz = (df == 0.0f || (df > 0.0f) == (hf > 0.0f)) ? 1.0f : -1.0f;
                const bool dbig = adf >= ahf;
                const float z = ahf == 0.0f ? 0.0f : (dbig ? __fdividef(ahf, adf) : __fdividef(adf, ahf));
                const float r2 = rsqrtf(fmaf(z, z, 1.0f));
                const float c2 = dbig ? r2 : z * r2, s2 = dbig ? z * r2 : r2;
                const float u2 = 1.0f + c2;
                const float q2 = rsqrtf(2.0f * u2);
                const float cf = u2 * q2, sf = sz * (s2 * q2);
                if (h == 0) {
                    // (c0, s0) scaled to unit length to FP64 precision: e = c0^2 + s0^2 - 1 (exact
                    // in FP64, |e| ~ 2^-24), f = 1 - e/2 + 3e^2/8 = (1 + e)^(-1/2) + O(e^3)
                    const double c0 = os_to_double(cf), s0 = os_to_double(sf);
                    const double ee = fma(c0, c0, fma(s0, s0, -1.0));
                    const double f = fma(ee, fma(ee, 0.375, -0.5), 1.0);
                    if (lane == 0) { s_rot2[a][0] = c0 * f; s_rot2[a][1] = s0 * f; }
                } else {
                    // Within a sweep the squared norms only steer later angles and tests; they
                    // follow the exact-angle update a_pp - t g, a_qq + t g.  Every sweep starts
                    // from exact norms, and the final sweep (no rotation) uses only those.  A
                    // norm that dropped by 16x is recomputed (cancellation in the update).
                    const double tg = os_to_double(sz * __fdividef(s2, u2)) * g;
                    const double u2 = app - tg, v2 = aqq + tg;
                    if (lane == 0) {
                        s_nrm[a][0] = u2;
                        s_nrm[a][1] = v2;
                        s_rcf[a] = (os_hi(u2) < os_hi(app) - (4 << 20) ? 1 : 0) |
                                   (os_hi(v2) < os_hi(aqq) - (4 << 20) ? 2 : 0);
                    }
                }
                os_pair_bar(a);
                const double cs = s_rot2[a][0], sn = s_rot2[a][1];
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    nr[i] = fma(cs, pr[i], -sn * qr[i]);
                    mr[i] = fma(sn, pr[i], cs * qr[i]);
                }
                np2 = s_nrm[a][0];
                nq2 = s_nrm[a][1];
                const int rc = s_rcf[a];
                if (rc) {
                    double r1 = 0.0, r2 = 0.0;
#pragma unroll
                    for (int i = 0; i < RPL; ++i) { r1 = fma(nr[i], nr[i], r1); r2 = fma(mr[i], mr[i], r2); }
                    r1 = (rc & 1) ? warp_sum(r1) : 0.0;
                    r2 = (rc & 2) ? warp_sum(r2) : 0.0;
                    if (lane == 0) { s_rc[a][0][h] = r1; s_rc[a][1][h] = r2; }
                    os_pair_bar(a);
                    if (rc & 1) np2 = s_rc[a][0][0] + s_rc[a][0][1];
                    if (rc & 2) nq2 = s_rc[a][1][0] + s_rc[a][1][1];
                }
                if (h == 0 && lane == 0) atomicAdd(&s_rot, 1);
            }
            // top[P-1] leaves to the right, bot[0] to the left, from registers with its norm
            // and id (half 1 sends those); every other column is written back in place
            const bool lead = h == 1 && lane == 0;
            if (a == P - 1 && c < C - 1) {
                const uint32_t dst = os_mapa(bufs + (size_t)(RL0 + ring) * LD, c + 1);
                const uint32_t rb = os_mapa(&rbar[0][ring], c + 1);
#pragma unroll
                for (int i = 0; i < RPL; ++i) os_st_async(dst + 8u * (unsigned)(row + 64 * i), nr[i], rb);
                if (lead) {
                    os_st_async(dst + 8u * (unsigned)ROWS, np2, rb);
                    os_st_async(dst + 8u * (unsigned)(ROWS + 1), __longlong_as_double(idp), rb);
                }
            } else {
#pragma unroll
                for (int i = 0; i < RPL; ++i) xp[row + 64 * i] = nr[i];
                if (lead) xp[ROWS] = np2;
            }
            if (a == 0 && c > 0) {
                const uint32_t dst = os_mapa(bufs + (size_t)(RR0 + ring) * LD, c - 1);
                const uint32_t rb = os_mapa(&rbar[1][ring], c - 1);
#pragma unroll
                for (int i = 0; i < RPL; ++i) os_st_async(dst + 8u * (unsigned)(row + 64 * i), mr[i], rb);
                if (lead) {
                    os_st_async(dst + 8u * (unsigned)ROWS, nq2, rb);
                    os_st_async(dst + 8u * (unsigned)(ROWS + 1), __longlong_as_double(idq), rb);
                }
            } else {
#pragma unroll
                for (int i = 0; i < RPL; ++i) xq[row + 64 * i] = mr[i];
                if (lead) xq[ROWS] = nq2;
            }
            // the columns arriving in this step (every thread acquires them itself); after one
            // wait has run out the rest fail at once, so a lost neighbour costs one limit
            const long long lim = timed_out ? 0 : prm.wait_limit;
            const bool got_l = c > 0 && os_wait(&rbar[0][ring], phase, lim);
            const bool got_r = c < C - 1 && os_wait(&rbar[1][ring], phase, lim);
            if ((c > 0 && !got_l) || (c < C - 1 && !got_r)) { timed_out = true; s_timeout = 1; }
            if (tid == 0) {
                // this slot's next use (step K + D) expects one column again (only once the
                // phase has completed: an arrival on an incomplete phase would be one too many)
                if (got_l) os_arm(&rbar[0][ring], colbytes);
                if (got_r) os_arm(&rbar[1][ring], colbytes);
            }
            if (++ring == D) { ring = 0; phase ^= 1u; }
            // the next step's slots, off the path that follows the barrier
            bt = os_buf(c, C, P, D, K + 1, ring, a, true);
            bb = os_buf(c, C, P, D, K + 1, ring, a, false);
            __syncthreads();
        }
        // cluster-wide rotation count and largest scaled |g| of this sweep
        const int sp = sweep & 1;
        if (lane == 0) atomicMax(&s_lmax, __float_as_int(sweep_mx));
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&cluster.map_shared_rank(s_cnt, 0)[sp], s_rot);
            atomicMax(&cluster.map_shared_rank(s_mx, 0)[sp], s_lmax);
        }
        cluster.sync();
        if (tid == 0) {
            s_total = cluster.map_shared_rank(s_cnt, 0)[sp];
            s_mx_total = cluster.map_shared_rank(s_mx, 0)[sp];
        }
        __syncthreads();
        const int total = s_total;
        const float mx = __int_as_float(s_mx_total);
        if (c == 0 && tid == 0) { s_cnt[sp ^ 1] = 0; s_mx[sp ^ 1] = 0; }
        if (total == 0) { converged = true; break; }
        // Jacobi converges quadratically: after a sweep whose largest scaled |g| was mx the pairs
        // are left near mx^2, and after a sweep with few rotations (at most n) the next one
        // usually has none.  Then, instead of a sweep that would only confirm convergence, every
        // pair of the current columns is tested at once (the same scaled test, exact norms), and
        // a sweep runs only if some pair fails.  When the pairs that fail are all deep in the
        // quadratic range, one simultaneous first-order step replaces the sweep: with
        // A = X^T X = D + F (F off-diagonal), X (I + E) for the antisymmetric
        // E_vu = g_uv / (a_u - a_v) leaves off-diagonals of order |E| |F|, and (I + E)^T (I + E)
        // = I - E^2 is orthogonal to FP64 precision when every column of E has
        // sum_v E_vu^2 <= 2^-53 (each |E_vu| <= 2^-27 besides).  The check then runs again.
        // A check is one pass over the pairs (a few microseconds), a sweep n - 1 dependent steps.
        const bool near = mx < 0x1p-20f || (double)mx * (double)mx <= prm.tol || total <= n || mx <= 0x1p-14f;
        if (near && sweep < prm.max_sweeps) {
            const int slots = 2 * P, cols = slots * C;
            // where each column of the cluster sits during the check (CTA v / slots, this offset)
            for (int v = tid; v < cols; v += blockDim.x) {
                const int w = v % slots, rk = v / slots;
                s_colofs[v] = (w < P ? os_buf(rk, C, P, D, K, ring, w, true) : os_buf(rk, C, P, D, K, ring, w - P, false)) * LD;
            }
            // with one row per lane the whole cluster's columns are copied into this CTA (many
            // independent remote loads at once); otherwise they are read in place
            double* s_all = bufs + (size_t)(2 * P + 2 * D) * LD;
            auto col = [&](int v) -> const double* {
                if constexpr (RPL == 1) return s_all + (size_t)v * LD;
                else return cluster.map_shared_rank(bufs, v / slots) + s_colofs[v];
            };
            for (int pass = 0; pass < 3; ++pass) {
                for (int u = warp; u < slots; u += nwarps) {
                    double* b = bufs + (size_t)(u < P ? os_buf(c, C, P, D, K, ring, u, true)
                                                      : os_buf(c, C, P, D, K, ring, u - P, false)) * LD;
                    double s2 = 0.0;
                    for (int r = lane; r < ROWS; r += 32) s2 = fma(b[r], b[r], s2);
                    s2 = warp_sum(s2);
                    if (lane == 0) b[ROWS] = s2;
                }
                cluster.sync();
                if constexpr (RPL == 1) {
                    for (int idx = tid; idx < cols * LD; idx += blockDim.x) {
                        const int v = idx / LD, r = idx - v * LD;
                        s_all[idx] = cluster.map_shared_rank(bufs, v / slots)[s_colofs[v] + r];
                    }
                    __syncthreads();
                }
                int fails = 0, napp = 0;
                const int items = slots * cols;
                for (int it = tid; it < items; it += blockDim.x) {
                    const int u = it % slots, v = it / slots;
                    const double* bu = col(c * slots + u);
                    const double* bv = col(v);
                    const long long iu = __double_as_longlong(bu[ROWS + 1]), iv = __double_as_longlong(bv[ROWS + 1]);
                    const double au = bu[ROWS], av = bv[ROWS];
                    double e = 0.0;
                    if (iu < n && iv < n && iu != iv && au > 0.0 && av > 0.0) {
                        double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
#pragma unroll
                        for (int r = 0; r < ROWS; r += 4) {
                            g0 = fma(bu[r], bv[r], g0);
                            g1 = fma(bu[r + 1], bv[r + 1], g1);
                            g2 = fma(bu[r + 2], bv[r + 2], g2);
                            g3 = fma(bu[r + 3], bv[r + 3], g3);
                        }
                        const double g = (g0 + g1) + (g2 + g3);  // the same value in both columns' CTAs
                        if (iu < iv && g * g > tol2 * (au * av)) ++fails;
                        const double dd = au - av;
                        if (fabs(g) <= 0x1p-27 * fabs(dd)) e = g / dd;
                        else if (g * g > tol2 * (au * av)) ++napp;  // a failing pair outside the range
                    }
                    s_coef[u][v] = e;
                }
                __syncthreads();
                // columns whose first-order step would not be orthogonal to FP64 precision
                for (int u = warp; u < slots; u += nwarps) {
                    double s2 = 0.0;
                    for (int v = lane; v < cols; v += 32) s2 = fma(s_coef[u][v], s_coef[u][v], s2);
                    s2 = warp_sum(s2);
                    if (lane == 0 && s2 > 0x1p-53) ++napp;
                }
                const int cp = checks & 1;
                ++checks;
                if (fails) atomicAdd(&cluster.map_shared_rank(s_fail, 0)[cp], fails);
                if (napp) atomicAdd(&cluster.map_shared_rank(s_napp, 0)[cp], napp);
                cluster.sync();
                if (tid == 0) {
                    s_fail_total = cluster.map_shared_rank(s_fail, 0)[cp];
                    s_napp_total = cluster.map_shared_rank(s_napp, 0)[cp];
                }
                __syncthreads();
                const int f = s_fail_total, na = s_napp_total;
                if (c == 0 && tid == 0) { s_fail[cp ^ 1] = 0; s_napp[cp ^ 1] = 0; }
                if (f == 0) { converged = true; break; }
                if (na != 0 || pass == 2) break;  // not deep in the quadratic range: sweep on
                // the first-order step x_u <- x_u + sum_v x_v E(u, v) (E = 0 leaves x_u as it is)
                double acc[2 * RPL];
#pragma unroll
                for (int i = 0; i < 2 * RPL; ++i) acc[i] = 0.0;
                const int u = warp;  // one warp per local column (nwarps = 2P)
#pragma unroll 4
                for (int v = 0; v < cols; ++v) {
                    const double e = s_coef[u][v];
                    const double* bv = col(v);
#pragma unroll
                    for (int i = 0; i < 2 * RPL; ++i) acc[i] = fma(bv[lane + 32 * i], e, acc[i]);
                }
                // in place, once no CTA reads this CTA's columns any more (with the copies, every
                // CTA finished copying before the counts were summed)
                if constexpr (RPL != 1) cluster.sync();
                {
                    double* b = bufs + (size_t)(u < P ? os_buf(c, C, P, D, K, ring, u, true)
                                                      : os_buf(c, C, P, D, K, ring, u - P, false)) * LD;
#pragma unroll
                    for (int i = 0; i < 2 * RPL; ++i) b[lane + 32 * i] += acc[i];
                }
                __syncthreads();
            }
            if (converged) break;
        }
    }
    // outputs: lambda_j = ||x_j||^2, v_j = P^T x_j / ||x_j||
    for (int u = warp; u < 2 * P; u += nwarps) {
        const double* b = bufs + (size_t)(u < P ? os_buf(c, C, P, D, K, ring, u, true)
                                                : os_buf(c, C, P, D, K, ring, u - P, false)) * LD;
        const int j = (int)__double_as_longlong(b[ROWS + 1]);
        if (j >= n) continue;
        double s2 = 0.0;
        for (int r = lane; r < ROWS; r += 32) s2 = fma(b[r], b[r], s2);
        s2 = warp_sum(s2);
        const double nrm = sqrt(s2);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int r = lane; r < n; r += 32) prm.V[prm.perm[r] + (size_t)j * n] = b[r] * inv;
        if (lane == 0) prm.lam[j] = s2;
    }
    // info: sweeps and the largest scaled |g| seen in the last sweep
    if (lane == 0 && warp < 16) s_off[warp] = best_off;
    __syncthreads();
    if (tid == 0) {
        float off = 0.0f;
        for (int w = 0; w < nwarps && w < 16; ++w) off = fmaxf(off, s_off[w]);
        s_off_cta = off;
    }
    cluster.sync();
    if (c == 0 && tid == 0) {
        float off = 0.0f;
        for (int r = 0; r < C; ++r) off = fmaxf(off, *cluster.map_shared_rank(&s_off_cta, r));
        prm.info->sweeps = sweep;
        prm.info->off_norm = (double)off;
        if (!converged) atomicOr(&prm.info->flags, FLAG_NO_CONVERGENCE);
    }
    if (s_timeout && tid == 0) atomicOr(&prm.info->flags, FLAG_TIMEOUT);
    cluster.sync();  // no CTA leaves while a neighbour may still read or write its shared memory
}

// ---------------------------------------------------------------- kappa(B) estimate
// L = rows of X scaled by 1/d_pos (d_pos = sqrt of M's diagonal at the pivot's original
// index) is lower triangular with L L^T = P C P^T, C = D^-1 M D^-1 with unit diagonal, so
// kappa(B) = (lambda_max / lambda_min)^(1/2) of L L^T.  One warp, FP32 (an estimate):
// power iteration for lambda_max, inverse iteration (two triangular solves) for lambda_min.
// Lane l holds rows l and l + 32.
constexpr int KAPPA_ITERS = 16;
constexpr int KLD = 65;  // padded column stride: row-wise reads hit distinct banks

__global__ void __launch_bounds__(32)
    kappa_kernel(const double* __restrict__ X, const int* __restrict__ perm, const double* __restrict__ M,
                 int64_t ldm, int n, DevInfo* info) {
    __shared__ float Lc[64 * KLD];  // column-major: Lc[i + KLD j] = L[i][j]
    __shared__ float v[64], w[64];
    const int lane = threadIdx.x;
    bool bad = false;
    for (int idx = lane; idx < 64 * 64; idx += 32) {
        const int i = idx & 63, j = idx >> 6;
        float val = 0.0f;
        if (i < n && j < n && i >= j) {
            const int o = perm[i];
            const double dd = M[o + (size_t)o * ldm];
            val = dd > 0.0 ? (float)(X[i + (size_t)j * n] / sqrt(dd)) : 0.0f;
        }
        Lc[i + KLD * j] = val;
    }
    __syncwarp();
    for (int j = lane; j < n; j += 32)
        if (!(Lc[j + KLD * j] != 0.0f)) bad = true;
    bad = __any_sync(0xffffffffu, bad);
    float lmax = 0.0f, lmin = 0.0f;
    if (!bad) {
        // lambda_max of L^T L (= that of L L^T): v <- L^T (L v), normalised
        for (int i = lane; i < 64; i += 32) v[i] = i < n ? 1.0f + 0.01f * (float)i : 0.0f;
        __syncwarp();
        for (int it = 0; it < KAPPA_ITERS; ++it) {
            // w = L v
            for (int i = lane; i < 64; i += 32) {
                float s = 0.0f;
                for (int j = 0; j <= i && j < n; ++j) s = fmaf(Lc[i + KLD * j], v[j], s);
                w[i] = s;
            }
            __syncwarp();
            // v = L^T w
            float nn = 0.0f;
            float nv[2] = {0.0f, 0.0f};
            for (int q = 0; q < 2; ++q) {
                const int j = lane + 32 * q;
                float s = 0.0f;
                for (int i = j; i < n; ++i) s = fmaf(Lc[i + KLD * j], w[i], s);
                nv[q] = s;
                nn = fmaf(s, s, nn);
            }
            for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
            // ||L^T L v|| / ||v|| with ||v|| = 1 after the first iteration
            const float scale = rsqrtf(nn);
            float vv = 0.0f;
            for (int q = 0; q < 2; ++q) vv = fmaf(v[lane + 32 * q], v[lane + 32 * q], vv);
            for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
            lmax = sqrtf(nn) * rsqrtf(vv);
            __syncwarp();
            for (int q = 0; q < 2; ++q) v[lane + 32 * q] = nv[q] * scale;
            __syncwarp();
        }
        // lambda_min: w = (L^T L)^-1 v by L^T y = v (backward), then L w = y (forward)
        for (int i = lane; i < 64; i += 32) v[i] = i < n ? 1.0f - 0.01f * (float)i : 0.0f;
        __syncwarp();
        for (int it = 0; it < KAPPA_ITERS; ++it) {
            float r0 = v[lane], r1 = v[lane + 32];
            // L^T y = v: for j = n-1 .. 0, y_j = r_j / L[j][j]; r_i -= L[j][i] y_j for i < j
            for (int j = n - 1; j >= 0; --j) {
                const float rj = __shfl_sync(0xffffffffu, j < 32 ? r0 : r1, j & 31);
                const float yj = rj / Lc[j + KLD * j];
                if (lane == (j & 31)) { if (j < 32) r0 = yj; else r1 = yj; }
                if (lane < j) r0 = fmaf(-Lc[j + KLD * lane], yj, r0);
                if (lane + 32 < j) r1 = fmaf(-Lc[j + KLD * (lane + 32)], yj, r1);
            }
            // L w = y: for j = 0 .. n-1, w_j = r_j / L[j][j]; r_i -= L[i][j] w_j for i > j
            for (int j = 0; j < n; ++j) {
                const float rj = __shfl_sync(0xffffffffu, j < 32 ? r0 : r1, j & 31);
                const float wj = rj / Lc[j + KLD * j];
                if (lane == (j & 31)) { if (j < 32) r0 = wj; else r1 = wj; }
                if (lane > j) r0 = fmaf(-Lc[lane + KLD * j], wj, r0);
                if (lane + 32 > j && lane + 32 < n) r1 = fmaf(-Lc[lane + 32 + KLD * j], wj, r1);
            }
            if (lane >= n) r0 = 0.0f;
            if (lane + 32 >= n) r1 = 0.0f;
            float nn = r0 * r0 + r1 * r1, vv = v[lane] * v[lane] + v[lane + 32] * v[lane + 32];
            for (int o = 16; o > 0; o >>= 1) {
                nn += __shfl_xor_sync(0xffffffffu, nn, o);
                vv += __shfl_xor_sync(0xffffffffu, vv, o);
            }
            lmin = sqrtf(vv) * rsqrtf(nn);  // ||v|| / ||(L^T L)^-1 v|| -> lambda_min
            const float scale = rsqrtf(nn);
            __syncwarp();
            v[lane] = r0 * scale;
            v[lane + 32] = r1 * scale;
            __syncwarp();
        }
    }
    if (lane == 0)
        info->kappa = (bad || !(lmin > 0.0f)) ? __longlong_as_double(0x7ff0000000000000ll)
                                               : sqrt((double)lmax / (double)lmin);
}

// The FP64 pipe of one SM sets the pace, so the pairs are spread over as many
// SMs as a cluster allows (16 needs the non-portable cluster size; 8 otherwise).
int cluster_size_for(int n, bool allow16) {
    if (n <= 8) return 1;
    if (n <= 16) return 2;
    if (n <= 32) return allow16 ? 8 : 4;
    return allow16 ? 16 : 8;
}

// rows per lane and half of the column buffers: n <= 64, 128 or 256
int rows_per_lane(int n) { return n <= 64 ? 1 : (n <= 128 ? 2 : 4); }

template <int RPL>
cudaError_t launch_cluster_jacobi_t(OsParams prm, int C, cudaStream_t s) {
    prm.np = ((prm.n < 4 ? 4 : prm.n) + 4 * C - 1) / (4 * C) * (4 * C);
    prm.P = prm.np / (2 * C);
    if (prm.P > OS_MAXP) return cudaErrorNotSupported;
    // ring slots, plus (one row per lane) room for a copy of every column of the cluster
    const size_t smem = sizeof(double) * ((size_t)(2 * prm.P + 2 * (2 * prm.P + 2)) + (RPL == 1 ? (size_t)prm.np : 0)) *
                        (64 * RPL + 2);
    cudaError_t e =
        cudaFuncSetAttribute(onesided_jacobi_kernel<RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(64 * prm.P, 1, 1);  // two warps per pair
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, onesided_jacobi_kernel<RPL>, prm);
}

template <int RPL>
bool allow_cluster16() {
    const bool ok = cudaFuncSetAttribute(onesided_jacobi_kernel<RPL>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                         1) == cudaSuccess;
    if (!ok) (void)cudaGetLastError();
    return ok;
}

template <int RPL>
cudaError_t launch_cluster_jacobi(OsParams prm, cudaStream_t s) {
    const int C = cluster_size_for(prm.n, allow_cluster16<RPL>());
    cudaError_t e = launch_cluster_jacobi_t<RPL>(prm, C, s);
    if (e != cudaSuccess && C == 16) {
        // the device may not schedule a 16-CTA cluster: the portable size instead
        (void)cudaGetLastError();
        e = launch_cluster_jacobi_t<RPL>(prm, 8, s);
    }
    return e;
}

}  // namespace

cudaError_t launch_cholesky(const double* M, int n, int64_t ldm, double* X, int* perm, DevInfo* info, bool pivot,
                            cudaStream_t s, double* gm_scratch) {
    if (n > 256 || (n > 64 && gm_scratch == nullptr)) return cudaErrorNotSupported;
    if (n > 64) {
        chol_piv_gm_kernel<<<1, 1024, 0, s>>>(M, n, ldm, gm_scratch, gm_scratch + (size_t)n * n, X, perm, info,
                                              pivot ? 1 : 0);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(chol_piv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * sizeof(double) * 64 * 64));
    if (e != cudaSuccess) return e;
    chol_piv_kernel<<<1, CHL_THREADS, 2 * sizeof(double) * (size_t)n * n, s>>>(M, n, ldm, X, perm, info,
                                                                       pivot ? 1 : 0);
    return cudaGetLastError();
}

// scratch: X (n^2 doubles), perm (n ints in n doubles' room), and for n > 64 the Cholesky's
// global Schur complement and rows of R (2 n^2 doubles): (3 n^2 + n) doubles in all
cudaError_t launch_eig_onesided(const double* M, int n, int64_t ldm, double tol, int max_sweeps,
                                void* scratch, double* lam_ws, double* V_ws, DevInfo* info,
                                cudaStream_t s, const EigSide* side, long long wait_cycles) {
    if (n > 256) return cudaErrorNotSupported;
    double* X = reinterpret_cast<double*>(scratch);
    int* perm = reinterpret_cast<int*>(X + (size_t)n * n);
    double* gm = X + (size_t)n * n + n;
    cudaError_t e = launch_cholesky(M, n, ldm, X, perm, info, true, s, gm);
    if (e != cudaSuccess) return e;
    // kappa(B) on the side stream, beside the Jacobi (joined before the caller's next launch);
    // estimated for n <= 64
    const bool fork = n <= 64 && side != nullptr && side->stream != nullptr;
    if (fork) {
        e = cudaEventRecord(side->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side->stream, side->fork, 0);
        if (e != cudaSuccess) return e;
    }
    if (n <= 64) {
        kappa_kernel<<<1, 32, 0, fork ? side->stream : s>>>(X, perm, M, ldm, n, info);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (fork) {
        e = cudaEventRecord(side->join, side->stream);
        if (e != cudaSuccess) return e;
    }
    OsParams prm{X, perm, n, 0, 0, tol, max_sweeps, wait_limit_of(wait_cycles), lam_ws, V_ws, info};
    const int rpl = rows_per_lane(n);
    e = rpl == 1 ? launch_cluster_jacobi<1>(prm, s) : rpl == 2 ? launch_cluster_jacobi<2>(prm, s)
                                                                : launch_cluster_jacobi<4>(prm, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && fork) e = cudaStreamWaitEvent(s, side->join, 0);
    return e;
}

}  // namespace tsvd
