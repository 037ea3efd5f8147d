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
//      a thread-block cluster: each CTA owns P pair slots (one warp per
//      pair); after each step one column moves to each neighbouring CTA
//      through distributed shared memory, signalled on the neighbour's
//      mbarrier (no cluster-wide barrier within a sweep).
//
// The rotation angle and (c0, s0) are computed in FP32 while the applied
// rotation is made orthogonal to FP64 precision by one FP64 correction
// factor: an inexact angle only leaves a residual g * O(2^-24) on a pair,
// which later sweeps remove, whereas a non-orthogonal rotation would change
// the singular values.  On GB300 a dependent FP64 operation costs about 60
// cycles and an FP64 reciprocal square root about 350, so every division and
// square root goes to the FP32 units.  Squared norms are updated within a sweep by the exact quadratic
// form of the rotation, recomputed at the start of every sweep and whenever
// a norm drops below 1/16 of its previous value; the stopping test of the
// final, rotation-free sweep therefore uses exact norms.
#include <climits>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace tsvd {
namespace {

// ---------------------------------------------------------------- pivoted Cholesky
// One CTA.  M (n x n, ldm) -> X = R^T (n x n, ld n, lower triangular, rows in pivot
// order) and perm (pivot position -> original index).  Nothing is swapped in memory:
// the trailing matrix stays in the original index order and the pivot order lives
// in a permutation, so each step needs two barriers.  Every warp finds the pivot
// itself (the largest remaining diagonal, lowest position on ties).
__global__ void __launch_bounds__(256)
    chol_piv_kernel(const double* __restrict__ M, int n, int64_t ldm, double* __restrict__ X,
                    int* __restrict__ perm_out, DevInfo* info) {
    extern __shared__ double sa[];  // [n][n] trailing Schur complement (original indices), then R rows
    double* Rr = sa + (size_t)n * n;  // [n][n]: row k of R by original column index
    __shared__ int perm[2][64];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    for (int idx = tid; idx < n * n; idx += nt) {
        const int r = idx % n, c = idx / n;
        sa[idx] = M[r + (size_t)c * ldm];
        Rr[idx] = 0.0;
    }
    if (tid < 64) perm[0][tid] = tid;
    __syncthreads();
    bool deficient = false;
    int kend = n;
    for (int k = 0; k < n; ++k) {
        const int* pc = perm[k & 1];
        int* pn = perm[(k & 1) ^ 1];
        // pivot: largest remaining diagonal.  The bit patterns of non-negative doubles order
        // like the values; every negative value (rank deficiency) sorts below them.
        long long best = LLONG_MIN;
        int bq = k;
        for (int q = k + lane; q < n; q += 32) {
            const int o = pc[q];
            const long long dd = __double_as_longlong(sa[o + (size_t)o * n]);
            const long long key = dd < 0 ? LLONG_MIN + 1 : dd;
            if (key > best) { best = key; bq = q; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oq = __shfl_xor_sync(0xffffffffu, bq, off);
            if (ob > best || (ob == best && oq < bq)) { best = ob; bq = oq; }
        }
        const int ok = pc[bq];
        const double d = sa[ok + (size_t)ok * n];
        if (!(d > 0.0)) { deficient = true; kend = k; break; }
        // the permutation with positions k and bq exchanged
        if (tid < n) pn[tid] = (tid == k) ? ok : (tid == bq) ? pc[k] : pc[tid];
        const double rinv = rsqrt(d);  // 1 / r_kk
        // row k of R: R[k][o] = S[ok][o] / r_kk over the remaining original indices o
        for (int t = tid; t < n - k; t += nt) {
            const int q = k + t;
            const int o = (q == k) ? ok : (q == bq) ? pc[k] : pc[q];
            Rr[(size_t)k * n + o] = (q == k) ? d * rinv : sa[ok + (size_t)o * n] * rinv;
        }
        __syncthreads();
        // trailing update S[a][b] -= R[k][a] R[k][b] over the remaining positions > k
        const int rem = n - k - 1;
        const double* rk = Rr + (size_t)k * n;
        for (int idx = tid; idx < rem * rem; idx += nt) {
            const int oa = pn[k + 1 + idx % rem], ob = pn[k + 1 + idx / rem];
            sa[oa + (size_t)ob * n] -= rk[oa] * rk[ob];
        }
        __syncthreads();
    }
    // X = R^T with rows in pivot order: X[pos][c] = R[c][perm[pos]] for pos >= c
    const int* pf = perm[kend & 1];
    for (int idx = tid; idx < n * n; idx += nt) {
        const int pos = idx % n, c = idx / n;
        X[idx] = (pos >= c && c < kend) ? Rr[(size_t)c * n + pf[pos]] : 0.0;
    }
    for (int i = tid; i < n; i += nt) perm_out[i] = pf[i];
    if (tid == 0 && deficient) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
}

// ---------------------------------------------------------------- cluster one-sided Jacobi
struct OsParams {
    const double* X;  // n x n (ld n): columns to orthogonalise (X = R^T)
    const int* perm;
    int n;            // true size
    int np;           // padded column count (multiple of 4 * clusterSize)
    int P;            // pairs per CTA
    double tol;
    int max_sweeps;
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
__device__ __forceinline__ int os_hi(double x) { return __double2hiint(x); }
__device__ __forceinline__ uint32_t os_mapa(const void* local, int rank) {
    uint32_t raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(os_smem(local)), "r"(rank));
    return raddr;
}
// this CTA expects `bytes` more on its own mbarrier (and counts as its one arrival)
__device__ __forceinline__ void os_arm(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(os_smem(bar)), "r"(bytes) : "memory");
}
// bulk copy of `bytes` from this CTA's shared memory into CTA `rank`'s, completing the
// transaction on that CTA's mbarrier (no fence on the sender's critical path)
__device__ __forceinline__ void os_bulk_to(const void* src, const void* dst_local_equiv, const uint64_t* bar_local_equiv,
                                           int rank, unsigned bytes) {
    const uint32_t dst = os_mapa(dst_local_equiv, rank), bar = os_mapa(bar_local_equiv, rank);
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "r"(os_smem(src)), "r"(bytes), "r"(bar)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the source of this thread's bulk copies has been read
__device__ __forceinline__ void os_bulk_read_done() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// bounded wait (about 1 s of GPU clock) with cluster-scope acquire
__device__ __forceinline__ bool os_wait(const uint64_t* bar, unsigned parity) {
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
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

// Each step: every warp rotates its pair; then one column moves to each
// neighbouring CTA (warp 0 owns the link to the right, warp 1 the link to the
// left): the sender stores it into the neighbour's receive buffer and arrives
// on the neighbour's mbarrier; the receiver waits only for its two
// neighbours, so no cluster-wide barrier is needed within a sweep.
__global__ void __launch_bounds__(512) onesided_jacobi_kernel(OsParams prm) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int c = (int)cluster.block_rank();
    const int n = prm.n, np = prm.np, P = prm.P;
    const int LD = ((n + 2) + 1) & ~1;  // x[0..n-1], idx, nrm
    extern __shared__ __align__(16) double sm[];
    double* bufs = sm;                       // [2P][LD]
    double* recv = sm + (size_t)2 * P * LD;  // [2 parity][2 side: 0 from the left, 1 from the right][LD]
    __shared__ uint64_t rbar[2][2];          // same indexing as recv
    __shared__ int map_top[2][32], map_bot[2][32];  // slot -> buffer, double-buffered by step parity
    __shared__ int s_rot;
    __shared__ int s_cnt[2];                 // used in CTA 0: per-sweep cluster totals
    __shared__ int s_total;
    __shared__ int s_lmax;                   // this CTA's largest scaled |g| of the sweep (float bits)
    __shared__ int s_mx[2];                  // used in CTA 0: per-sweep cluster maxima (float bits)
    __shared__ int s_mx_total;
    __shared__ int s_fail[2];                // used in CTA 0: failed pairs of a convergence check
    __shared__ int s_fail_total;
    __shared__ int s_timeout;
    __shared__ float s_off[32];              // per warp: the largest scaled |g| left in the sweep
    __shared__ float s_off_cta;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = np - 1;
    const double tol2 = prm.tol * prm.tol;
    const float tol_f = (float)prm.tol;

    if (tid == 0) {
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(os_smem(&rbar[a][b])));
        // each receive buffer expects one column at steps 0 and 1 (re-armed after every use)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) os_arm(&rbar[a][b], (unsigned)(sizeof(double) * LD));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_cnt[0] = 0;
        s_cnt[1] = 0;
        s_mx[0] = 0;
        s_mx[1] = 0;
        s_fail[0] = 0;
        s_fail[1] = 0;
        s_timeout = 0;
    }
    // initial placement: local top u <- column cP+u, bottom u <- column np-1-cP-u
    for (int u = warp; u < 2 * P; u += blockDim.x / 32) {
        const int col = (u < P) ? c * P + u : np - 1 - c * P - (u - P);
        double* b = bufs + (size_t)u * LD;
        double s2 = 0.0;
        for (int r = lane; r < n; r += 32) {
            const double v = (col < n) ? prm.X[r + (size_t)col * n] : 0.0;
            b[r] = v;
            s2 += v * v;
        }
        s2 = warp_sum(s2);
        if (lane == 0) { b[n] = __longlong_as_double((long long)col); b[n + 1] = s2; }
    }
    if (tid < P) { map_top[0][tid] = tid; map_bot[0][tid] = P + tid; }
    cluster.sync();

    int sweep = 0;
    bool converged = false;
    unsigned K = 0;  // global step counter (parity of buffers and mbarrier phases)
    float best_off = 0.0f;
    float sweep_mx = 0.0f;  // lane 0 of a pair warp: the largest scaled |g| met in the sweep
    int checks = 0;
    while (sweep < prm.max_sweeps) {
        ++sweep;
        if (tid == 0) { s_rot = 0; s_lmax = 0; }
        best_off = 0.0f;
        sweep_mx = 0.0f;
        // exact squared norms at the start of the sweep
        for (int u = warp; u < 2 * P; u += blockDim.x / 32) {
            double* b = bufs + (size_t)u * LD;
            double s2 = 0.0;
            for (int r = lane; r < n; r += 32) s2 += b[r] * b[r];
            s2 = warp_sum(s2);
            if (lane == 0) b[n + 1] = s2;
        }
        __syncthreads();
        for (int k = 0; k < N; ++k, ++K) {
            const int par = (int)(K & 1u);
            const int* top = map_top[par];
            const int* bot = map_bot[par];
            // one warp per pair: g = x_p^T x_q, the rotation, and its application.  Every FP64
            // warp instruction holds its SMSP's FP64 pipe for about 64 cycles on GB300, so the
            // scalar work is kept to the few FP64 operations that set the result.
            if (warp < P) {
                double* xp = bufs + (size_t)top[warp] * LD;
                double* xq = bufs + (size_t)bot[warp] * LD;
                const double app = xp[n + 1], aqq = xq[n + 1];
                double g = 0.0;
                for (int r = lane; r < n; r += 32) g = fma(xp[r], xq[r], g);
                g = warp_sum(g);
                // column ids are stored as integer bit patterns; positive doubles have positive
                // patterns (integer compares keep these tests off the FP64 pipe)
                const bool live = __double_as_longlong(xp[n]) < n && __double_as_longlong(xq[n]) < n &&
                                  __double_as_longlong(app) > 0 && __double_as_longlong(aqq) > 0;
                // the scaled test |g| > tol sqrt(a_pp a_qq): decided in FP32 when the FP32 ratio
                // is clearly on one side (factor 4), exactly in FP64 otherwise
                bool rot = false;
                if (live && g != 0.0) {
                    const float gf = fabsf(os_to_float(g)), af = os_to_float(app), bf = os_to_float(aqq);
                    // all three well inside the FP32 range: r = |g| / sqrt(a_pp a_qq) to ~2^-22
                    const bool in_range = af > 1e-30f && af < 1e30f && bf > 1e-30f && bf < 1e30f &&
                                          gf > 1e-30f && gf < 1e30f;
                    const float rr = in_range ? gf * rsqrtf(af) * rsqrtf(bf) : 0.0f;
                    const float tl = tol_f;
                    if (in_range && rr > 2.0f * tl) rot = true;
                    else if (!in_range || rr > 0.5f * tl) rot = g * g > tol2 * (app * aqq);
                    if (!rot && lane == 0) best_off = fmaxf(best_off, rr);
                    if (lane == 0) sweep_mx = fmaxf(sweep_mx, in_range ? rr : (rot ? 1.0f : 0.0f));
                }
                if (rot) {
                    // Rotation angle from Rutishauser's t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)),
                    // zeta = (a_qq - a_pp) / 2g, sgn(0) = +1, evaluated in FP32 from ratios <= 1
                    // (its accuracy only sets how far g is reduced), and c0 = 1/sqrt(1 + t^2),
                    // s0 = t c0 in FP32.  The applied rotation (c0, s0) f is orthogonal to FP64
                    // precision: with e = c0^2 + s0^2 - 1 (exact in FP64, |e| ~ 2^-24),
                    // f = 1 - e/2 + 3e^2/8 = (1 + e)^(-1/2) + O(e^3).
                    // a_qq - a_pp in FP64 first: for nearly equal norms (clustered sigma) the difference of
                    // two FP32 roundings would be noise and the angle would not shrink g
                    const float df = os_to_float(aqq - app);
                    const float hf = 2.0f * os_to_float(g);
                    const float adf = fabsf(df), ahf = fabsf(hf);
                    const float sz = (df == 0.0f || (df > 0.0f) == (hf > 0.0f)) ? 1.0f : -1.0f;
                    float tf;
                    if (adf >= ahf) {
                        const float z = ahf / adf;
                        tf = sz * z / (1.0f + sqrtf(fmaf(z, z, 1.0f)));
                    } else {
                        const float w = adf / ahf;
                        tf = sz / (w + sqrtf(fmaf(w, w, 1.0f)));
                    }
                    const float cf = rsqrtf(fmaf(tf, tf, 1.0f));
                    const double c0 = os_to_double(cf), s0 = os_to_double(tf * cf);
                    const double e = fma(c0, c0, fma(s0, s0, -1.0));
                    const double f = fma(e, fma(e, 0.375, -0.5), 1.0);
                    const double cs = c0 * f, sn = s0 * f;
                    for (int r = lane; r < n; r += 32) {
                        const double a = xp[r], b = xq[r];
                        xp[r] = fma(cs, a, -sn * b);
                        xq[r] = fma(sn, a, cs * b);
                    }
                    // Within a sweep the squared norms only steer later angles and tests; they
                    // follow the exact-angle update a_pp - t g, a_qq + t g.  Every sweep starts
                    // from exact norms, and the final sweep (no rotation) uses only those.
                    const double tg = os_to_double(tf) * g;
                    double np2 = app - tg, nq2 = aqq + tg;
                    __syncwarp();
                    // a norm that dropped by 16x is recomputed (cancellation in the update)
                    if (os_hi(np2) < os_hi(app) - (4 << 20)) {
                        double s2 = 0.0;
                        for (int r = lane; r < n; r += 32) s2 = fma(xp[r], xp[r], s2);
                        np2 = warp_sum(s2);
                    }
                    if (os_hi(nq2) < os_hi(aqq) - (4 << 20)) {
                        double s2 = 0.0;
                        for (int r = lane; r < n; r += 32) s2 = fma(xq[r], xq[r], s2);
                        nq2 = warp_sum(s2);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        xp[n + 1] = np2;
                        xq[n + 1] = nq2;
                        atomicAdd(&s_rot, 1);
                    }
                }
                // The links: warp P-1 (holding the last top column) moves it to the right
                // neighbour, warp 0 (holding the first bottom column) moves it to the left one,
                // each as soon as its own pair is done, by a bulk copy into the neighbour's
                // receive buffer; each receives into the buffer it sent once that copy has read it.
                const unsigned ph = (K >> 1) & 1u;
                const unsigned colb = (unsigned)(sizeof(double) * LD);
                if (warp == P - 1 && c < C - 1) {
                    __syncwarp();
                    if (lane == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        os_bulk_to(xp, recv + (size_t)(par * 2 + 0) * LD, &rbar[par][0], c + 1, colb);
                    }
                    if (!os_wait(&rbar[par][1], ph)) s_timeout = 1;
                    if (lane == 0) {
                        os_arm(&rbar[par][1], colb);  // for step K + 2
                        os_bulk_read_done();
                    }
                    __syncwarp();
                    const double* rs = recv + (size_t)(par * 2 + 1) * LD;
                    for (int r = lane; r < n + 2; r += 32) xp[r] = rs[r];
                }
                if (warp == 0 && c > 0) {
                    __syncwarp();
                    if (lane == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        os_bulk_to(xq, recv + (size_t)(par * 2 + 1) * LD, &rbar[par][1], c - 1, colb);
                    }
                    if (!os_wait(&rbar[par][0], ph)) s_timeout = 1;
                    if (lane == 0) {
                        os_arm(&rbar[par][0], colb);  // for step K + 2
                        os_bulk_read_done();
                    }
                    __syncwarp();
                    const double* rs = recv + (size_t)(par * 2 + 0) * LD;
                    for (int r = lane; r < n + 2; r += 32) xq[r] = rs[r];
                }
            }
            // circle tournament move: slot j -> j+1 (1 <= j <= np-2), slot np-1 -> 1, slot 0 fixed.
            // The buffer sent away on each link is reused for the column received on it.
            const int free_a = top[P - 1];  // sent to the right (when there is a right neighbour)
            const int free_b = bot[0];      // sent to the left
            if (tid == 0) {
                int* nt = map_top[par ^ 1];
                int* nb = map_bot[par ^ 1];
                nt[0] = (c == 0) ? top[0] : free_b;
                nt[1] = (c == 0) ? bot[0] : top[0];
                for (int u = 2; u < P; ++u) nt[u] = top[u - 1];
                for (int u = 0; u < P - 1; ++u) nb[u] = bot[u + 1];
                nb[P - 1] = (c == C - 1) ? top[P - 1] : free_a;
            }
            __syncthreads();
        }
        // cluster-wide rotation count and largest scaled |g| of this sweep
        const int sp = sweep & 1;
        if (lane == 0 && warp < P) atomicMax(&s_lmax, __float_as_int(sweep_mx));
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
        // Jacobi converges quadratically: after a sweep in which every pair's scaled |g| was
        // below 2^-20, the next sweep would normally only confirm convergence.  Instead, every
        // pair of the current columns is tested at once (the same scaled test, exact norms);
        // the sweep runs only if some pair fails.
        if (mx < 0x1p-20f && sweep < prm.max_sweeps) {
            for (int u = warp; u < 2 * P; u += blockDim.x / 32) {
                double* b = bufs + (size_t)u * LD;
                double s2 = 0.0;
                for (int r = lane; r < n; r += 32) s2 += b[r] * b[r];
                s2 = warp_sum(s2);
                if (lane == 0) b[n + 1] = s2;
            }
            cluster.sync();
            int fails = 0;
            const int slots = 2 * P;
            const int items = slots * slots * C;
            for (int it = tid; it < items; it += blockDim.x) {
                const int u = it % slots, w = (it / slots) % slots, rk = it / (slots * slots);
                const double* bu = bufs + (size_t)u * LD;
                const double* bv = cluster.map_shared_rank(bufs, rk) + (size_t)w * LD;
                const long long iu = __double_as_longlong(bu[n]), iv = __double_as_longlong(bv[n]);
                if (!(iu < iv && iv < n)) continue;
                const double au = bu[n + 1], av = bv[n + 1];
                if (!(au > 0.0 && av > 0.0)) continue;
                double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
                int r = 0;
                for (; r + 3 < n; r += 4) {
                    g0 = fma(bu[r], bv[r], g0);
                    g1 = fma(bu[r + 1], bv[r + 1], g1);
                    g2 = fma(bu[r + 2], bv[r + 2], g2);
                    g3 = fma(bu[r + 3], bv[r + 3], g3);
                }
                for (; r < n; ++r) g0 = fma(bu[r], bv[r], g0);
                const double g = (g0 + g1) + (g2 + g3);
                if (g * g > tol2 * (au * av)) ++fails;
            }
            const int cp = checks & 1;
            ++checks;
            if (fails) atomicAdd(&cluster.map_shared_rank(s_fail, 0)[cp], fails);
            cluster.sync();
            if (tid == 0) s_fail_total = cluster.map_shared_rank(s_fail, 0)[cp];
            __syncthreads();
            const int f = s_fail_total;
            if (c == 0 && tid == 0) s_fail[cp ^ 1] = 0;
            if (f == 0) { converged = true; break; }
        }
    }
    // outputs: lambda_j = ||x_j||^2, v_j = P^T x_j / ||x_j||
    for (int u = warp; u < 2 * P; u += blockDim.x / 32) {
        const double* b = bufs + (size_t)u * LD;
        const int j = (int)__double_as_longlong(b[n]);
        if (j >= n) continue;
        double s2 = 0.0;
        for (int r = lane; r < n; r += 32) s2 += b[r] * b[r];
        s2 = warp_sum(s2);
        const double nrm = sqrt(s2);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int r = lane; r < n; r += 32) prm.V[prm.perm[r] + (size_t)j * n] = b[r] * inv;
        if (lane == 0) prm.lam[j] = s2;
    }
    // info: sweeps and the largest scaled |g| seen in the last sweep
    if (lane == 0 && warp < 32) s_off[warp] = best_off;
    __syncthreads();
    if (tid == 0) {
        float off = 0.0f;
        for (int w = 0; w < P && w < 32; ++w) off = fmaxf(off, s_off[w]);
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
    cluster.sync();  // no CTA leaves while a neighbour may still read its shared memory
}

// The FP64 pipe of one SM sets the pace, so the pairs are spread over as many
// SMs as a cluster allows (16 needs the non-portable cluster size; 8 otherwise).
int cluster_size_for(int n, bool allow16) {
    if (n <= 8) return 1;
    if (n <= 16) return 2;
    if (n <= 32) return allow16 ? 8 : 4;
    return allow16 ? 16 : 8;
}

}  // namespace

size_t eig_onesided_scratch_bytes(int n) { return sizeof(double) * (size_t)n * n + sizeof(int) * 256 + 256; }

cudaError_t launch_eig_onesided(const double* M, int n, int64_t ldm, double tol, int max_sweeps,
                                void* scratch, double* lam_ws, double* V_ws, DevInfo* info,
                                cudaStream_t s) {
    if (n > 64) return cudaErrorNotSupported;
    double* X = reinterpret_cast<double*>(scratch);
    int* perm = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch) + sizeof(double) * (size_t)n * n);
    const size_t chol_smem = 2 * sizeof(double) * (size_t)n * n;
    cudaError_t e = cudaFuncSetAttribute(chol_piv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * sizeof(double) * 64 * 64));
    if (e != cudaSuccess) return e;
    chol_piv_kernel<<<1, 256, chol_smem, s>>>(M, n, ldm, X, perm, info);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    const bool allow16 =
        cudaFuncSetAttribute(onesided_jacobi_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    if (!allow16) (void)cudaGetLastError();
    int C = cluster_size_for(n, allow16);
    int np = ((n < 4 ? 4 : n) + 4 * C - 1) / (4 * C) * (4 * C);
    const int P = np / (2 * C);
    const int LD = ((n + 2) + 1) & ~1;
    const size_t smem = sizeof(double) * ((size_t)2 * P * LD + (size_t)4 * LD);
    OsParams prm{X, perm, n, np, P, tol, max_sweeps, lam_ws, V_ws, info};
    e = cudaFuncSetAttribute(onesided_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(32 * (P < 2 ? 2 : P), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, onesided_jacobi_kernel, prm);
    if (e != cudaSuccess && C == 16) {
        // the device may not schedule a 16-CTA cluster: the portable size instead
        (void)cudaGetLastError();
        C = 8;
        np = ((n < 4 ? 4 : n) + 4 * C - 1) / (4 * C) * (4 * C);
        prm.np = np;
        prm.P = np / (2 * C);
        const size_t smem8 = sizeof(double) * ((size_t)2 * prm.P * LD + (size_t)4 * LD);
        e = cudaFuncSetAttribute(onesided_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem8);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(32 * (prm.P < 2 ? 2 : prm.P), 1, 1);
        cfg.dynamicSmemBytes = smem8;
        attr[0].val.clusterDim.x = C;
        e = cudaLaunchKernelEx(&cfg, onesided_jacobi_kernel, prm);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace tsvd
