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
//      through distributed shared memory, followed by one cluster barrier.
//
// The rotation angle is estimated in FP32 while the applied rotation is kept
// orthogonal to FP64 precision (c = rsqrt(1 + t^2) in FP64): an inexact angle
// only leaves a residual g * O(2^-24) on a pair, which later sweeps remove,
// whereas a non-orthogonal rotation would change the singular values.  On
// GB300 every FP64 warp instruction occupies the thin FP64 pipe for tens of
// cycles, so the divisions and square roots of the angle go to the FP32
// units.  Squared norms are updated within a sweep by the exact quadratic
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
// One CTA.  M (n x n, ldm) -> X = R^T (n x n, ld n, lower triangular) and perm.
__global__ void __launch_bounds__(256)
    chol_piv_kernel(const double* __restrict__ M, int n, int64_t ldm, double* __restrict__ X,
                    int* __restrict__ perm_out, DevInfo* info) {
    extern __shared__ double sa[];  // [n][n] working copy (trailing Schur complement)
    __shared__ int perm[256];
    __shared__ int s_piv;
    __shared__ double s_d;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int idx = tid; idx < n * n; idx += nt) {
        const int r = idx % n, c = idx / n;
        sa[idx] = M[r + (size_t)c * ldm];
        X[idx] = 0.0;
    }
    for (int i = tid; i < n; i += nt) perm[i] = i;
    __syncthreads();
    bool deficient = false;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {  // pivot: largest remaining diagonal (lowest index on ties)
            // the bit patterns of non-negative doubles order like the values, and
            // every negative value (rank deficiency) sorts below them as a signed int
            long long best = LLONG_MIN;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const long long d = __double_as_longlong(sa[i + (size_t)i * n]);
                const long long key = d < 0 ? LLONG_MIN + 1 : d;
                if (key > best) { best = key; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) { s_piv = bi; s_d = sa[bi + (size_t)bi * n]; }
        }
        __syncthreads();
        const int p = s_piv;
        const double d = s_d;
        if (!(d > 0.0)) { deficient = true; break; }
        if (p != k) {  // symmetric swap of rows/cols k and p (trailing block) and of R's columns
            for (int i = tid; i < n; i += nt) {
                if (i >= k) {
                    const double a = sa[k + (size_t)i * n], b = sa[p + (size_t)i * n];
                    sa[k + (size_t)i * n] = b;
                    sa[p + (size_t)i * n] = a;
                }
            }
            __syncthreads();
            for (int i = tid; i < n; i += nt) {
                if (i >= k) {
                    const double a = sa[i + (size_t)k * n], b = sa[i + (size_t)p * n];
                    sa[i + (size_t)k * n] = b;
                    sa[i + (size_t)p * n] = a;
                }
                if (i < k) {  // X = R^T: row k and row p of X, columns < k
                    const double a = X[k + (size_t)i * n], b = X[p + (size_t)i * n];
                    X[k + (size_t)i * n] = b;
                    X[p + (size_t)i * n] = a;
                }
            }
            if (tid == 0) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
            __syncthreads();
        }
        const double rinv = rsqrt(d);  // 1 / r_kk
        // R[k][j] = A[k][j] / r_kk for j >= k, stored as X[j][k]
        for (int j = k + tid; j < n; j += nt)
            X[j + (size_t)k * n] = (j == k) ? d * rinv : sa[k + (size_t)j * n] * rinv;
        __syncthreads();
        // trailing update A[i][j] -= R[k][i] R[k][j], i, j > k
        const int rem = n - k - 1;
        for (int idx = tid; idx < rem * rem; idx += nt) {
            const int i = k + 1 + idx % rem, j = k + 1 + idx / rem;
            sa[i + (size_t)j * n] -= X[i + (size_t)k * n] * X[j + (size_t)k * n];
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) perm_out[i] = perm[i];
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

__global__ void __launch_bounds__(512) onesided_jacobi_kernel(OsParams prm) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int c = (int)cluster.block_rank();
    const int n = prm.n, np = prm.np, P = prm.P;
    const int LD = ((n + 2) + 1) & ~1;  // x[0..n-1], idx, nrm
    extern __shared__ double sm[];
    double* bufs = sm;                       // [2P][LD]
    double* recv = sm + (size_t)2 * P * LD;  // [2 parity][2 side][LD]
    __shared__ int top_buf[32], bot_buf[32], new_top[32], new_bot[32];
    __shared__ int s_rot;
    __shared__ unsigned long long s_off;     // bits of a non-negative double
    __shared__ int s_cnt[2];                 // used in CTA 0: per-sweep cluster totals
    __shared__ int s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = np - 1;
    const double tol2 = prm.tol * prm.tol;

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
        if (lane == 0) { b[n] = (double)col; b[n + 1] = s2; }
    }
    if (tid < P) { top_buf[tid] = tid; bot_buf[tid] = P + tid; }
    if (tid == 0) { s_cnt[0] = 0; s_cnt[1] = 0; s_off = 0ull; }
    cluster.sync();

    int sweep = 0;
    bool converged = false;
    unsigned step_par = 0;
    while (sweep < prm.max_sweeps) {
        ++sweep;
        if (tid == 0) { s_rot = 0; s_off = 0ull; }
        // exact squared norms at the start of the sweep
        for (int u = warp; u < 2 * P; u += blockDim.x / 32) {
            double* b = bufs + (size_t)u * LD;
            double s2 = 0.0;
            for (int r = lane; r < n; r += 32) s2 += b[r] * b[r];
            s2 = warp_sum(s2);
            if (lane == 0) b[n + 1] = s2;
        }
        __syncthreads();
        for (int k = 0; k < N; ++k) {
            // one warp per pair: g = x_p^T x_q, the rotation, and its application
            if (warp < P) {
                double* xp = bufs + (size_t)top_buf[warp] * LD;
                double* xq = bufs + (size_t)bot_buf[warp] * LD;
                double g = 0.0;
                for (int r = lane; r < n; r += 32) g += xp[r] * xq[r];
                g = warp_sum(g);
                const double app = xp[n + 1], aqq = xq[n + 1];
                const bool live = (int)xp[n] < n && (int)xq[n] < n && app > 0.0 && aqq > 0.0;
                const double g2 = g * g, pq = app * aqq;
                if (live && lane == 0 && g2 > __longlong_as_double((long long)s_off) * pq)
                    atomicMax(&s_off, (unsigned long long)__double_as_longlong(g2 / pq));
                if (live && g != 0.0 && g2 > tol2 * pq) {
                    // Rotation angle from Rutishauser's t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)),
                    // zeta = (a_qq - a_pp) / 2g, evaluated in FP32 (its accuracy only sets how
                    // far g is reduced); the rotation itself is made orthogonal to FP64
                    // precision by c = rsqrt(1 + t^2), s = t c computed in FP64.
                    const float df = (float)(aqq - app), hf = 2.0f * (float)g;
                    float tf;
                    if (df == 0.0f) {
                        tf = 1.0f;
                    } else {
                        const float rf = sqrtf(df * df + hf * hf);
                        tf = (df > 0.0f ? hf : -hf) / (fabsf(df) + rf);
                    }
                    const double t = (double)tf;
                    const double cs = rsqrt(1.0 + t * t);
                    const double sn = t * cs;
                    for (int r = lane; r < n; r += 32) {
                        const double a = xp[r], b = xq[r];
                        xp[r] = cs * a - sn * b;
                        xq[r] = sn * a + cs * b;
                    }
                    // ||x_p'||^2 = c^2 a_pp - 2cs g + s^2 a_qq (exact for any angle)
                    double np2 = cs * cs * app - 2.0 * cs * sn * g + sn * sn * aqq;
                    double nq2 = sn * sn * app + 2.0 * cs * sn * g + cs * cs * aqq;
                    __syncwarp();
                    if (np2 < 0.0625 * app) {
                        double s2 = 0.0;
                        for (int r = lane; r < n; r += 32) s2 += xp[r] * xp[r];
                        np2 = warp_sum(s2);
                    }
                    if (nq2 < 0.0625 * aqq) {
                        double s2 = 0.0;
                        for (int r = lane; r < n; r += 32) s2 += xq[r] * xq[r];
                        nq2 = warp_sum(s2);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        xp[n + 1] = np2;
                        xq[n + 1] = nq2;
                        atomicAdd(&s_rot, 1);
                    }
                }
            }
            __syncthreads();
            // circle tournament move: slot j -> j+1 (1 <= j <= np-2), slot np-1 -> 1, slot 0 fixed
            const int par = (int)(step_par & 1u);
            if (C > 1) {
                if (c < C - 1 && warp == 0) {  // my last top goes to the next CTA's first top
                    double* dst = cluster.map_shared_rank(recv + (size_t)(par * 2 + 0) * LD, c + 1);
                    const double* src = bufs + (size_t)top_buf[P - 1] * LD;
                    for (int r = lane; r < n + 2; r += 32) dst[r] = src[r];
                }
                if (c > 0 && warp == (blockDim.x / 32 > 1 ? 1 : 0)) {  // my first bottom goes left
                    double* dst = cluster.map_shared_rank(recv + (size_t)(par * 2 + 1) * LD, c - 1);
                    const double* src = bufs + (size_t)bot_buf[0] * LD;
                    for (int r = lane; r < n + 2; r += 32) dst[r] = src[r];
                }
                cluster.sync();
            }
            if (tid == 0) {
                // new tops
                if (c == 0) {
                    new_top[0] = top_buf[0];
                    new_top[1] = bot_buf[0];
                    for (int u = 2; u < P; ++u) new_top[u] = top_buf[u - 1];
                } else {
                    new_top[0] = -1;  // received from the left
                    for (int u = 1; u < P; ++u) new_top[u] = top_buf[u - 1];
                }
                // new bottoms
                for (int u = 0; u < P - 1; ++u) new_bot[u] = bot_buf[u + 1];
                new_bot[P - 1] = (c == C - 1) ? top_buf[P - 1] : -2;  // -2: received from the right
                // free buffers: what was sent away
                int free_a = -1, free_b = -1;
                if (c < C - 1) free_a = top_buf[P - 1];
                if (c > 0) free_b = bot_buf[0];
                if (new_top[0] == -1) new_top[0] = (free_b >= 0) ? free_b : free_a;
                if (new_bot[P - 1] == -2) new_bot[P - 1] = (free_a >= 0) ? free_a : free_b;
                for (int u = 0; u < P; ++u) { top_buf[u] = new_top[u]; bot_buf[u] = new_bot[u]; }
            }
            __syncthreads();
            if (C > 1) {
                if (c > 0 && warp == 0) {
                    const double* src = recv + (size_t)(par * 2 + 0) * LD;
                    double* dst = bufs + (size_t)top_buf[0] * LD;
                    for (int r = lane; r < n + 2; r += 32) dst[r] = src[r];
                }
                if (c < C - 1 && warp == (blockDim.x / 32 > 1 ? 1 : 0)) {
                    const double* src = recv + (size_t)(par * 2 + 1) * LD;
                    double* dst = bufs + (size_t)bot_buf[P - 1] * LD;
                    for (int r = lane; r < n + 2; r += 32) dst[r] = src[r];
                }
                __syncthreads();
            }
            ++step_par;
        }
        // cluster-wide rotation count of this sweep
        const int sp = sweep & 1;
        if (tid == 0) {
            int* cnt0 = cluster.map_shared_rank(s_cnt, 0);
            atomicAdd(&cnt0[sp], s_rot);
        }
        cluster.sync();
        if (tid == 0) {
            int* cnt0 = cluster.map_shared_rank(s_cnt, 0);
            s_total = cnt0[sp];
        }
        __syncthreads();
        const int total = s_total;
        if (c == 0 && tid == 0) s_cnt[sp ^ 1] = 0;
        if (total == 0) { converged = true; break; }
    }
    // outputs: lambda_j = ||x_j||^2, v_j = P^T x_j / ||x_j||
    for (int u = warp; u < 2 * P; u += blockDim.x / 32) {
        const double* b = bufs + (size_t)u * LD;
        const int j = (int)b[n];
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
    if (tid == 0) {
        unsigned long long* off0 = cluster.map_shared_rank(&s_off, 0);
        if (c != 0) atomicMax(off0, s_off);
    }
    cluster.sync();
    if (c == 0 && tid == 0) {
        prm.info->sweeps = sweep;
        prm.info->off_norm = sqrt(__longlong_as_double((long long)s_off));
        if (!converged) atomicOr(&prm.info->flags, FLAG_NO_CONVERGENCE);
    }
}

int cluster_size_for(int n) {
    if (n <= 8) return 1;
    if (n <= 16) return 2;
    if (n <= 32) return 4;
    return 8;
}

}  // namespace

size_t eig_onesided_scratch_bytes(int n) { return sizeof(double) * (size_t)n * n + sizeof(int) * 256 + 256; }

cudaError_t launch_eig_onesided(const double* M, int n, int64_t ldm, double tol, int max_sweeps,
                                void* scratch, double* lam_ws, double* V_ws, DevInfo* info,
                                cudaStream_t s) {
    if (n > 64) return cudaErrorNotSupported;
    double* X = reinterpret_cast<double*>(scratch);
    int* perm = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch) + sizeof(double) * (size_t)n * n);
    const size_t chol_smem = sizeof(double) * (size_t)n * n;
    cudaError_t e = cudaFuncSetAttribute(chol_piv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * 64 * 64));
    if (e != cudaSuccess) return e;
    chol_piv_kernel<<<1, 256, chol_smem, s>>>(M, n, ldm, X, perm, info);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    const int C = cluster_size_for(n);
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
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace tsvd
