// eig_dd.cu -- the eigen stage of Alg. 1 (lines 3-5) in double-double for FP64
// working precision (u_h ~ 2^-104), in the preconditioned form of Alg. 2:
// a pivoted Cholesky P^T M P = R^T R, then a one-sided Jacobi SVD of X = R^T
// (Hestenes), whose converged columns y_c give lambda_c = |y_c|^2 and the
// eigenvectors of P^T M P as y_c / |y_c| (no rotation is accumulated).
//
// One CTA of 256 threads, n <= 64, M and then X in shared memory as (hi, lo)
// pairs.  Column pairs follow the round-robin tournament (n/2 disjoint pairs
// per round, n - 1 rounds per sweep); each pair is handled by a group of 8
// lanes, each owning every 8th row.  The double-double operations keep an
// absolute error of a few 2^-105 times the size of their operands, which is
// the rounding model of the usual Jacobi error analysis with u = 2^-104.
//
// Rotation (p, q): with alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p . x_q,
// the pair is skipped when |gamma| <= tol sqrt(alpha beta); otherwise
// zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
// (FP64 suffices: an inexact angle only leaves a smaller gamma for the next
// sweep), and the applied rotation c = 1 / sqrt(1 + t^2), s = t c is formed in
// double-double so that it is orthogonal to 2^-104:
//     x_p <- c x_p - s x_q,   x_q <- s x_p + c x_q,
//     alpha <- alpha - t gamma,   beta <- beta + t gamma.
// The norms are recomputed from the columns at the start of every sweep.
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int DD_THREADS = 256;
constexpr int DD_GROUP = 8;  // lanes per column pair

struct dd {
    double h, l;
};

__device__ __forceinline__ dd quick_two_sum(double a, double b) {
    const double s = a + b;
    return {s, b - (s - a)};
}

// a + b, absolute error ~ 2^-105 (|a| + |b|)
__device__ __forceinline__ dd add(dd a, dd b) {
    const double s = a.h + b.h;
    const double bb = s - a.h;
    double e = (a.h - (s - bb)) + (b.h - bb);
    e += a.l + b.l;
    return quick_two_sum(s, e);
}
__device__ __forceinline__ dd neg(dd a) { return {-a.h, -a.l}; }

// a * b, left unnormalised (|l| may reach a few ulps of h); add() accepts it
__device__ __forceinline__ dd mul_raw(dd a, dd b) {
    const double p = a.h * b.h;
    double e = fma(a.h, b.h, -p);
    e = fma(a.h, b.l, e);
    e = fma(a.l, b.h, e);
    return {p, e};
}
__device__ __forceinline__ dd mul_d(dd a, double b) {
    const double p = a.h * b;
    double e = fma(a.h, b, -p);
    e = fma(a.l, b, e);
    return quick_two_sum(p, e);
}

// a / b (b > 0 or b < 0, normalised operands)
__device__ __forceinline__ dd div(dd a, dd b) {
    const double q1 = a.h / b.h;
    const double p = q1 * b.h;
    const double e = fma(q1, b.h, -p) + q1 * b.l;
    const double r = ((a.h - p) - e) + a.l;
    return quick_two_sum(q1, r / b.h);
}

// sqrt(a), a > 0
__device__ __forceinline__ dd sqrt_dd(dd a) {
    const double r0 = sqrt(a.h);
    const double res = fma(-r0, r0, a.h) + a.l;
    return quick_two_sum(r0, res / (2.0 * r0));
}

// The 8 lanes of a group take their branches together, but the groups of one
// warp need not (a pair may be skipped): every shuffle names its group only.
__device__ __forceinline__ unsigned group_mask() { return 0xffu << (threadIdx.x & 24); }
__device__ __forceinline__ dd shfl_xor(dd a, int o, unsigned mask) {
    return {__shfl_xor_sync(mask, a.h, o), __shfl_xor_sync(mask, a.l, o)};
}
__device__ __forceinline__ dd group_sum(dd a) {
    const unsigned mask = group_mask();
#pragma unroll
    for (int o = DD_GROUP / 2; o > 0; o >>= 1) a = add(a, shfl_xor(a, o, mask));
    return a;
}

// player at position pos of round r in the circle method over N players
__device__ __forceinline__ int player(int pos, int r, int N) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (N - 1); }

__global__ void __launch_bounds__(DD_THREADS, 1)
    eig_dd_kernel(const double* __restrict__ G, const double* __restrict__ G_lo, int n, int64_t ldm, double tol,
                  int max_sweeps, double* __restrict__ lam_ws, double* __restrict__ V_ws, DevInfo* info) {
    extern __shared__ double sm[];
    const int LD = n + 1;
    double* Mh = sm;              // [n][LD]: M, then R's rows = the columns of X
    double* Ml = sm + n * LD;
    __shared__ dd nrm[64];
    __shared__ int perm[64];
    __shared__ int s_piv, s_fail;
    __shared__ dd s_rkk;
    __shared__ int s_count[2];
    __shared__ unsigned long long s_off;
    const int tid = threadIdx.x;

    for (int idx = tid; idx < n * n; idx += DD_THREADS) {
        const int i = idx % n, j = idx / n;
        Mh[i * LD + j] = G[i + (size_t)j * ldm];
        Ml[i * LD + j] = G_lo ? G_lo[i + (size_t)j * ldm] : 0.0;
    }
    if (tid < n) perm[tid] = tid;
    if (tid == 0) {
        s_fail = 0;
        s_count[0] = s_count[1] = 0;
        s_off = 0ull;
    }
    __syncthreads();

    // ---- pivoted Cholesky, in place: row k of Mh/Ml becomes row k of R
    int k = 0;
    for (; k < n; ++k) {
        if (tid < 32) {
            double bv = -1.0;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const double v = Mh[i * LD + i];
                if (v > bv) { bv = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (tid == 0) {
                s_piv = bi;
                if (!(bv > 0.0) || !isfinite(bv)) s_fail = 1;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const int p = s_piv;
        if (p != k) {
            for (int j = tid; j < n; j += DD_THREADS) {
                double t = Mh[k * LD + j]; Mh[k * LD + j] = Mh[p * LD + j]; Mh[p * LD + j] = t;
                t = Ml[k * LD + j]; Ml[k * LD + j] = Ml[p * LD + j]; Ml[p * LD + j] = t;
            }
            __syncthreads();
            for (int i = tid; i < n; i += DD_THREADS) {
                double t = Mh[i * LD + k]; Mh[i * LD + k] = Mh[i * LD + p]; Mh[i * LD + p] = t;
                t = Ml[i * LD + k]; Ml[i * LD + k] = Ml[i * LD + p]; Ml[i * LD + p] = t;
            }
            if (tid == 0) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
            __syncthreads();
        }
        if (tid == 0) s_rkk = sqrt_dd(dd{Mh[k * LD + k], Ml[k * LD + k]});
        __syncthreads();
        const dd rkk = s_rkk;
        for (int j = k + 1 + tid; j < n; j += DD_THREADS) {
            const dd r = div(dd{Mh[k * LD + j], Ml[k * LD + j]}, rkk);
            Mh[k * LD + j] = r.h;
            Ml[k * LD + j] = r.l;
        }
        if (tid == 0) { Mh[k * LD + k] = rkk.h; Ml[k * LD + k] = rkk.l; }
        __syncthreads();
        const int t = n - k - 1;
        for (int idx = tid; idx < t * t; idx += DD_THREADS) {
            const int i = k + 1 + idx % t, j = k + 1 + idx / t;
            const dd upd = mul_raw(dd{Mh[k * LD + i], Ml[k * LD + i]}, dd{Mh[k * LD + j], Ml[k * LD + j]});
            const dd r = add(dd{Mh[i * LD + j], Ml[i * LD + j]}, neg(upd));
            Mh[i * LD + j] = r.h;
            Ml[i * LD + j] = r.l;
        }
        __syncthreads();
    }
    // rows >= k of R stay zero when the factorisation stopped early (rank deficient)
    for (int idx = tid; idx < n * n; idx += DD_THREADS) {
        const int c = idx / n, r = idx % n;
        if (r < c || c >= k) { Mh[c * LD + r] = 0.0; Ml[c * LD + r] = 0.0; }
    }
    if (tid == 0 && k < n) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
    __syncthreads();

    // ---- one-sided Jacobi on the columns x_c = row c of R
    const int N = (n + 1) & ~1;
    const int grp = tid / DD_GROUP, gl = tid % DD_GROUP;
    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        // column norms from the columns themselves, then tracked through the sweep
        for (int c = grp; c < n; c += DD_THREADS / DD_GROUP) {
            dd a{0.0, 0.0};
            for (int i = gl; i < n; i += DD_GROUP) {
                const dd x{Mh[c * LD + i], Ml[c * LD + i]};
                a = add(a, mul_raw(x, x));
            }
            a = group_sum(a);
            if (gl == 0) nrm[c] = a;
        }
        if (tid == 0) s_off = 0ull;
        __syncthreads();
        unsigned long long off_bits = 0ull;
        for (int r = 0; r < N - 1; ++r) {
            if (grp < N / 2) {
                int p = player(grp, r, N), q = player(N - 1 - grp, r, N);
                if (p > q) { const int t = p; p = q; q = t; }
                if (q < n) {
                    double* xph = Mh + p * LD; double* xpl = Ml + p * LD;
                    double* xqh = Mh + q * LD; double* xql = Ml + q * LD;
                    dd g{0.0, 0.0};
                    for (int i = gl; i < n; i += DD_GROUP) g = add(g, mul_raw(dd{xph[i], xpl[i]}, dd{xqh[i], xql[i]}));
                    g = group_sum(g);
                    dd a = nrm[p], b = nrm[q];
                    const double scale = sqrt(a.h) * sqrt(b.h);
                    const double ratio = scale > 0.0 ? fabs(g.h) / scale : 0.0;
                    if (ratio > tol) {
                        const double d = add(b, neg(a)).h;
                        const double zeta = d / (2.0 * g.h);
                        const double az = fabs(zeta);
                        double t = az > 1e150 ? 0.5 / az : 1.0 / (az + sqrt(fma(az, az, 1.0)));
                        t = copysign(t, zeta);
                        // c = 1 / sqrt(1 + t^2), s = t c in double-double
                        const double tt = t * t;
                        const dd one_tt = add(dd{1.0, 0.0}, dd{tt, fma(t, t, -tt)});
                        const dd c = div(dd{1.0, 0.0}, sqrt_dd(one_tt));
                        const dd s = mul_d(c, t);
                        for (int i = gl; i < n; i += DD_GROUP) {
                            const dd xp{xph[i], xpl[i]}, xq{xqh[i], xql[i]};
                            const dd np = add(mul_raw(c, xp), neg(mul_raw(s, xq)));
                            const dd nq = add(mul_raw(s, xp), mul_raw(c, xq));
                            xph[i] = np.h; xpl[i] = np.l;
                            xqh[i] = nq.h; xql[i] = nq.l;
                        }
                        const dd tg = mul_d(g, t);
                        a = add(a, neg(tg));
                        b = add(b, tg);
                        if (gl == 0) {
                            nrm[p] = a;
                            nrm[q] = b;
                            atomicAdd(&s_count[sweep & 1], 1);
                        }
                    }
                    if (gl == 0) off_bits = max(off_bits, (unsigned long long)__double_as_longlong(ratio));
                }
            }
            __syncthreads();
        }
        if (off_bits) atomicMax(&s_off, off_bits);
        ++sweep;
        const int cnt = s_count[(sweep - 1) & 1];
        __syncthreads();
        if (tid == 0) s_count[(sweep - 1) & 1] = 0;
        if (cnt == 0) {
            converged = true;
            break;
        }
    }

    // ---- lambda_c = |x_c|^2, V (by original index) = x_c / |x_c|
    for (int c = grp; c < n; c += DD_THREADS / DD_GROUP) {
        dd a{0.0, 0.0};
        for (int i = gl; i < n; i += DD_GROUP) {
            const dd x{Mh[c * LD + i], Ml[c * LD + i]};
            a = add(a, mul_raw(x, x));
        }
        a = group_sum(a);
        const double nrm_c = a.h > 0.0 ? sqrt(a.h) : 0.0;
        if (gl == 0) lam_ws[c] = a.h;
        for (int i = gl; i < n; i += DD_GROUP) {
            const dd x{Mh[c * LD + i], Ml[c * LD + i]};
            V_ws[perm[i] + (size_t)c * n] = nrm_c > 0.0 ? div(x, dd{nrm_c, 0.0}).h : (perm[i] == c ? 1.0 : 0.0);
        }
    }
    if (tid == 0) {
        info->sweeps = sweep;
        info->off_norm = __longlong_as_double((long long)s_off);
        if (!converged) atomicOr(&info->flags, FLAG_NO_CONVERGENCE);
    }
}

}  // namespace

cudaError_t launch_eig_dd(const double* M, const double* M_lo, int n, int64_t ldm, double tol, int max_sweeps,
                          double* lam_ws, double* V_ws, DevInfo* info, cudaStream_t s) {
    if (n < 1 || n > 64) return cudaErrorInvalidValue;
    const size_t smem = 2 * sizeof(double) * (size_t)n * (n + 1);
    cudaError_t e = cudaFuncSetAttribute(eig_dd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    eig_dd_kernel<<<1, DD_THREADS, smem, s>>>(M, M_lo, n, ldm, tol, max_sweeps, lam_ws, V_ws, info);
    return cudaGetLastError();
}

}  // namespace tsvd
