// jacobi.cu -- the n x n eigen stage (Alg. 1 lines 3-5; Sec. 2.1, Remark 1).
//
// Two-sided Jacobi on the symmetric positive definite M_h in FP64.  One CTA
// runs the parallel (round-robin tournament) ordering: in each of the n'-1
// steps of a sweep (n' = n rounded up to even) the n'/2 disjoint pairs are
// rotated together, M <- J^T M J and V <- V J, with the rotation of each
// pair computed from the step's starting M by Rutishauser's formulas
//   zeta = (m_qq - m_pp) / (2 m_pq),  t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2),  s = t c,
// and the 2x2 block set to diag(m_pp - t m_pq, m_qq + t m_pq).  A pair is
// skipped when |m_pq| <= tol * sqrt(m_pp m_qq): the stopping test is scaled
// by the column norms D = diag(M)^(1/2) of A = B D (Sec. 3), which is what
// gives eigenvalues of high relative accuracy.  The sweep loop ends after a
// sweep without any rotation (or at max_sweeps: TSVD_ERR_NO_CONVERGENCE).
//
// The finish kernel sorts lambda descending, applies the sign rule, takes
// sigma = sqrt(lambda) in FP64 and rounds sigma and V to working precision
// (RN-even), and forms W = RN(V / sigma) column by column for line 6.
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int JAC_MAX_PAIRS = 128;  // n <= 256

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

__global__ void __launch_bounds__(512)
    jacobi_kernel(const double* __restrict__ M_in, int n, int64_t ldm, double tol, int max_sweeps,
                  double* __restrict__ scratch, double* __restrict__ lam_ws,
                  double* __restrict__ V_ws, DevInfo* info) {
    extern __shared__ double sm[];
    const bool in_smem = (n <= 64);
    double* Mx = in_smem ? sm : scratch;
    double* Vx = in_smem ? sm + (size_t)n * n : V_ws;
    __shared__ double s_c[JAC_MAX_PAIRS], s_s[JAC_MAX_PAIRS], s_t[JAC_MAX_PAIRS];
    __shared__ double s_mpq[JAC_MAX_PAIRS], s_mpp[JAC_MAX_PAIRS], s_mqq[JAC_MAX_PAIRS];
    __shared__ int s_p[JAC_MAX_PAIRS], s_q[JAC_MAX_PAIRS], s_rot[JAC_MAX_PAIRS];
    __shared__ int s_count;
    __shared__ double s_off;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int idx = tid; idx < n * n; idx += nt) {
        const int r = idx % n, c = idx / n;
        Mx[idx] = M_in[r + (size_t)c * ldm];
        Vx[idx] = (r == c) ? 1.0 : 0.0;
    }
    if (tid == 0) s_off = 0.0;
    __syncthreads();

    const int np = n + (n & 1);
    const int N = np - 1;  // steps per sweep
    const int npairs = np / 2;
    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        ++sweep;
        if (tid == 0) s_count = 0;
        __syncthreads();
        for (int k = 0; k < N; ++k) {
            for (int pr = tid; pr < npairs; pr += nt) {
                int a, b;
                if (pr == 0) { a = N; b = k; }
                else { a = (k + pr) % N; b = (k - pr + N) % N; }
                const int p = min(a, b), q = max(a, b);
                int rot = 0;
                double c = 1.0, s = 0.0, t = 0.0, mpq = 0.0, mpp = 0.0, mqq = 0.0;
                if (q < n && N > 0) {
                    mpq = Mx[p + (size_t)q * n];
                    mpp = Mx[p + (size_t)p * n];
                    mqq = Mx[q + (size_t)q * n];
                    if (mpq != 0.0 && fabs(mpq) > tol * sqrt(fabs(mpp * mqq))) {
                        const double zeta = (mqq - mpp) / (2.0 * mpq);
                        const double sg = zeta >= 0.0 ? 1.0 : -1.0;
                        t = sg / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        rot = 1;
                    }
                }
                s_p[pr] = p; s_q[pr] = q; s_c[pr] = c; s_s[pr] = s; s_t[pr] = t;
                s_mpq[pr] = mpq; s_mpp[pr] = mpp; s_mqq[pr] = mqq; s_rot[pr] = rot;
                if (rot) atomicAdd(&s_count, 1);
            }
            __syncthreads();
            // M <- M J and V <- V J (columns p, q of every pair)
            for (int idx = tid; idx < npairs * n; idx += nt) {
                const int pr = idx / n, r = idx - pr * n;
                if (!s_rot[pr]) continue;
                const int p = s_p[pr], q = s_q[pr];
                const double c = s_c[pr], s = s_s[pr];
                const double xp = Mx[r + (size_t)p * n], xq = Mx[r + (size_t)q * n];
                Mx[r + (size_t)p * n] = c * xp - s * xq;
                Mx[r + (size_t)q * n] = s * xp + c * xq;
                const double vp = Vx[r + (size_t)p * n], vq = Vx[r + (size_t)q * n];
                Vx[r + (size_t)p * n] = c * vp - s * vq;
                Vx[r + (size_t)q * n] = s * vp + c * vq;
            }
            __syncthreads();
            // M <- J^T M (rows p, q of every pair)
            for (int idx = tid; idx < npairs * n; idx += nt) {
                const int pr = idx / n, col = idx - pr * n;
                if (!s_rot[pr]) continue;
                const int p = s_p[pr], q = s_q[pr];
                const double c = s_c[pr], s = s_s[pr];
                const double xp = Mx[p + (size_t)col * n], xq = Mx[q + (size_t)col * n];
                Mx[p + (size_t)col * n] = c * xp - s * xq;
                Mx[q + (size_t)col * n] = s * xp + c * xq;
            }
            __syncthreads();
            for (int pr = tid; pr < npairs; pr += nt) {
                if (!s_rot[pr]) continue;
                const int p = s_p[pr], q = s_q[pr];
                const double t = s_t[pr], mpq = s_mpq[pr];
                Mx[p + (size_t)p * n] = s_mpp[pr] - t * mpq;
                Mx[q + (size_t)q * n] = s_mqq[pr] + t * mpq;
                Mx[p + (size_t)q * n] = 0.0;
                Mx[q + (size_t)p * n] = 0.0;
            }
            __syncthreads();
        }
        const int cnt = s_count;
        __syncthreads();
        if (cnt == 0) { converged = true; break; }
    }
    // scaled off-diagonal norm at exit
    for (int idx = tid; idx < n * n; idx += nt) {
        const int r = idx % n, c = idx / n;
        if (r < c) {
            const double d = sqrt(fabs(Mx[r + (size_t)r * n] * Mx[c + (size_t)c * n]));
            const double v = d > 0.0 ? fabs(Mx[idx]) / d : 0.0;
            atomic_max_nonneg(&s_off, v);
        }
    }
    for (int i = tid; i < n; i += nt) lam_ws[i] = Mx[i + (size_t)i * n];
    if (in_smem)
        for (int idx = tid; idx < n * n; idx += nt) V_ws[idx] = Vx[idx];
    __syncthreads();
    if (tid == 0) {
        info->sweeps = sweep;
        info->off_norm = s_off;
        if (!converged) atomicOr(&info->flags, FLAG_NO_CONVERGENCE);
    }
}

template <typename WT>
__global__ void __launch_bounds__(256)
    finish_kernel(const double* __restrict__ lam, const double* __restrict__ V, int n,
                  WT* __restrict__ sigma_w, WT* __restrict__ V_w, int64_t ldv, WT* __restrict__ W_w,
                  double* __restrict__ lam_sorted, double* __restrict__ V_sorted, int64_t ld_vs,
                  DevInfo* info, double uh) {
    __shared__ int order[256];
    __shared__ double sig[256];
    __shared__ double sgn[256];
    const int tid = threadIdx.x;
    if (tid < n) {
        const double li = lam[tid];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = lam[j];
            if (lj > li || (lj == li && j < tid)) ++rank;
        }
        order[rank] = tid;
    }
    __syncthreads();
    if (tid < n) {
        const int src = order[tid];
        const double l = lam[src];
        if (!(l > 0.0)) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
        sig[tid] = l > 0.0 ? sqrt(l) : 0.0;
        int best = 0;
        double bv = fabs(V[(size_t)src * n]);
        for (int r = 1; r < n; ++r) {
            const double v = fabs(V[r + (size_t)src * n]);
            if (v > bv) { bv = v; best = r; }
        }
        sgn[tid] = V[best + (size_t)src * n] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    if (tid == 0 && n > 1 && sig[n - 1] < uh * sig[0])
        atomicOr(&info->flags, FLAG_NOT_FULL_RANK);  // sigma_n / sigma_1 below u_h
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx % n, k = idx / n;
        const int src = order[k];
        const double v = sgn[k] * V[r + (size_t)src * n];
        if (V_sorted) V_sorted[r + (size_t)k * ld_vs] = v;
        const WT vw = (WT)v;
        if (V_w) V_w[r + (size_t)k * ldv] = vw;
        if (W_w) {
            const WT sw = (WT)sig[k];
            W_w[r + (size_t)k * n] = vw / sw;
        }
    }
    if (tid < n) {
        if (sigma_w) sigma_w[tid] = (WT)sig[tid];
        if (lam_sorted) lam_sorted[tid] = lam[order[tid]];
    }
}

__global__ void finalize_info_kernel(DevInfo* info) {
    const int f = info->flags;
    int st = TSVD_OK;
    if (f & FLAG_NONFINITE) st = TSVD_ERR_NONFINITE;
    else if (f & FLAG_BAD_SCALE) st = TSVD_ERR_ARG;
    else if (f & FLAG_TIMEOUT) st = TSVD_ERR_TIMEOUT;
    else if (f & FLAG_NOT_FULL_RANK) st = TSVD_ERR_NOT_FULL_RANK;
    else if (f & FLAG_NO_CONVERGENCE) st = TSVD_ERR_NO_CONVERGENCE;
    info->flags = st;
}

}  // namespace

cudaError_t launch_jacobi(const double* M, int n, int64_t ldm, double tol, int max_sweeps,
                          double* scratch, double* lam_ws, double* V_ws, DevInfo* info,
                          cudaStream_t s) {
    if (n > 256) return cudaErrorNotSupported;
    const bool in_smem = n <= 64;
    const size_t smem = in_smem ? 2 * sizeof(double) * n * n : 0;
    cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * sizeof(double) * 64 * 64));
    if (e != cudaSuccess) return e;
    const int threads = in_smem ? 256 : 512;
    jacobi_kernel<<<1, threads, smem, s>>>(M, n, ldm, tol, max_sweeps, scratch, lam_ws, V_ws, info);
    return cudaGetLastError();
}

cudaError_t launch_finish(const double* lam_ws, const double* V_ws, int n, int working,
                          void* sigma_w, void* V_w, int64_t ldv, void* W_w, double* lam_sorted,
                          double* V_sorted, int64_t ld_vs, DevInfo* info, cudaStream_t s, double uh) {
    if (n > 256) return cudaErrorNotSupported;
    if (working == 0)
        finish_kernel<float><<<1, 256, 0, s>>>(lam_ws, V_ws, n, (float*)sigma_w, (float*)V_w, ldv,
                                               (float*)W_w, lam_sorted, V_sorted, ld_vs, info, uh);
    else
        finish_kernel<double><<<1, 256, 0, s>>>(lam_ws, V_ws, n, (double*)sigma_w, (double*)V_w,
                                                ldv, (double*)W_w, lam_sorted, V_sorted, ld_vs, info, uh);
    return cudaGetLastError();
}

cudaError_t launch_finalize_info(DevInfo* info, cudaStream_t s) {
    finalize_info_kernel<<<1, 1, 0, s>>>(info);
    return cudaGetLastError();
}

}  // namespace tsvd
