// eig_alg2.cu -- Algorithm 2 of the paper (its mixed precision eigensolver for
// the Gram matrix) as an n x n stage, n <= 64, FP32 working precision:
//   line 1  plain Cholesky M_h = R_h^T R_h at the higher precision (FP64,
//           launch_cholesky without pivoting),
//   line 2  R = RN_32(R_h),
//   line 3  SVD of R at the working precision: one-sided Jacobi in FP32 on the
//           columns of R with the rotations accumulated (R J = U_R Sigma, V = J);
//           then M_h ~= V Sigma^2 V^T.  The columns of R carry the column
//           scaling D of A = B D (R = R_C D), which one-sided Jacobi on columns
//           resolves to relative accuracy u kappa(B).
// Accuracy (Remark 2): O(u) kappa(B) + O(u_h) kappa(B)^2, against O(u) +
// O(u_h) kappa(B)^2 for the FP64 eigen stages.  Speed: FP32 has ~14x lower
// latency and ~60x the throughput of FP64 on GB300, so one CTA holds the whole
// factor in shared memory and needs no cluster.
//
// One CTA, one warp per column pair (round-robin "circle" tournament over the
// n rounded up to even columns, column 0 fixed; every warp finds its pair's columns
// from the step count), lane l holds rows l and l + 32;
// per step: g = x_p^T x_q and both squared norms in FP32 (one reduction of three
// values), the scaled skip test |g| <= tol ||x_p|| ||x_q||, Rutishauser's angle,
// the rotation of the two columns and of the same two columns of V.  A sweep
// without rotation ends the iteration.  The squared norms of the final columns
// are summed in FP64 from the FP32 entries.
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int A2_ROWS = 64;

__device__ __forceinline__ float a2_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(1024)
    alg2_jacobi_kernel(const double* __restrict__ X, const int* __restrict__ perm, int n, int np, float tol,
                       int max_sweeps, double* __restrict__ lam, double* __restrict__ V, DevInfo* info) {
    __shared__ float col[64][A2_ROWS];  // column c of R, cast to FP32
    __shared__ float vcol[64][A2_ROWS]; // column c of V = J (the accumulated rotations)
    __shared__ int s_rot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = np / 2;
    for (int idx = tid; idx < 64 * A2_ROWS; idx += blockDim.x) {
        const int c = idx / A2_ROWS, r = idx % A2_ROWS;
        // R[r][c] = X[c][r] (X = R^T, ld n); Alg. 2 line 2: RN to FP32
        col[c][r] = (c < n && r < n) ? (float)X[c + (size_t)r * n] : 0.0f;
        vcol[c][r] = (c == r) ? 1.0f : 0.0f;
    }
    __syncthreads();
    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        ++sweep;
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int k = 0; k < np - 1; ++k) {
            if (warp < P) {
                // circle tournament in closed form: position 0 keeps column 0, position p >= 1
                // holds after k steps the column that started at 1 + ((p - 1 - k) mod (np - 1))
                const int L = np - 1;
                const int cp = warp == 0 ? 0 : 1 + ((warp - 1 - k) % L + L) % L;
                const int cq = 1 + ((np - 2 - warp - k) % L + L) % L;
                float* xp = col[cp];
                float* xq = col[cq];
                const float p0 = xp[lane], p1 = xp[lane + 32], q0 = xq[lane], q1 = xq[lane + 32];
                const float g = a2_sum(fmaf(p0, q0, p1 * q1));
                const float a = a2_sum(fmaf(p0, p0, p1 * p1));
                const float b = a2_sum(fmaf(q0, q0, q1 * q1));
                if (cp < n && cq < n && a > 0.0f && b > 0.0f && fabsf(g) > tol * sqrtf(a) * sqrtf(b)) {
                    // t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / 2g, sgn(0) = +1,
                    // from ratios <= 1
                    const float df = b - a, hf = 2.0f * g;
                    const float adf = fabsf(df), ahf = fabsf(hf);
                    const float sz = (df == 0.0f || (df > 0.0f) == (hf > 0.0f)) ? 1.0f : -1.0f;
                    float t;
                    if (adf >= ahf) {
                        const float z = ahf / adf;
                        t = sz * z / (1.0f + sqrtf(fmaf(z, z, 1.0f)));
                    } else {
                        const float w = adf / ahf;
                        t = sz / (w + sqrtf(fmaf(w, w, 1.0f)));
                    }
                    const float cs = rsqrtf(fmaf(t, t, 1.0f)), sn = t * cs;
                    xp[lane] = fmaf(cs, p0, -sn * q0);
                    xp[lane + 32] = fmaf(cs, p1, -sn * q1);
                    xq[lane] = fmaf(sn, p0, cs * q0);
                    xq[lane + 32] = fmaf(sn, p1, cs * q1);
                    float* vp = vcol[cp];
                    float* vq = vcol[cq];
                    const float a0 = vp[lane], a1 = vp[lane + 32], b0 = vq[lane], b1 = vq[lane + 32];
                    vp[lane] = fmaf(cs, a0, -sn * b0);
                    vp[lane + 32] = fmaf(cs, a1, -sn * b1);
                    vq[lane] = fmaf(sn, a0, cs * b0);
                    vq[lane + 32] = fmaf(sn, a1, cs * b1);
                    if (lane == 0) atomicAdd(&s_rot, 1);
                }
            }
            __syncthreads();
        }
        if (s_rot == 0) { converged = true; break; }
        __syncthreads();  // every thread has read s_rot before the next sweep clears it
    }
    // lambda_j = ||r_j||^2 of the final columns (FP64 sum of the FP32 entries); v_j = column j
    // of J, by original index
    for (int c = warp; c < n; c += blockDim.x >> 5) {
        const double r0 = (double)col[c][lane], r1 = (double)col[c][lane + 32];
        double s2 = fma(r0, r0, r1 * r1);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane < n) V[perm[lane] + (size_t)c * n] = (double)vcol[c][lane];
        if (lane + 32 < n) V[perm[lane + 32] + (size_t)c * n] = (double)vcol[c][lane + 32];
        if (lane == 0) lam[c] = s2;
    }
    if (tid == 0) {
        info->sweeps = sweep;
        if (!converged) atomicOr(&info->flags, FLAG_NO_CONVERGENCE);
    }
}

}  // namespace

cudaError_t launch_eig_alg2(const double* M, int n, int64_t ldm, float tol, int max_sweeps, void* scratch,
                            double* lam_ws, double* V_ws, DevInfo* info, cudaStream_t s) {
    if (n > 64) return cudaErrorNotSupported;
    double* X = reinterpret_cast<double*>(scratch);
    int* perm = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch) + sizeof(double) * (size_t)n * n);
    cudaError_t e = launch_cholesky(M, n, ldm, X, perm, info, false, s);
    if (e != cudaSuccess) return e;
    const int np = n < 2 ? 2 : n + (n & 1);
    alg2_jacobi_kernel<<<1, 32 * (np / 2), 0, s>>>(X, perm, n, np, tol, max_sweeps, lam_ws, V_ws, info);
    return cudaGetLastError();
}

}  // namespace tsvd
