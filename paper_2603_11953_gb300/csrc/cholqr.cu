// cholqr.cu -- the mixed precision Cholesky QR algorithm that motivates the
// paper (Sec. 3.1 and Theorem 3), on the same Gram kernels:
//   1. M_h = A^T A at the higher precision (the tensor-core Gram),
//   2. M_h = R^T R by the plain Cholesky factorization in FP64,
//   3. Q from the linear systems Q R = A at the working precision: every row
//      q of Q solves q R_w = a by forward substitution in FP32, R_w = RN_32(R).
// With u_h = 2^-53 <= u^2 (u = 2^-24), Theorem 3 bounds ||Q^T Q - I|| by
// O(u) kappa(B) instead of the O(u) kappa(B)^2 of a same-precision Cholesky QR.
//
// cholqr_q_kernel: one thread per row, the row's n running values in registers, R_w in shared
// memory with its rows contiguous (entry (j, k) at Rw[j][k]).  Right-looking order: once q_j =
// s_j / r_jj is known, every s_k (k > j) takes its term -q_j r_jk, so a step's FMAs are
// independent of each other and the dependent chain is n divisions long instead of n^2 / 2
// FMAs.  Each s_k still receives its terms in the order of j, so the result is bitwise that of
// the left-looking substitution.  16-byte shared loads broadcast four entries of row j to the
// warp.  A is read once and Q written once (coalesced: consecutive threads hold consecutive rows
// of the column-major arrays).
#include "internal.cuh"

namespace tsvd {
namespace {

template <int NP>
__global__ void __launch_bounds__(256)
    cholqr_q_kernel(const float* __restrict__ A, int64_t m, int n, int64_t lda, const double* __restrict__ X,
                    float* __restrict__ Q, int64_t ldq) {
    __shared__ __align__(16) float Rw[NP][NP];  // Rw[j][k] = RN_32(R[j][k]), j <= k < n; zero elsewhere
    __shared__ float Rd[NP];                     // the diagonal
    for (int idx = threadIdx.x; idx < NP * NP; idx += blockDim.x) {
        const int j = idx / NP, k = idx % NP;
        // X = R^T with ld n: R[j][k] = X[k + j n]
        Rw[j][k] = (j <= k && k < n) ? (float)X[k + (size_t)j * n] : 0.0f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NP; j += blockDim.x) Rd[j] = j < n ? Rw[j][j] : 1.0f;
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        float s[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) s[j] = j < n ? A[r + (size_t)j * lda] : 0.0f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            // q_j = (a_j - sum_{i<j} q_i r_ij) / r_jj, the sum in FP32 in the order of i
            s[j] = s[j] / Rd[j];
            // one row of R_w at a time in registers (the compiler would otherwise hoist the loads
            // of all rows)
            asm volatile("" ::: "memory");
            const float4* row = reinterpret_cast<const float4*>(Rw[j]);
#pragma unroll
            for (int k4 = (j + 1) / 4; k4 < NP / 4; ++k4) {
                if ((k4 & 3) == 0) asm volatile("" ::: "memory");  // at most four loads ahead
                const float4 c = row[k4];
                if (4 * k4 + 0 > j) s[4 * k4 + 0] = fmaf(-s[j], c.x, s[4 * k4 + 0]);
                if (4 * k4 + 1 > j) s[4 * k4 + 1] = fmaf(-s[j], c.y, s[4 * k4 + 1]);
                if (4 * k4 + 2 > j) s[4 * k4 + 2] = fmaf(-s[j], c.z, s[4 * k4 + 2]);
                if (4 * k4 + 3 > j) s[4 * k4 + 3] = fmaf(-s[j], c.w, s[4 * k4 + 3]);
            }
        }
#pragma unroll
        for (int j = 0; j < NP; ++j)
            if (j < n) Q[r + (size_t)j * ldq] = s[j];
    }
}

// R (the caller's, FP64 upper triangular, ldr) from X = R^T (ld n)
__global__ void cholqr_copy_r_kernel(const double* __restrict__ X, int n, double* __restrict__ R, int64_t ldr) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx % n, j = idx / n;
    R[i + (size_t)j * ldr] = i <= j ? X[j + (size_t)i * n] : 0.0;
}

}  // namespace

cudaError_t launch_cholqr_q(const float* A, int64_t m, int n, int64_t lda, const double* X, float* Q, int64_t ldq,
                            double* R, int64_t ldr, int sm_count, cudaStream_t s) {
    if (n > 64) return cudaErrorNotSupported;
    if (R) {
        cholqr_copy_r_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(X, n, R, ldr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (m == 0 || !Q) return cudaSuccess;
    const int64_t need = (m + 255) / 256;
    const int grid = (int)(need < 4LL * sm_count ? need : 4LL * sm_count);
    if (n <= 16) cholqr_q_kernel<16><<<grid, 256, 0, s>>>(A, m, n, lda, X, Q, ldq);
    else if (n <= 32) cholqr_q_kernel<32><<<grid, 256, 0, s>>>(A, m, n, lda, X, Q, ldq);
    else if (n <= 48) cholqr_q_kernel<48><<<grid, 256, 0, s>>>(A, m, n, lda, X, Q, ldq);
    else cholqr_q_kernel<64><<<grid, 256, 0, s>>>(A, m, n, lda, X, Q, ldq);
    return cudaGetLastError();
}

}  // namespace tsvd
