// cholqr.cu -- the mixed precision Cholesky QR algorithm that motivates the
// paper (Sec. 3.1 and Theorem 3), on the same Gram kernels:
//   1. M_h = A^T A at the higher precision (the tensor-core Gram),
//   2. M_h = R^T R by the plain Cholesky factorization in FP64,
//   3. Q from the linear systems Q R = A at the working precision: every row
//      q of Q solves q R_w = a by forward substitution in FP32, R_w = RN_32(R).
// With u_h = 2^-53 <= u^2 (u = 2^-24), Theorem 3 bounds ||Q^T Q - I|| by
// O(u) kappa(B) instead of the O(u) kappa(B)^2 of a same-precision Cholesky QR.
//
// cholqr_q_kernel: one thread per row, the row's n solutions in registers; R_w
// is in shared memory with its columns contiguous (entry (i, j) at Rt[j][i]),
// so the 16-byte shared loads of q_j's sum broadcast four entries of column j
// to the warp.  A is read once and Q written once (coalesced: consecutive
// threads hold consecutive rows of the column-major arrays).  The n^2 / 2 FMAs
// per row cost about 0.7 of the time A and Q take over HBM at n = 64.
#include "internal.cuh"

namespace tsvd {
namespace {

template <int NP>
__global__ void __launch_bounds__(256)
    cholqr_q_kernel(const float* __restrict__ A, int64_t m, int n, int64_t lda, const double* __restrict__ X,
                    float* __restrict__ Q, int64_t ldq) {
    __shared__ __align__(16) float Rt[NP][NP];  // Rt[j][i] = RN_32(R[i][j]), i <= j; zero elsewhere
    __shared__ float Rd[NP];                     // the diagonal
    for (int idx = threadIdx.x; idx < NP * NP; idx += blockDim.x) {
        const int j = idx / NP, i = idx % NP;
        // X = R^T with ld n: R[i][j] = X[j + i n]
        Rt[j][i] = (i <= j && j < n) ? (float)X[j + (size_t)i * n] : 0.0f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NP; j += blockDim.x) Rd[j] = j < n ? Rt[j][j] : 1.0f;
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        float a[NP], q[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) a[j] = j < n ? A[r + (size_t)j * lda] : 0.0f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            // q_j = (a_j - sum_{i<j} q_i r_ij) / r_jj, the sum in FP32 in the order of i
            float s = a[j];
            const float4* col = reinterpret_cast<const float4*>(Rt[j]);
#pragma unroll
            for (int i4 = 0; i4 < (j + 3) / 4; ++i4) {
                const float4 c = col[i4];
                if (4 * i4 + 0 < j) s = fmaf(-q[4 * i4 + 0], c.x, s);
                if (4 * i4 + 1 < j) s = fmaf(-q[4 * i4 + 1], c.y, s);
                if (4 * i4 + 2 < j) s = fmaf(-q[4 * i4 + 2], c.z, s);
                if (4 * i4 + 3 < j) s = fmaf(-q[4 * i4 + 3], c.w, s);
            }
            q[j] = s / Rd[j];
        }
#pragma unroll
        for (int j = 0; j < NP; ++j)
            if (j < n) Q[r + (size_t)j * ldq] = q[j];
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
