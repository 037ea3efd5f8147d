// compute_u.cu -- U = A (V Sigma^{-1}) in working precision (Alg. 1 line 6,
// eq. (AV-0)).  W = RN(V / sigma) (n x n, column-major, formed by the finish
// kernel) is staged in shared memory 64 output columns at a time; each
// thread owns 4 consecutive rows x 16 output columns, streams the 4 rows of
// A column by column (128-bit loads when aligned) and accumulates in the
// working precision (FP32 FMA for FP32 working).  A is read once per
// 64-column block of U (once in total for n <= 64), U is written once.
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int U_NB = 64;        // output columns per CTA
constexpr int U_ROWS = 256;     // rows per CTA (64 threads x 4 rows)
constexpr int U_THREADS = 256;  // 4 column groups of 16

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4;
};

template <typename T, bool VEC>
__global__ void __launch_bounds__(U_THREADS)
    compute_u_kernel(const T* __restrict__ A, int64_t m, int n, int64_t lda, const T* __restrict__ W,
                     T* __restrict__ U, int64_t ldu) {
    extern __shared__ __align__(16) unsigned char usmem[];
    T* Ws = reinterpret_cast<T*>(usmem);  // [n][U_NB]
    const int j0 = blockIdx.y * U_NB;
    const int nb = min(U_NB, n - j0);
    for (int idx = threadIdx.x; idx < n * U_NB; idx += U_THREADS) {
        const int c = idx / U_NB, k = idx % U_NB;
        Ws[idx] = k < nb ? W[c + (size_t)(j0 + k) * n] : T(0);
    }
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * U_ROWS + 4 * (threadIdx.x & 63);
    const int cg = threadIdx.x >> 6;
    if (cg * 16 >= nb || r0 >= m) return;
    const bool full = (r0 + 3 < m);
    T acc[4][16];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[r][k] = T(0);
    for (int c = 0; c < n; ++c) {
        const T* src = A + (size_t)c * lda + r0;
        T a[4];
        if (VEC && full) {
            const typename Vec4<T>::type v = *reinterpret_cast<const typename Vec4<T>::type*>(src);
            a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = (r0 + r < m) ? src[r] : T(0);
        }
        const T* w = Ws + c * U_NB + cg * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const T wk = w[k];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r][k] = fma(a[r], wk, acc[r][k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int j = j0 + cg * 16 + k;
        if (j < n) {
            T* dst = U + (size_t)j * ldu + r0;
            if (VEC && full) {
                typename Vec4<T>::type v;
                v.x = acc[0][k]; v.y = acc[1][k]; v.z = acc[2][k]; v.w = acc[3][k];
                *reinterpret_cast<typename Vec4<T>::type*>(dst) = v;
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r0 + r < m) dst[r] = acc[r][k];
            }
        }
    }
}

template <typename T>
cudaError_t launch_u_t(const T* A, int64_t m, int n, int64_t lda, const T* W, T* U, int64_t ldu,
                       cudaStream_t s) {
    const size_t smem = sizeof(T) * n * U_NB;
    const bool vec = ((uintptr_t)A % (4 * sizeof(T)) == 0) && (lda % 4 == 0) &&
                     ((uintptr_t)U % (4 * sizeof(T)) == 0) && (ldu % 4 == 0);
    dim3 grid((unsigned)((m + U_ROWS - 1) / U_ROWS), (unsigned)((n + U_NB - 1) / U_NB));
    cudaError_t e;
    if (vec) {
        e = cudaFuncSetAttribute(compute_u_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(T) * 256 * U_NB));
        if (e != cudaSuccess) return e;
        compute_u_kernel<T, true><<<grid, U_THREADS, smem, s>>>(A, m, n, lda, W, U, ldu);
    } else {
        e = cudaFuncSetAttribute(compute_u_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(T) * 256 * U_NB));
        if (e != cudaSuccess) return e;
        compute_u_kernel<T, false><<<grid, U_THREADS, smem, s>>>(A, m, n, lda, W, U, ldu);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_compute_u(const void* A, int working, int64_t m, int n, int64_t lda,
                             const void* W, void* U, int64_t ldu, cudaStream_t s) {
    if (n > 256) return cudaErrorNotSupported;
    if (working == 0)
        return launch_u_t<float>((const float*)A, m, n, lda, (const float*)W, (float*)U, ldu, s);
    if (n > 128) return cudaErrorNotSupported;  // 256 x 64 doubles exceed shared memory
    return launch_u_t<double>((const double*)A, m, n, lda, (const double*)W, (double*)U, ldu, s);
}

}  // namespace tsvd
