// compute_u.cu -- U = A (V Sigma^{-1}) in working precision (Alg. 1 line 6,
// eq. (AV-0)).  W = RN(V / sigma) (n x n, column-major, formed by the finish
// kernel) is staged in shared memory 64 output columns at a time; each
// thread owns 4 consecutive rows x 16 output columns, streams the 4 rows of
// A column by column (128-bit loads when aligned) and accumulates in the
// working precision (FP32 FMA for FP32 working).  A is read once per
// 64-column block of U (once in total for n <= 64), U is written once.
#include "internal.cuh"
#include "tma_util.cuh"

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

// ---------------------------------------------------------------- v2: FP32, n <= 64
// Persistent CTAs (one per SM, 8 warps) stream 128-row x n tiles of A through
// a 3-stage shared-memory ring, one 2-D TMA load per tile (rows past m are
// zero-filled by the TMA unit), so two tiles are in flight while the third
// is consumed.  Each thread owns an 8-row x 4-column block of the U tile and
// accumulates with packed FP32 FMAs (fma.rn.f32x2): row pairs of A times a
// duplicated W entry, W being stored pre-duplicated ({w, w}) in shared
// memory so that no operand shuffles are needed.
constexpr int U2_ROWS = 128;
constexpr int U2_THREADS = 256;
constexpr int U2_STAGES = 3;

__device__ __forceinline__ void f2unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__global__ void __launch_bounds__(U2_THREADS, 1)
    compute_u_v2_kernel(const __grid_constant__ CUtensorMap tmapA, int64_t m, int n,
                        const float* __restrict__ W, float* __restrict__ U, int64_t ldu, int64_t ntiles,
                        DevInfo* info) {
    extern __shared__ __align__(128) unsigned char u2smem[];
    float* Ast = reinterpret_cast<float*>(u2smem);     // [STAGES][n][128] (TMA box, rows fastest)
    float* Wd = Ast + (size_t)U2_STAGES * 64 * U2_ROWS;  // [64][128] = {w,w} pairs
    __shared__ __align__(8) uint64_t full[U2_STAGES];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int tr = tid & 15;   // rows 8 tr .. 8 tr + 7 of the tile
    const int tc = tid >> 4;   // columns 4 tc .. 4 tc + 3
    const unsigned tile_bytes = (unsigned)(U2_ROWS * n * sizeof(float));
    if (tid == 0) {
        tma_prefetch_desc(&tmapA);
        for (int s = 0; s < U2_STAGES; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
        s_abort = 0;
    }
    for (int idx = tid; idx < 64 * 64; idx += U2_THREADS) {
        const int c = idx >> 6, j = idx & 63;
        const float w = (c < n && j < n) ? W[c + (size_t)j * n] : 0.f;
        Wd[c * 128 + 2 * j] = w;
        Wd[c * 128 + 2 * j + 1] = w;
    }
    __syncthreads();
    const int64_t first = blockIdx.x;
    if (tid == 0) {
        for (int k = 0; k < U2_STAGES - 1; ++k) {
            const int64_t t = first + (int64_t)k * gridDim.x;
            if (t < ntiles) {
                mbar_expect_tx(&full[k], tile_bytes);
                tma_load_2d(Ast + (size_t)k * 64 * U2_ROWS, &tmapA, (int)(t * U2_ROWS), 0, &full[k]);
            }
        }
    }
    unsigned phase_bits = 0u;  // bit s: parity to wait for on full[s]
    int stage = 0;
    for (int64_t tile = first; tile < ntiles; tile += gridDim.x) {
        const int64_t ahead = tile + (int64_t)(U2_STAGES - 1) * gridDim.x;
        const int astage = (stage + U2_STAGES - 1) % U2_STAGES;
        if (tid == 0 && ahead < ntiles) {
            mbar_expect_tx(&full[astage], tile_bytes);
            tma_load_2d(Ast + (size_t)astage * 64 * U2_ROWS, &tmapA, (int)(ahead * U2_ROWS), 0, &full[astage]);
        }
        if (!mbar_wait(&full[stage], (phase_bits >> stage) & 1u)) {
            atomicOr(&info->flags, FLAG_TIMEOUT);
            atomicExch(&s_abort, 1);
        }
        phase_bits ^= 1u << stage;
        __syncthreads();
        if (s_abort) break;
        const float* At = Ast + (size_t)stage * 64 * U2_ROWS + 8 * tr;
        const float* Wt = Wd + 8 * tc;
        unsigned long long acc[4][4];  // [row pair][column]
#pragma unroll
        for (int rp = 0; rp < 4; ++rp)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[rp][k] = 0ull;
#pragma unroll 4
        for (int c = 0; c < n; ++c) {
            const ulonglong2 a01 = *reinterpret_cast<const ulonglong2*>(At + c * U2_ROWS);
            const ulonglong2 a23 = *reinterpret_cast<const ulonglong2*>(At + c * U2_ROWS + 4);
            const ulonglong2 w01 = *reinterpret_cast<const ulonglong2*>(Wt + c * 128);
            const ulonglong2 w23 = *reinterpret_cast<const ulonglong2*>(Wt + c * 128 + 4);
            const unsigned long long ap[4] = {a01.x, a01.y, a23.x, a23.y};
            const unsigned long long wp[4] = {w01.x, w01.y, w23.x, w23.y};
#pragma unroll
            for (int rp = 0; rp < 4; ++rp)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[rp][k] = ffma2(ap[rp], wp[k], acc[rp][k]);
        }
        const int64_t r0 = tile * U2_ROWS + 8 * tr;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = 4 * tc + k;
            if (j >= n) continue;
            float v[8];
#pragma unroll
            for (int rp = 0; rp < 4; ++rp) f2unpack(acc[rp][k], v[2 * rp], v[2 * rp + 1]);
            float* dst = U + (size_t)j * ldu + r0;
            if (r0 + 7 < m) {
                reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
                reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    if (r0 + r < m) dst[r] = v[r];
            }
        }
        stage = (stage + 1) % U2_STAGES;
        __syncthreads();  // every thread is done with this stage before it is refilled
    }
    if (s_abort && tid == 0) {
        // leave no TMA load in flight: wait (bounded) on every stage's pending phase
        for (int s = 0; s < U2_STAGES; ++s) (void)mbar_wait(&full[s], (phase_bits >> s) & 1u);
    }
}

}  // namespace

size_t compute_u_v2_smem() { return sizeof(float) * ((size_t)U2_STAGES * 64 * U2_ROWS + 64 * 128); }

cudaError_t launch_compute_u_v2(const float* A, int64_t m, int n, int64_t lda, const float* W, float* U,
                                int64_t ldu, int sm_count, DevInfo* info, cudaStream_t s) {
    CUtensorMap tmap;
    cudaError_t e = make_tmap_2d(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), A, (uint64_t)m,
                                 (uint64_t)n, (uint64_t)lda, U2_ROWS, (uint32_t)n, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (e != cudaSuccess) return e;
    const size_t smem = compute_u_v2_smem();
    e = cudaFuncSetAttribute(compute_u_v2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (m + U2_ROWS - 1) / U2_ROWS;
    int64_t grid = (int64_t)sm_count;
    if (grid > ntiles) grid = ntiles;
    compute_u_v2_kernel<<<(unsigned)grid, U2_THREADS, smem, s>>>(tmap, m, n, W, U, ldu, ntiles, info);
    return cudaGetLastError();
}

bool compute_u_v2_ok(const void* A, int working, int64_t m, int n, int64_t lda, const void* U, int64_t ldu) {
    // TMA: 16-byte aligned base and column stride; 128-bit stores of U
    return working == 0 && n <= 64 && m >= 1 && ((uintptr_t)A % 16 == 0) && (lda % 4 == 0) &&
           ((uintptr_t)U % 16 == 0) && (ldu % 4 == 0);
}

cudaError_t launch_compute_u(const void* A, int working, int64_t m, int n, int64_t lda,
                             const void* W, void* U, int64_t ldu, cudaStream_t s) {
    if (n > 256) return cudaErrorNotSupported;
    if (working == 0)
        return launch_u_t<float>((const float*)A, m, n, lda, (const float*)W, (float*)U, ldu, s);
    if (n > 128) return cudaErrorNotSupported;  // 256 x 64 doubles exceed shared memory
    return launch_u_t<double>((const double*)A, m, n, lda, (const double*)W, (double*)U, ldu, s);
}

}  // namespace tsvd
