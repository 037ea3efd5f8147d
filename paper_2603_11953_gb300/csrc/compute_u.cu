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
// Persistent CTAs (two per SM, 4 warps each) stream 128-row x n tiles of A
// through a 2-stage shared-memory ring, one 2-D TMA load per tile (rows past
// m are zero-filled by the TMA unit).  Each thread owns 8 rows (4tr..4tr+3
// and 64+4tr..64+4tr+3, so the 16-byte shared reads of consecutive lanes are
// contiguous) by 8 columns of the U tile, and accumulates with packed FP32
// FMAs (fma.rn.f32x2): a row pair of A times a duplicated W entry, W being
// stored pre-duplicated ({w, w}) in shared memory.
constexpr int U2_ROWS = 128;
constexpr int U2_THREADS = 128;
constexpr int U2_STAGES = 2;

__device__ __forceinline__ void f2unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__global__ void __launch_bounds__(U2_THREADS, 2)
    compute_u_v2_kernel(const __grid_constant__ CUtensorMap tmapA, int64_t m, int n,
                        const float* __restrict__ W, float* __restrict__ U, int64_t ldu, int64_t ntiles,
                        DevInfo* info) {
    extern __shared__ __align__(128) unsigned char u2smem[];
    float* Ast = reinterpret_cast<float*>(u2smem);     // [STAGES][n][128] (TMA box, rows fastest)
    float* Wd = Ast + (size_t)U2_STAGES * 64 * U2_ROWS;  // [64][128] = {w,w} pairs
    __shared__ __align__(8) uint64_t full[U2_STAGES];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int tr = tid & 15;   // rows 4 tr .. 4 tr + 3 and 64 + 4 tr .. 64 + 4 tr + 3
    const int tc = tid >> 4;   // columns 8 tc .. 8 tc + 7
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
    if (tid == 0 && first < ntiles) {
        mbar_expect_tx(&full[0], tile_bytes);
        tma_load_2d(Ast, &tmapA, (int)(first * U2_ROWS), 0, &full[0]);
    }
    unsigned phase_bits = 0u;  // bit s: parity to wait for on full[s]
    int stage = 0;
    for (int64_t tile = first; tile < ntiles; tile += gridDim.x) {
        const int64_t next = tile + gridDim.x;
        if (tid == 0 && next < ntiles) {
            mbar_expect_tx(&full[stage ^ 1], tile_bytes);
            tma_load_2d(Ast + (size_t)(stage ^ 1) * 64 * U2_ROWS, &tmapA, (int)(next * U2_ROWS), 0, &full[stage ^ 1]);
        }
        if (!mbar_wait(&full[stage], (phase_bits >> stage) & 1u)) {
            atomicOr(&info->flags, FLAG_TIMEOUT);
            atomicExch(&s_abort, 1);
        }
        phase_bits ^= 1u << stage;
        __syncthreads();
        if (s_abort) break;
        const float* At = Ast + (size_t)stage * 64 * U2_ROWS + 4 * tr;
        const float* Wt = Wd + 16 * tc;
        unsigned long long acc[4][8];  // [row pair][column]
#pragma unroll
        for (int rp = 0; rp < 4; ++rp)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[rp][k] = 0ull;
#pragma unroll 2
        for (int c = 0; c < n; ++c) {
            const ulonglong2 a01 = *reinterpret_cast<const ulonglong2*>(At + c * U2_ROWS);
            const ulonglong2 a23 = *reinterpret_cast<const ulonglong2*>(At + c * U2_ROWS + 64);
            const ulonglong2* wv = reinterpret_cast<const ulonglong2*>(Wt + c * 128);
            const ulonglong2 w01 = wv[0], w23 = wv[1], w45 = wv[2], w67 = wv[3];
            const unsigned long long ap[4] = {a01.x, a01.y, a23.x, a23.y};
            const unsigned long long wp[8] = {w01.x, w01.y, w23.x, w23.y, w45.x, w45.y, w67.x, w67.y};
#pragma unroll
            for (int rp = 0; rp < 4; ++rp)
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[rp][k] = ffma2(ap[rp], wp[k], acc[rp][k]);
        }
        const int64_t rbase = tile * U2_ROWS;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = 8 * tc + k;
            if (j >= n) continue;
            float v[8];
#pragma unroll
            for (int rp = 0; rp < 4; ++rp) f2unpack(acc[rp][k], v[2 * rp], v[2 * rp + 1]);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int64_t r0 = rbase + 64 * hh + 4 * tr;
                float* dst = U + (size_t)j * ldu + r0;
                if (r0 + 3 < m) {
                    *reinterpret_cast<float4*>(dst) = make_float4(v[4 * hh], v[4 * hh + 1], v[4 * hh + 2], v[4 * hh + 3]);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r0 + r < m) dst[r] = v[4 * hh + r];
                }
            }
        }
        stage ^= 1;
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
    int64_t grid = (int64_t)sm_count * 2;
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
