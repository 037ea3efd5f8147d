// gram_sharded.cu -- the Gram matrix of a row-partitioned A (Sec. 4.2.1: the
// rows are distributed over the processes and A^T A needs one global sum), in
// a form whose result does not depend on the partition.
//
// The tensor-core Gram (gram_tc.cu) is given one exponent per column, E_j with
// max_r |a_rj| < 2^E_j over the WHOLE matrix (all ranks: an all-reduce of the
// maxima), instead of its running per-CTA scales.  Then every digit of every
// entry is a fixed function of that entry, every digit-pair product is summed
// exactly (the s + t = 6 blocks through their exact residuals), and every
// rank's partial is an exact integer in units 2^(E_i + E_j - 63).  Its four
// 32-bit limbs (value = sum_k limb_k 2^(32 k), limbs 0-2 in [0, 2^32), limb 3
// signed, each held in an int64) add exactly in any order and over up to 2^31
// ranks without overflow; the sum is rounded once to FP64 (and a double-double)
// at the end.  The result is bitwise the same for every row partition, every
// split over CTAs and every order of the rows, and equals the single-GPU Gram
// with fixed scales (tsvd_opts.fixed_scale).
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int CM_THREADS = 256;

// max |a_rj| over the block's rows of column blockIdx.y, as a float bit pattern
// (non-negative floats order like their patterns; Inf and NaN order above all)
__global__ void __launch_bounds__(CM_THREADS)
    colmax_f32_kernel(const float* __restrict__ A, int64_t m, int64_t lda, int64_t rows_per_block,
                      unsigned* __restrict__ colmax) {
    const int j = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < m ? r0 + rows_per_block : m;
    const float* col = A + (size_t)j * lda;
    unsigned mx = 0u;
    int64_t r = r0 + threadIdx.x;
    for (; r + 3 * CM_THREADS < r1; r += 4 * CM_THREADS) {
        const unsigned a = __float_as_uint(col[r]), b = __float_as_uint(col[r + CM_THREADS]);
        const unsigned c = __float_as_uint(col[r + 2 * CM_THREADS]), d = __float_as_uint(col[r + 3 * CM_THREADS]);
        mx = max(mx, max(max(a & 0x7fffffffu, b & 0x7fffffffu), max(c & 0x7fffffffu, d & 0x7fffffffu)));
    }
    for (; r < r1; r += CM_THREADS) mx = max(mx, __float_as_uint(col[r]) & 0x7fffffffu);
    mx = __reduce_max_sync(0xffffffffu, mx);
    __shared__ unsigned s_mx[CM_THREADS / 32];
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned v = 0u;
        for (int w = 0; w < CM_THREADS / 32; ++w) v = max(v, s_mx[w]);
        if (v) atomicMax(&colmax[j], v);
    }
}

// E_j: the least e with max_r |a_rj| < 2^e (as the tensor-core Gram's deciders define it),
// EXP_EMPTY for an all-zero column; Inf or NaN flags the input
__global__ void colexp_kernel(const unsigned* __restrict__ colmax, int n, int* __restrict__ E, DevInfo* info) {
    const int j = threadIdx.x;
    if (j >= n) return;
    const unsigned mx = colmax[j];
    int e = EXP_EMPTY;
    if (mx >= 0x7f800000u) atomicOr(&info->flags, FLAG_NONFINITE);
    else if (mx != 0u) {
        const int be = (int)((mx >> 23) & 0xff);
        e = be == 0 ? -126 : be - 126;
    }
    E[j] = e;
}

// One warp per entry (i, j), i <= j: the exact sum over the CTAs' partials (which all share
// the fixed exponents), as four 32-bit limbs at [k][i][j] and [k][j][i] (limbs k, n x n,
// column-major).
__global__ void __launch_bounds__(256)
    gram_limbs_kernel(const long long* __restrict__ part_hi, const long long* __restrict__ part_lo, int P, int n,
                      const int* __restrict__ E, long long* __restrict__ limbs) {
    const int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (idx >= n * (n + 1) / 2) return;  // whole warps only
    int j = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= idx) ++j;
    while (j * (j + 1) / 2 > idx) --j;
    const int i = idx - j * (j + 1) / 2;
    __int128 acc = 0;
    if (E[i] != EXP_EMPTY && E[j] != EXP_EMPTY) {
        for (int c = lane; c < P; c += 32) {
            const size_t a = (size_t)c * 64 * 64 + (size_t)i * 64 + j, b = (size_t)c * 64 * 64 + (size_t)j * 64 + i;
            const __int128 h = (__int128)part_hi[a] + (__int128)part_hi[b];
            const __int128 l = (__int128)part_lo[a] + (__int128)part_lo[b];
            acc += h * ((__int128)1 << 16) + l;  // units 2^(E_i + E_j - 63)
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += shfl_xor_i128(acc, o);
    }
    if (lane < 4) {
        const size_t nn = (size_t)n * n;
        const long long limb = lane < 3 ? (long long)(((unsigned __int128)acc >> (32 * lane)) & 0xffffffffu)
                                        : (long long)(acc >> 96);
        limbs[lane * nn + i + (size_t)j * n] = limb;
        limbs[lane * nn + j + (size_t)i * n] = limb;
    }
}

// G_ij = RN(sum_k limb_k 2^(32 k) * 2^(E_i + E_j - 63)) (and the double-double low part);
// the limb sum is taken modulo 2^128, exact whenever the true sum fits (always: it is below
// 2^(90 + log2 of the number of partials)).
__global__ void gram_finish_kernel(const long long* __restrict__ limbs, int n, const int* __restrict__ E,
                                   double* __restrict__ G, double* __restrict__ G_lo, int64_t ldg) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx % n, j = idx / n;
    const size_t nn = (size_t)n * n;
    double hi = 0.0, lo = 0.0;
    if (E[i] != EXP_EMPTY && E[j] != EXP_EMPTY) {
        unsigned __int128 t = 0;
        for (int k = 0; k < 4; ++k) t += (unsigned __int128)(__int128)limbs[k * nn + idx] << (32 * k);
        __int128 r1, r2;
        hi = round_i128((__int128)t, E[i] + E[j] - 63, r1);
        lo = round_i128((__int128)t - r1, E[i] + E[j] - 63, r2);
    }
    G[i + (size_t)j * ldg] = hi;
    if (G_lo) G_lo[i + (size_t)j * ldg] = lo;
}

}  // namespace

cudaError_t launch_colexp(const float* A, int64_t m, int n, int64_t lda, unsigned* colmax_ws, int* E, DevInfo* info,
                          int sm_count, cudaStream_t s) {
    if (n < 1 || n > 64) return cudaErrorNotSupported;
    cudaError_t e = cudaMemsetAsync(colmax_ws, 0, sizeof(unsigned) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    // about four CTAs per SM over all columns, at least 4096 rows each
    int64_t blocks = (4 * (int64_t)sm_count + n - 1) / n;
    const int64_t max_blocks = (m + 4095) / 4096;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    const int64_t rows = (m + blocks - 1) / blocks;
    colmax_f32_kernel<<<dim3((unsigned)blocks, (unsigned)n), CM_THREADS, 0, s>>>(A, m, lda, rows, colmax_ws);
    colexp_kernel<<<1, 64, 0, s>>>(colmax_ws, n, E, info);
    return cudaGetLastError();
}

cudaError_t launch_gram_limbs(const GramPlan& plan, const void* part, int n, const int* E, long long* limbs,
                              cudaStream_t s) {
    const long long* ph = reinterpret_cast<const long long*>(part);
    const long long* pl = ph + (size_t)plan.P * 64 * 64;
    const int npairs = n * (n + 1) / 2;
    gram_limbs_kernel<<<(npairs + 7) / 8, 256, 0, s>>>(ph, pl, plan.P, n, E, limbs);
    return cudaGetLastError();
}

cudaError_t launch_gram_finish(const long long* limbs, int n, const int* E, double* G, double* G_lo, int64_t ldg,
                               cudaStream_t s) {
    gram_finish_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(limbs, n, E, G, G_lo, ldg);
    return cudaGetLastError();
}

}  // namespace tsvd
