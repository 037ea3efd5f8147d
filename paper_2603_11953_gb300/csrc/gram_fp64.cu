// gram_fp64.cu -- the double-double Gram of an FP64 working-precision A
// (Alg. 1 lines 1-2 with u = 2^-53 and u_h = double-double), computed on the
// same exact tensor-core Gram as FP32 inputs.
//
// Column j is scaled by 2^-e_j (exact), e_j the least integer with
// max_k |a_kj| < 2^e_j, and the scaled entry s (|s| < 1) is cut into four
// 23-bit fixed-point pieces by truncation toward zero (formed from the IEEE
// bit pattern with integer shifts):
//     s = x_0 + x_1 + x_2 + x_3 + r,   x_p an integer times 2^-23(p+1),
//     |x_p| < 2^-23p,  |r| < 2^-92.
// Every x_p is exact in FP32.  The pieces go to an m x 4NB FP32 matrix X
// (piece p of column j in column p NB + j, NB = n rounded up to 32, padding
// columns zero).  A column of X has at most 23 significant bits above its
// grid 2^-23(p+1), so the tensor-core Gram of X needs at most three digits per
// entry and loses nothing on a re-grid: each needed entry of X^T X is exact
// before its final rounding to double-double.  Then
//     (A^T A)_ij ~= 2^(e_i + e_j) sum_{p + q <= 3} (X_p^T X_q)_ij
// with |error| <= 8 * 2^-92 m 2^(e_i + e_j) (the remainder r and the six
// pairs p + q >= 4 that are left out), plus the double-double rounding.
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int PIECES = 4;
constexpr int PIECE_BITS = 23;

// per column: the largest |a| as a bit pattern (non-negative doubles order like
// their patterns); blocks over (row range, column), one atomicMax per block
// into cmax (zeroed by the caller)
__global__ void __launch_bounds__(256) colmax_kernel(const double* __restrict__ A, int64_t m, int64_t lda,
                                                     unsigned long long* __restrict__ cmax) {
    const int j = blockIdx.y;
    const long long* col = reinterpret_cast<const long long*>(A) + (size_t)j * lda;
    unsigned long long mx = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned long long)col[r] & 0x7fffffffffffffffull);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ unsigned long long s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, s[w]);
        if (mx) atomicMax(&cmax[j], mx);
    }
}

// least e with m < 2^e for the finite non-negative double with bit pattern mb
// (0 for an all-zero column; non-finite columns are flagged and scaled by 1)
__device__ __forceinline__ int col_exponent(unsigned long long mb) {
    if (mb == 0ull || mb >= 0x7ff0000000000000ull) return 0;
    int ex;
    frexp(__longlong_as_double((long long)mb), &ex);  // mb = f 2^ex, f in [1/2, 1)
    return ex;
}

// |a| 2^(92 - e) truncated to an integer F < 2^92, as (hi, lo) 64-bit words,
// from the bit pattern of a (integer arithmetic only: the FP64 pipe is narrow)
__device__ __forceinline__ void fixed92(unsigned long long bits, int e, unsigned long long& hi,
                                        unsigned long long& lo) {
    const int eb = (int)((bits >> 52) & 0x7ff);
    unsigned long long M = bits & 0xfffffffffffffull;
    int q = -1074;  // |a| = M 2^q
    if (eb != 0) {
        M |= 1ull << 52;
        q = eb - 1075;
    }
    const int sh = q + 92 - e;  // <= 91; F = M 2^sh < 2^92 because |a| < 2^e
    hi = 0ull;
    lo = 0ull;
    if (eb == 0x7ff || M == 0ull) return;
    if (sh >= 64) {
        hi = M << (sh - 64);
    } else if (sh > 0) {
        lo = M << sh;
        hi = M >> (64 - sh);
    } else if (sh > -64) {
        lo = M >> (-sh);
    }
}

// piece p of column j -> X[:, p NB + j]: bits [69 - 23p, 92 - 23p) of F, times 2^-23(p+1), with a's sign
__global__ void __launch_bounds__(256) split_kernel(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                    const unsigned long long* __restrict__ cmax, int NB,
                                                    float* __restrict__ X, int64_t ldx, int* __restrict__ e_out,
                                                    DevInfo* info) {
    const int j = blockIdx.y;  // 0 .. NB - 1
    int ex = 0;
    if (j < n) {
        const unsigned long long mb = cmax[j];
        ex = col_exponent(mb);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            e_out[j] = ex;
            if (mb >= 0x7ff0000000000000ull) atomicOr(&info->flags, FLAG_NONFINITE);
        }
    }
    const long long* col = reinterpret_cast<const long long*>(A) + (size_t)j * lda;
    constexpr unsigned MASK = (1u << PIECE_BITS) - 1u;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < ldx; r += (int64_t)gridDim.x * blockDim.x) {
        float x[PIECES] = {0.f, 0.f, 0.f, 0.f};
        if (j < n && r < m) {
            const unsigned long long bits = (unsigned long long)col[r];
            unsigned long long hi, lo;
            fixed92(bits, ex, hi, lo);
            const float sg = (bits >> 63) ? -1.f : 1.f;
            x[0] = sg * __uint2float_rn((unsigned)(hi >> 5) & MASK) * 0x1p-23f;
            x[1] = sg * __uint2float_rn((unsigned)((lo >> 46) | (hi << 18)) & MASK) * 0x1p-46f;
            x[2] = sg * __uint2float_rn((unsigned)(lo >> 23) & MASK) * 0x1p-69f;
            x[3] = sg * __uint2float_rn((unsigned)lo & MASK) * 0x1p-92f;
        }
#pragma unroll
        for (int p = 0; p < PIECES; ++p) X[r + (size_t)(p * NB + j) * ldx] = x[p];
    }
}

// double-double a + b (TwoSum of the high parts, then the low parts)
__device__ __forceinline__ void dd_add(double& ah, double& al, double bh, double bl) {
    const double s = ah + bh;
    const double bb = s - ah;
    double err = (ah - (s - bb)) + (bh - bb);
    err += al + bl;
    ah = s + err;
    al = err - (ah - s);
}

// G_ij = 2^(e_i + e_j) sum_{p + q <= 3} G3[p NB + i][q NB + j], smallest terms first
__global__ void __launch_bounds__(256) fold_kernel(const double* __restrict__ G3, const double* __restrict__ G3lo,
                                                   int64_t ld3, int n, int NB, const int* __restrict__ e,
                                                   double* __restrict__ G, double* __restrict__ G_lo, int64_t ldg) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx % n, j = idx / n;
    double h = 0.0, l = 0.0;
    for (int w = PIECES - 1; w >= 0; --w)
        for (int p = 0; p <= w; ++p) {
            const int q = w - p;
            const size_t k = (size_t)(p * NB + i) + (size_t)(q * NB + j) * ld3;
            dd_add(h, l, G3[k], G3lo[k]);
        }
    const int sh = e[i] + e[j];
    G[i + (size_t)j * ldg] = ldexp(h, sh);
    if (G_lo) G_lo[i + (size_t)j * ldg] = ldexp(l, sh);
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

struct Fp64Layout {
    size_t X, G3, G3lo, cmax, e, total;
};
Fp64Layout fp64_layout(int64_t m, int n) {
    const int NB = fp64_block_cols(n);
    const size_t C = (size_t)PIECES * NB;
    Fp64Layout L;
    size_t off = 0;
    L.X = off; off += up256(sizeof(float) * (size_t)fp64_split_ld(m) * C);
    L.G3 = off; off += up256(sizeof(double) * C * C);
    L.G3lo = off; off += up256(sizeof(double) * C * C);
    L.cmax = off; off += up256(sizeof(unsigned long long) * n);
    L.e = off; off += up256(sizeof(int) * n);
    L.total = off;
    return L;
}

}  // namespace

int fp64_block_cols(int n) { return (n + 31) / 32 * 32; }
int64_t fp64_split_ld(int64_t m) { return (m + 3) / 4 * 4; }
size_t fp64_extra_bytes(int64_t m, int n) { return fp64_layout(m, n).total; }

bool fp64_pair_needed(int n, int b1, int b2) {
    const int per = fp64_block_cols(n) / 32;  // 32-column blocks per piece
    return b1 / per + b2 / per <= PIECES - 1;
}

const float* fp64_split_matrix(const void* extra) { return static_cast<const float*>(extra); }

double* fp64_g3(void* extra, int64_t m, int n, double** g3lo) {
    const Fp64Layout L = fp64_layout(m, n);
    char* p = static_cast<char*>(extra);
    *g3lo = reinterpret_cast<double*>(p + L.G3lo);
    return reinterpret_cast<double*>(p + L.G3);
}

cudaError_t launch_fp64_split(const double* A, int64_t m, int n, int64_t lda, void* extra, DevInfo* info,
                              cudaStream_t s) {
    const Fp64Layout L = fp64_layout(m, n);
    char* p = static_cast<char*>(extra);
    unsigned long long* cmax = reinterpret_cast<unsigned long long*>(p + L.cmax);
    const int64_t ldx = fp64_split_ld(m);
    int64_t bx = (ldx + 255) / 256;
    if (bx > 148) bx = 148;
    cudaError_t err = cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * n, s);
    if (err != cudaSuccess) return err;
    colmax_kernel<<<dim3((unsigned)bx, (unsigned)n), 256, 0, s>>>(A, m, lda, cmax);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int NB = fp64_block_cols(n);
    split_kernel<<<dim3((unsigned)bx, (unsigned)NB), 256, 0, s>>>(A, m, n, lda, cmax, NB,
                                                                   reinterpret_cast<float*>(p + L.X), ldx,
                                                                   reinterpret_cast<int*>(p + L.e), info);
    return cudaGetLastError();
}

cudaError_t launch_fp64_fold(void* extra, int64_t m, int n, double* G, double* G_lo, int64_t ldg, cudaStream_t s) {
    const Fp64Layout L = fp64_layout(m, n);
    char* p = static_cast<char*>(extra);
    const int NB = fp64_block_cols(n);
    fold_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const double*>(p + L.G3),
                                                    reinterpret_cast<const double*>(p + L.G3lo),
                                                    (int64_t)PIECES * NB, n, NB,
                                                    reinterpret_cast<const int*>(p + L.e), G, G_lo, ldg);
    return cudaGetLastError();
}

}  // namespace tsvd
