// gram_ozaki.cu -- higher-precision Gram matrix M_h = A^T A (Alg. 1 lines 1-2).
//
// The Gram is formed EXACTLY up to a controlled truncation, on BF16 tensor
// cores, by an Ozaki-style split:
//
//   * Rows are processed in chunks of KC = 128.  For every column j a CTA
//     keeps a running power-of-two scale 2^E_j with |a_rj| < 2^E_j for every
//     row seen so far (E_j only grows; when it grows the accumulators of row
//     and column j are shifted right, i.e. re-expressed on the coarser grid).
//   * Each entry x = a * 2^-E_j (|x| < 1) is split exactly into k = 7 signed
//     digits by round-to-nearest:  y_0 = 128 x,  q_s = rint(y_s),
//     y_{s+1} = 256 (y_s - q_s);  x = sum_s q_s 2^(-7-8s) + r,
//     |q_s| <= 128 (exact in bf16), |r| <= 2^-56.
//   * For every digit pair (s, t) with s <= t and s + t <= 6 (0-based; the
//     16 pairs whose weight 2^(-14-8(s+t)) is at or above 2^-62) the chunk sum
//     P_st = sum_r q_s(r,i) q_t(r,j) is an integer of magnitude <= 128*128^2
//     = 2^21, so the BF16 MMA with FP32 accumulation computes it exactly.
//   * Each P_st is folded into two int64 fixed-point accumulators per (i, j):
//     hi in units of 2^(E_i+E_j-47) (pairs with s+t <= 4) and lo in units of
//     2^(E_i+E_j-63) (s+t = 5, 6).  With W = sum_{s<t} P_st + 1/2 sum_s P_ss
//     the Gram is W + W^T, so only the pairs s <= t are ever multiplied.
//   * The cross-CTA combine aligns all CTA partials to the largest exponent in
//     a 128-bit integer and rounds once (to FP64, and to a double-double).
//
// Error: only the digit truncation (r) and the dropped pairs s + t >= 7
// (weight <= 2^-70 each) and the rare right shifts when E grows; the MMA,
// the fold and the combine are exact.  The plain all-FP64 Gram (DFMA,
// fixed-order combine) is the comparison form of the same step.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace tsvd {
namespace {

struct BlockSpec {
    int s, t, to_lo, shift;
};
// (s, t) digit pairs, target accumulator, left shift of the chunk sum.
// hi unit 2^-47: shift = 47 - 14 - 8(s+t) - [s==t];
// lo unit 2^-63: shift = 63 - 14 - 8(s+t) - [s==t].
__constant__ BlockSpec c_blocks[16] = {
    {0, 0, 0, 32}, {0, 1, 0, 25}, {0, 2, 0, 17}, {1, 1, 0, 16}, {0, 3, 0, 9}, {1, 2, 0, 9},
    {0, 4, 0, 1},  {1, 3, 0, 1},  {2, 2, 0, 0},  {0, 5, 1, 9},  {1, 4, 1, 9}, {2, 3, 1, 9},
    {0, 6, 1, 1},  {1, 5, 1, 1},  {2, 4, 1, 1},  {3, 3, 1, 0}};
constexpr int NBLOCKS = 16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                            uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldmatrix_x2(uint32_t& r0, uint32_t& r1, uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                               uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// a * 2^k, exact whenever the result is a normal float (two normal factors).
__device__ __forceinline__ float scale_pow2(float a, int k) {
    int k1 = k / 2, k2 = k - k1;
    return (a * __int_as_float((k1 + 127) << 23)) * __int_as_float((k2 + 127) << 23);
}

// Exponent e with max < 2^e (max > 0, finite).
__device__ __forceinline__ int exp_above(float mx) {
    unsigned b = __float_as_uint(mx);
    int be = (b >> 23) & 0xff;
    return be == 0 ? -126 : be - 126;
}

template <int NP>
struct GramSmem {
    static constexpr int KC = GRAM_KC;
    static constexpr int KP = GRAM_KC + 8;  // padded digit row (bf16 elements): conflict-free ldmatrix
    static constexpr size_t tile_bytes = sizeof(float) * NP * KC;
    static constexpr size_t dig_bytes = sizeof(__nv_bfloat16) * GRAM_DIGITS * NP * KP;
    static constexpr size_t bytes = tile_bytes + dig_bytes + 3 * NP * sizeof(int);
};

// The Gram partial of rows [r_begin, r_end) of A (n <= NP columns) by one CTA of
// 256 threads, written as NP x NP int64 hi / lo accumulators at ph / pl and the
// NP column exponents at pE.
template <int NP, bool VEC>
__device__ __forceinline__ void ozaki_rows(const float* __restrict__ A, int n, int64_t lda, int64_t r_begin,
                                           int64_t r_end, long long* __restrict__ ph, long long* __restrict__ pl,
                                           int* __restrict__ pE, DevInfo* info) {
    constexpr int KC = GRAM_KC;
    constexpr int KP = GramSmem<NP>::KP;
    constexpr int NT = (NP / 16) * (NP / 8);  // m16 x n8 output tiles
    constexpr int TPW = (NT + 7) / 8;         // tiles per warp
    extern __shared__ __align__(16) unsigned char smem[];
    float* tile = reinterpret_cast<float*>(smem);  // [NP][KC]
    __nv_bfloat16* dig = reinterpret_cast<__nv_bfloat16*>(smem + GramSmem<NP>::tile_bytes);  // [7][NP][KP]
    int* E_run = reinterpret_cast<int*>(smem + GramSmem<NP>::tile_bytes + GramSmem<NP>::dig_bytes);
    int* e_chk = E_run + NP;
    int* dE = e_chk + NP;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    __syncthreads();  // the previous row range (batched use) is done with the shared state
    if (tid < NP) E_run[tid] = EXP_EMPTY;
    long long acc_hi[TPW * 4], acc_lo[TPW * 4];
#pragma unroll
    for (int k = 0; k < TPW * 4; ++k) acc_hi[k] = acc_lo[k] = 0;
    bool bad = false;
    __syncthreads();

    for (int64_t r0 = r_begin; r0 < r_end; r0 += KC) {
        const int rows = (r_end - r0 < (int64_t)KC) ? (int)(r_end - r0) : KC;
        // (a) stage the FP32 chunk [NP][KC] (zero padding for ragged rows / columns)
        if (VEC) {
            for (int idx = tid; idx < NP * (KC / 4); idx += 256) {
                const int j = idx / (KC / 4), rr = 4 * (idx % (KC / 4));
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < n) {
                    const float* src = A + (size_t)j * lda + r0 + rr;
                    if (rr + 3 < rows) {
                        v = __ldcs(reinterpret_cast<const float4*>(src));
                    } else {
                        if (rr < rows) v.x = src[0];
                        if (rr + 1 < rows) v.y = src[1];
                        if (rr + 2 < rows) v.z = src[2];
                    }
                }
                if (!isfinite(v.x)) { bad = true; v.x = 0.f; }
                if (!isfinite(v.y)) { bad = true; v.y = 0.f; }
                if (!isfinite(v.z)) { bad = true; v.z = 0.f; }
                if (!isfinite(v.w)) { bad = true; v.w = 0.f; }
                *reinterpret_cast<float4*>(&tile[j * KC + rr]) = v;
            }
        } else {
            for (int idx = tid; idx < NP * KC; idx += 256) {
                const int j = idx / KC, rr = idx % KC;
                float v = 0.f;
                if (j < n && rr < rows) v = A[(size_t)j * lda + r0 + rr];
                if (!isfinite(v)) { bad = true; v = 0.f; }
                tile[j * KC + rr] = v;
            }
        }
        __syncthreads();
        // (b) per-column chunk maximum -> exponent
        for (int j = warp; j < NP; j += 8) {
            float mx = 0.f;
            for (int r = lane; r < KC; r += 32) mx = fmaxf(mx, fabsf(tile[j * KC + r]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) e_chk[j] = (mx == 0.f) ? EXP_EMPTY : exp_above(mx);
        }
        __syncthreads();
        // (c) running scale; dE = how far the grid of column j coarsens
        if (tid < NP) {
            const int old = E_run[tid], e = e_chk[tid];
            const int nw = max(old, e);
            dE[tid] = (old == EXP_EMPTY) ? 64 : nw - old;
            E_run[tid] = nw;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TPW; ++u) {
            const int t = warp + 8 * u;
            if (t < NT) {
                const int mi = t / (NP / 8), ni = t % (NP / 8), g = lane >> 2, tq = lane & 3;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int i = mi * 16 + g + (h >= 2 ? 8 : 0), j = ni * 8 + 2 * tq + (h & 1);
                    const int sh = dE[i] + dE[j];
                    if (sh > 0) {
                        if (sh >= 63) {
                            acc_hi[u * 4 + h] = 0;
                            acc_lo[u * 4 + h] = 0;
                        } else {
                            acc_hi[u * 4 + h] >>= sh;
                            acc_lo[u * 4 + h] >>= sh;
                        }
                    }
                }
            }
        }
        // (d) exact digit split, two consecutive rows per thread (bf16x2)
        for (int idx = tid; idx < NP * (KC / 2); idx += 256) {
            const int j = idx / (KC / 2), rp = idx % (KC / 2);
            const float2 a = *reinterpret_cast<const float2*>(&tile[j * KC + 2 * rp]);
            const int E = E_run[j];
            float y0 = 0.f, y1 = 0.f;
            if (E != EXP_EMPTY) {
                y0 = scale_pow2(a.x, 7 - E);
                y1 = scale_pow2(a.y, 7 - E);
            }
#pragma unroll
            for (int s = 0; s < GRAM_DIGITS; ++s) {
                const float q0 = rintf(y0), q1 = rintf(y1);
                *reinterpret_cast<__nv_bfloat162*>(&dig[(s * NP + j) * KP + 2 * rp]) =
                    __floats2bfloat162_rn(q0, q1);
                y0 = (y0 - q0) * 256.f;
                y1 = (y1 - q1) * 256.f;
            }
        }
        __syncthreads();
        // (e) exact digit-pair products on the tensor cores, folded into int64
#pragma unroll 1
        for (int b = 0; b < NBLOCKS; ++b) {
            const BlockSpec bs = c_blocks[b];
            const __nv_bfloat16* As = dig + bs.s * NP * KP;
            const __nv_bfloat16* Bs = dig + bs.t * NP * KP;
#pragma unroll
            for (int u = 0; u < TPW; ++u) {
                const int t = warp + 8 * u;
                if (t < NT) {
                    const int mi = t / (NP / 8), ni = t % (NP / 8);
                    float d[4] = {0.f, 0.f, 0.f, 0.f};
                    const int arow = mi * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                    const int acol = (lane >> 4) * 8;
                    const int brow = ni * 8 + (lane & 7);
                    const int bcol = ((lane >> 3) & 1) * 8;
                    const uint32_t a_addr = smem_u32(As + arow * KP + acol);
                    const uint32_t b_addr = smem_u32(Bs + brow * KP + bcol);
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        uint32_t a0, a1, a2, a3, b0, b1;
                        ldmatrix_x4(a0, a1, a2, a3, a_addr + kk * 32);
                        ldmatrix_x2(b0, b1, b_addr + kk * 32);
                        mma_bf16_16816(d, a0, a1, a2, a3, b0, b1);
                    }
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        // exact integer |d| <= 2^21: the 1.5*2^23 bias puts it in the mantissa
                        const int iv = __float_as_int(d[h] + 12582912.0f) - 0x4B400000;
                        const long long v =
                            (long long)((unsigned long long)(long long)iv << bs.shift);
                        if (bs.to_lo) acc_lo[u * 4 + h] += v;
                        else acc_hi[u * 4 + h] += v;
                    }
                }
            }
        }
        __syncthreads();
    }
    // (f) partials of this row range
#pragma unroll
    for (int u = 0; u < TPW; ++u) {
        const int t = warp + 8 * u;
        if (t < NT) {
            const int mi = t / (NP / 8), ni = t % (NP / 8), g = lane >> 2, tq = lane & 3;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = mi * 16 + g + (h >= 2 ? 8 : 0), j = ni * 8 + 2 * tq + (h & 1);
                ph[i * NP + j] = acc_hi[u * 4 + h];
                pl[i * NP + j] = acc_lo[u * 4 + h];
            }
        }
    }
    if (tid < NP) pE[tid] = E_run[tid];
    if (bad) atomicOr(&info->flags, FLAG_NONFINITE);
}

template <int NP, bool VEC>
__global__ void __launch_bounds__(256, 1)
    gram_ozaki_kernel(const float* __restrict__ A, int64_t m, int n, int64_t lda,
                      int64_t rows_per_cta, long long* __restrict__ part_hi,
                      long long* __restrict__ part_lo, int* __restrict__ part_E, DevInfo* info) {
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r_end = min(m, r_begin + rows_per_cta);
    ozaki_rows<NP, VEC>(A, n, lda, r_begin, r_end, part_hi + (size_t)blockIdx.x * NP * NP,
                        part_lo + (size_t)blockIdx.x * NP * NP, part_E + (size_t)blockIdx.x * NP, info);
}

// Batched: every CTA takes work items (instance, row range, partial slot) in turn; the
// partial of slot k sits at k * BATCH_SLOT (hi, lo) and k * 64 (exponents).
template <int NP, bool VEC>
__global__ void __launch_bounds__(256, 1)
    gram_ozaki_batch_kernel(const BatchInst* __restrict__ inst, const BatchGramItem* __restrict__ items, int nitems,
                            long long* __restrict__ part_hi, long long* __restrict__ part_lo,
                            int* __restrict__ part_E, DevInfo* __restrict__ infos) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const BatchGramItem it = items[w];
        const BatchInst& d = inst[it.inst];
        ozaki_rows<NP, VEC>(d.A, d.n, d.lda, it.r0, it.r1, part_hi + (size_t)it.slot * BATCH_SLOT,
                            part_lo + (size_t)it.slot * BATCH_SLOT, part_E + (size_t)it.slot * 64,
                            infos + it.inst);
    }
}

// ---------------------------------------------------------------- exact combine
// One warp per Gram entry (i, j), i <= j: the lanes take every 32nd partial, and the
// exact int128 sums are added across the warp (integer addition: the result does not
// depend on the order, so the Gram is bitwise reproducible).
// The exact sum over P partials (slot c at c * slot (hi, lo) and c * estride
// (exponents), NP x NP row-major) of entry (i, j), rounded to a double-double;
// all 32 lanes of the warp take part.
// halves = 2: every slot holds two tiles to add, at (i, j) and (32 + i, 32 + j).
__device__ __forceinline__ void combine_entry(const long long* __restrict__ part_hi,
                                              const long long* __restrict__ part_lo,
                                              const int* __restrict__ part_E, int P, size_t slot, int estride,
                                              int NP, int i0, int j0, int lane, double& hi, double& lo,
                                              int halves = 1) {
    const int PV = P * halves;
    int emax = EXP_EMPTY;
    for (int v = lane; v < PV; v += 32) {
        const int c = v / halves, off = (v % halves) * 32, i = i0 + off, j = j0 + off;
        const int Ei = part_E[(size_t)c * estride + i], Ej = part_E[(size_t)c * estride + j];
        if (Ei == EXP_EMPTY || Ej == EXP_EMPTY) continue;
        emax = max(emax, Ei + Ej);
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    hi = 0.0;
    lo = 0.0;
    if (emax != EXP_EMPTY) {
        // value_c = 2^(e_c - 63) * (h * 2^16 + l); fixed point unit 2^(emax - 63 - 29)
        __int128 acc = 0;
        for (int v = lane; v < PV; v += 32) {
            const int c = v / halves, off = (v % halves) * 32, i = i0 + off, j = j0 + off;
            const int Ei = part_E[(size_t)c * estride + i], Ej = part_E[(size_t)c * estride + j];
            if (Ei == EXP_EMPTY || Ej == EXP_EMPTY) continue;
            const int sh = emax - (Ei + Ej);
            if (sh >= 110) continue;  // below 2^-139 of the largest partial scale
            const size_t a = (size_t)c * slot + (size_t)i * NP + j, b = (size_t)c * slot + (size_t)j * NP + i;
            const __int128 h = (__int128)part_hi[a] + (__int128)part_hi[b];
            const __int128 l = (__int128)part_lo[a] + (__int128)part_lo[b];
            const __int128 X = h * ((__int128)1 << 16) + l;
            acc += (X * ((__int128)1 << 29)) >> sh;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += shfl_xor_i128(acc, o);
        __int128 r1, r2;
        hi = round_i128(acc, emax - 92, r1);
        lo = round_i128(acc - r1, emax - 92, r2);
    }
}

__device__ __forceinline__ void pair_of(int idx, int& i, int& j) {
    j = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= idx) ++j;
    while (j * (j + 1) / 2 > idx) --j;
    i = idx - j * (j + 1) / 2;
}

__global__ void __launch_bounds__(256) gram_combine_kernel(const long long* __restrict__ part_hi,
                                                           const long long* __restrict__ part_lo,
                                                           const int* __restrict__ part_E, int P, int NP, int n,
                                                           double* __restrict__ G, double* __restrict__ G_lo,
                                                           int64_t ldg, int c1, int c2, int wmask, int nglob) {
    const int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int npairs = n * (n + 1) / 2;
    if (idx >= npairs) return;  // whole warps only
    int i, j;
    pair_of(idx, i, j);
    double hi, lo;
    combine_entry(part_hi, part_lo, part_E, P, (size_t)NP * NP, NP, NP, i, j, lane, hi, lo);
    int gi = i, gj = j;
    if (c1 >= 0) {
        // two-group launch: map the local columns, keep only the tiles asked for
        const int tile = (j < 32) ? 1 : (i >= 32) ? 2 : 4;
        gi = i < 32 ? c1 + i : c2 + i - 32;
        gj = j < 32 ? c1 + j : c2 + j - 32;
        if (!(wmask & tile) || gi >= nglob || gj >= nglob) return;
    }
    if (lane == 0) {
        G[gi + (size_t)gj * ldg] = hi;
        G[gj + (size_t)gi * ldg] = hi;
        if (G_lo) {
            G_lo[gi + (size_t)gj * ldg] = lo;
            G_lo[gj + (size_t)gi * ldg] = lo;
        }
    }
}

// Batched: one CTA per instance, warps over its entries i <= j, G into the instance's
// n x n FP64 block (ld n).
__global__ void __launch_bounds__(256) gram_combine_batch_kernel(const BatchInst* __restrict__ inst,
                                                                 const long long* __restrict__ part_hi,
                                                                 const long long* __restrict__ part_lo,
                                                                 const int* __restrict__ part_E) {
    const BatchInst& d = inst[blockIdx.x];
    const int n = d.n, NP = d.NP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npairs = n * (n + 1) / 2;
    const size_t s0 = (size_t)d.slot0;
    for (int idx = warp; idx < npairs; idx += blockDim.x / 32) {
        int i, j;
        pair_of(idx, i, j);
        double hi, lo;
        combine_entry(part_hi + s0 * BATCH_SLOT, part_lo + s0 * BATCH_SLOT, part_E + s0 * 64, d.nslots, BATCH_SLOT,
                      64, NP, i, j, lane, hi, lo, d.halves);
        if (lane == 0) {
            d.G[i + (size_t)j * n] = hi;
            d.G[j + (size_t)i * n] = hi;
        }
    }
}

// ---------------------------------------------------------------- plain FP64 Gram
constexpr int PLAIN_KC = 64;
constexpr int PLAIN_THREADS = 256;

template <typename T, int MAXP>
__global__ void __launch_bounds__(PLAIN_THREADS)
    gram_plain_kernel(const T* __restrict__ A, int64_t m, int n, int64_t lda, int64_t rows_per_cta,
                      double* __restrict__ part, DevInfo* info) {
    extern __shared__ double tl[];  // [n][PLAIN_KC + 1]
    const int tid = threadIdx.x;
    const int npairs = n * (n + 1) / 2;
    int pi[MAXP], pj[MAXP];
    double acc[MAXP];
#pragma unroll
    for (int k = 0; k < MAXP; ++k) {
        const int idx = tid + k * PLAIN_THREADS;
        int j = 0;
        if (idx < npairs) {
            j = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
            while ((j + 1) * (j + 2) / 2 <= idx) ++j;
            while (j * (j + 1) / 2 > idx) --j;
        }
        pj[k] = j;
        pi[k] = idx < npairs ? idx - j * (j + 1) / 2 : 0;
        acc[k] = 0.0;
    }
    bool bad = false;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r_end = min(m, r_begin + rows_per_cta);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += PLAIN_KC) {
        const int rows = (r_end - r0 < (int64_t)PLAIN_KC) ? (int)(r_end - r0) : PLAIN_KC;
        for (int idx = tid; idx < n * PLAIN_KC; idx += PLAIN_THREADS) {
            const int j = idx / PLAIN_KC, rr = idx % PLAIN_KC;
            double v = 0.0;
            if (rr < rows) v = (double)A[(size_t)j * lda + r0 + rr];
            if (!isfinite(v)) { bad = true; v = 0.0; }
            tl[j * (PLAIN_KC + 1) + rr] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < MAXP; ++k) {
            if (tid + k * PLAIN_THREADS < npairs) {
                const double* x = tl + pi[k] * (PLAIN_KC + 1);
                const double* y = tl + pj[k] * (PLAIN_KC + 1);
                double s = acc[k];
                for (int r = 0; r < PLAIN_KC; ++r) s = fma(x[r], y[r], s);
                acc[k] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < MAXP; ++k) {
        const int idx = tid + k * PLAIN_THREADS;
        if (idx < npairs) part[(size_t)blockIdx.x * npairs + idx] = acc[k];
    }
    if (bad) atomicOr(&info->flags, FLAG_NONFINITE);
}

__global__ void gram_plain_combine_kernel(const double* __restrict__ part, int P, int n,
                                          double* __restrict__ G, int64_t ldg) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = n * (n + 1) / 2;
    if (idx >= npairs) return;
    int j = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= idx) ++j;
    while (j * (j + 1) / 2 > idx) --j;
    const int i = idx - j * (j + 1) / 2;
    double s = 0.0;
    for (int c = 0; c < P; ++c) s += part[(size_t)c * npairs + idx];  // fixed order
    G[i + (size_t)j * ldg] = s;
    G[j + (size_t)i * ldg] = s;
}

template <int NP>
cudaError_t launch_ozaki_np(const float* A, int64_t m, int n, int64_t lda, const GramPlan& plan,
                            long long* ph, long long* pl, int* pE, DevInfo* info, cudaStream_t s) {
    const size_t smem = GramSmem<NP>::bytes;
    const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
    cudaError_t e;
    if (vec) {
        e = cudaFuncSetAttribute(gram_ozaki_kernel<NP, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gram_ozaki_kernel<NP, true><<<plan.P, 256, smem, s>>>(A, m, n, lda, plan.rows_per_cta, ph, pl,
                                                              pE, info);
    } else {
        e = cudaFuncSetAttribute(gram_ozaki_kernel<NP, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gram_ozaki_kernel<NP, false><<<plan.P, 256, smem, s>>>(A, m, n, lda, plan.rows_per_cta, ph,
                                                               pl, pE, info);
    }
    return cudaGetLastError();
}

}  // namespace

GramPlan gram_plan(int64_t m, int n, int sm_count, int split_k_opt) {
    GramPlan p;
    p.NP = n <= 16 ? 16 : n <= 32 ? 32 : n <= 48 ? 48 : 64;
    const int64_t chunks = (m + GRAM_KC - 1) / GRAM_KC;
    int64_t P = split_k_opt > 0 ? split_k_opt : sm_count;
    const int64_t min_P = (m + GRAM_MAX_ROWS_PER_CTA - 1) / GRAM_MAX_ROWS_PER_CTA;
    if (P < min_P) P = min_P;
    if (P > chunks) P = chunks;
    if (P < 1) P = 1;
    const int64_t chunks_per = (chunks + P - 1) / P;
    p.rows_per_cta = chunks_per * GRAM_KC;
    p.P = (int)((m + p.rows_per_cta - 1) / p.rows_per_cta);
    if (p.P < 1) p.P = 1;
    return p;
}

size_t gram_partials_bytes(const GramPlan& p) {
    return (size_t)p.P * p.NP * p.NP * sizeof(long long) * 2 + (size_t)p.P * p.NP * sizeof(int) + 256;
}

cudaError_t launch_gram_ozaki(const void* A, int working, int64_t m, int n, int64_t lda,
                              const GramPlan& plan, void* part, DevInfo* info, cudaStream_t s) {
    if (working != 0 || n > 64) return cudaErrorNotSupported;
    long long* ph = reinterpret_cast<long long*>(part);
    long long* pl = ph + (size_t)plan.P * plan.NP * plan.NP;
    int* pE = reinterpret_cast<int*>(pl + (size_t)plan.P * plan.NP * plan.NP);
    const float* Af = reinterpret_cast<const float*>(A);
    switch (plan.NP) {
        case 16: return launch_ozaki_np<16>(Af, m, n, lda, plan, ph, pl, pE, info, s);
        case 32: return launch_ozaki_np<32>(Af, m, n, lda, plan, ph, pl, pE, info, s);
        case 48: return launch_ozaki_np<48>(Af, m, n, lda, plan, ph, pl, pE, info, s);
        default: return launch_ozaki_np<64>(Af, m, n, lda, plan, ph, pl, pE, info, s);
    }
}

cudaError_t launch_gram_combine(const GramPlan& plan, const void* part, int n, double* G,
                                double* G_lo, int64_t ldg, cudaStream_t s) {
    const long long* ph = reinterpret_cast<const long long*>(part);
    const long long* pl = ph + (size_t)plan.P * plan.NP * plan.NP;
    const int* pE = reinterpret_cast<const int*>(pl + (size_t)plan.P * plan.NP * plan.NP);
    const int npairs = n * (n + 1) / 2;
    gram_combine_kernel<<<(npairs + 7) / 8, 256, 0, s>>>(ph, pl, pE, plan.P, plan.NP, n, G, G_lo, ldg, -1, -1, 0,
                                                         n);
    return cudaGetLastError();
}

cudaError_t launch_gram_batch(const BatchInst* inst, const BatchGramItem* items, int nitems, int NP, bool vec,
                              void* part, int total_slots, DevInfo* infos, int grid, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    long long* ph = reinterpret_cast<long long*>(part);
    long long* pl = ph + (size_t)total_slots * BATCH_SLOT;
    int* pE = reinterpret_cast<int*>(pl + (size_t)total_slots * BATCH_SLOT);
    const int g = grid < nitems ? grid : nitems;
#define TSVD_BATCH_NP(NPV)                                                                                        \
    {                                                                                                              \
        const size_t smem = GramSmem<NPV>::bytes;                                                                  \
        if (vec) {                                                                                                 \
            cudaError_t e = cudaFuncSetAttribute(gram_ozaki_batch_kernel<NPV, true>,                               \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
            if (e != cudaSuccess) return e;                                                                        \
            int bps = 1;                                                                                           \
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gram_ozaki_batch_kernel<NPV, true>, 256,      \
                                                              smem) != cudaSuccess || bps < 1)                     \
                bps = 1;                                                                                           \
            const int gg = (int)std::min<long long>((long long)g * bps, nitems);                                   \
            gram_ozaki_batch_kernel<NPV, true><<<gg, 256, smem, s>>>(inst, items, nitems, ph, pl, pE, infos);      \
        } else {                                                                                                   \
            cudaError_t e = cudaFuncSetAttribute(gram_ozaki_batch_kernel<NPV, false>,                              \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
            if (e != cudaSuccess) return e;                                                                        \
            int bps = 1;                                                                                           \
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gram_ozaki_batch_kernel<NPV, false>, 256,     \
                                                              smem) != cudaSuccess || bps < 1)                     \
                bps = 1;                                                                                           \
            const int gg = (int)std::min<long long>((long long)g * bps, nitems);                                   \
            gram_ozaki_batch_kernel<NPV, false><<<gg, 256, smem, s>>>(inst, items, nitems, ph, pl, pE, infos);     \
        }                                                                                                          \
    }
    switch (NP) {
        case 16: TSVD_BATCH_NP(16) break;
        case 32: TSVD_BATCH_NP(32) break;
        case 48: TSVD_BATCH_NP(48) break;
        default: TSVD_BATCH_NP(64) break;
    }
#undef TSVD_BATCH_NP
    return cudaGetLastError();
}

size_t gram_batch_partials_bytes(int total_slots) {
    return (size_t)total_slots * (2 * BATCH_SLOT * sizeof(long long) + 64 * sizeof(int)) + 256;
}

cudaError_t launch_gram_combine_batch(const BatchInst* inst, int count, const void* part, int total_slots,
                                      cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const long long* ph = reinterpret_cast<const long long*>(part);
    const long long* pl = ph + (size_t)total_slots * BATCH_SLOT;
    const int* pE = reinterpret_cast<const int*>(pl + (size_t)total_slots * BATCH_SLOT);
    gram_combine_batch_kernel<<<count, 256, 0, s>>>(inst, ph, pl, pE);
    return cudaGetLastError();
}

cudaError_t launch_gram_combine2(const GramPlan& plan, const void* part, int n, int c1, int c2, int wmask, double* G,
                                 double* G_lo, int64_t ldg, cudaStream_t s) {
    const long long* ph = reinterpret_cast<const long long*>(part);
    const long long* pl = ph + (size_t)plan.P * plan.NP * plan.NP;
    const int* pE = reinterpret_cast<const int*>(pl + (size_t)plan.P * plan.NP * plan.NP);
    const int npairs = 64 * 65 / 2;
    gram_combine_kernel<<<(npairs + 7) / 8, 256, 0, s>>>(ph, pl, pE, plan.P, plan.NP, 64, G, G_lo, ldg, c1, c2, wmask,
                                                         n);
    return cudaGetLastError();
}

static int plain_P(int64_t m, int sm_count) {
    int64_t chunks = (m + PLAIN_KC - 1) / PLAIN_KC;
    int64_t P = 2 * (int64_t)sm_count;
    if (P > chunks) P = chunks;
    return (int)(P < 1 ? 1 : P);
}

size_t gram_plain_partials_bytes(int64_t m, int n, int sm_count) {
    return (size_t)plain_P(m, sm_count) * n * (n + 1) / 2 * sizeof(double) + 256;
}

cudaError_t launch_gram_plain(const void* A, int working, int64_t m, int n, int64_t lda,
                              int sm_count, void* part, double* G, int64_t ldg, DevInfo* info,
                              cudaStream_t s) {
    if (n > 64) return cudaErrorNotSupported;
    int P = plain_P(m, sm_count);
    const int64_t chunks = (m + PLAIN_KC - 1) / PLAIN_KC;
    const int64_t rows_per = (chunks + P - 1) / P * PLAIN_KC;
    P = (int)((m + rows_per - 1) / rows_per);
    const size_t smem = sizeof(double) * n * (PLAIN_KC + 1);
    double* pp = reinterpret_cast<double*>(part);
    if (working == 0)
        gram_plain_kernel<float, 9><<<P, PLAIN_THREADS, smem, s>>>(
            reinterpret_cast<const float*>(A), m, n, lda, rows_per, pp, info);
    else
        gram_plain_kernel<double, 9><<<P, PLAIN_THREADS, smem, s>>>(
            reinterpret_cast<const double*>(A), m, n, lda, rows_per, pp, info);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int npairs = n * (n + 1) / 2;
    gram_plain_combine_kernel<<<(npairs + 127) / 128, 128, 0, s>>>(pp, P, n, G, ldg);
    return cudaGetLastError();
}

}  // namespace tsvd
