// gram_tc.cu -- the higher-precision Gram matrix on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators, TMA), n <= 64, FP32 working precision.
// Alg. 1 lines 1-2, same arithmetic as gram_ozaki.cu (see there for the
// digit split and the error analysis); this file only changes where the
// exact integer sums are formed and how long they accumulate.
//
// Per CTA (one per SM, a contiguous range of rows, 640 threads):
//   warp 0      TMA producer -- 64-row x n FP32 sub-chunks into a 4-stage ring.
//   warp 1      TMEM owner (512 columns) and, on one lane, the MMA issuer.
//   warps 4-19  16 worker warps (4 per scheduler).  Per sub-chunk they split:
//               column maxima -> power-of-two scale E_j, then 7 signed 8-bit
//               digits per entry (|q| <= 128, exact in bf16) written as the
//               K-major, 128-byte-swizzled MMA operand.  When a period ends
//               they drain it: TMEM -> registers -> fixed point, each thread
//               owning one TMEM lane (row i of the Gram, digit half h) and 16
//               columns j.  hi (int64, units 2^(E_i+E_j-47)) takes the digit
//               pairs with s + t <= 4 exactly; lo (int32, units 2^(E_i+E_j-54))
//               takes s + t = 5 exactly and s + t = 6 (weight <= 2^-62) rounded
//               to its grid (at most 2 roundings of 2^-55 per (i, j) per period).
//               The partial is written in units 2^-63 like gram_ozaki.cu.
//
// Operand layout of one digit stage: 7 slices of 64 rows (one row per column
// j of A, 64 K-values = 128 bytes), slice positions holding digits
// (0-based) [6, 0, 1, 4, 2, 3, 5].  Five MMAs per 16-row K-step cover the 16
// digit-pair blocks needed (s <= t, s + t <= 6), each exactly once, in the
// 512 TMEM columns:
//   A=[0;1] x B=[1,4,2,3] (N=256, cols   0..255)
//   A=[0;1] x B=[5]       (N=64,  cols 256..319)
//   A=[6;0] x B=[0]       (N=64,  cols 320..383)
//   A=[4;2] x B=[2]       (N=64,  cols 384..447)
//   A=[2;3] x B=[3]       (N=64,  cols 448..511)
// (lanes 0..63 hold the first digit of A, lanes 64..127 the second).
//
// The FP32 accumulation in TMEM is exact while every partial sum stays below
// 2^24: with |q| <= 128 that is 1024 rows.  A period is closed when its
// budget of 16 units is spent (a sub-chunk costs 1 unit, 64 * 128^2 = 2^20)
// or when some column's scale must grow by more than one binade.  A growth of
// exactly one binade is absorbed in the running period: that column's top
// digit then lies in [-256, 256] (still exact in bf16) and the sub-chunk
// costs 4 units (64 * 256^2 = 2^22); the grown scale takes effect at the next
// period, whose digits are relative to it (the drain first shifts the
// accumulators onto the coarser grid).  Bounds with R <= 2^15 rows per CTA:
// |hi| <= (R + 3 * 1024) 2^47 < 2^62.1, |lo| <= R (2^15 + 2^14) + ... < 2^30.6.  Every wait on an
// mbarrier is bounded; on timeout the kernel records TSVD_ERR_TIMEOUT, stops
// issuing work, drains what it started and frees its TMEM.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tma_util.cuh"

namespace tsvd {
namespace {

constexpr int TC_SUB = 64;           // rows per sub-chunk (= MMA K of one digit stage)
constexpr int TC_PERIOD = 16;        // sub-chunks per exact accumulation period (1024 rows)
constexpr int TC_SF = 4;             // FP32 stages
constexpr int TC_SD = 2;             // digit stages
constexpr int TC_THREADS = 640;   // 4 control warps + 16 workers
constexpr int TC_WORKERS = 512;
constexpr int TC_FP_BYTES = 64 * TC_SUB * 4;       // [64 cols][64 rows] FP32
constexpr int TC_DIG_BYTES = 7 * 64 * 128;         // 7 slices x 64 rows x 128 B
constexpr int TC_SMEM = TC_SD * TC_DIG_BYTES + TC_SF * TC_FP_BYTES + 1024;  // + alignment slack

// slot position of each digit (0-based digit index -> position)
__constant__ int c_pos_of_digit[7] = {1, 2, 4, 5, 3, 6, 0};

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused: swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8-row groups 1024 B apart
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// packed FP32 pairs (two rows of one column), Blackwell f32x2 instructions
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float tc_scale_pow2(float a, int k) {
    const int k1 = k / 2, k2 = k - k1;
    return (a * __int_as_float((k1 + 127) << 23)) * __int_as_float((k2 + 127) << 23);
}
__device__ __forceinline__ int tc_exp_above(float mx) {
    const unsigned b = __float_as_uint(mx);
    const int be = (b >> 23) & 0xff;
    return be == 0 ? -126 : be - 126;
}

struct TcShared {
    uint64_t fp_full[TC_SF], fp_empty[TC_SF];
    uint64_t dig_full[TC_SD], dig_empty[TC_SD];
    uint64_t acc_full, acc_empty;
    uint32_t tmem_base;
    int abort;             // any role gave up (bounded wait expired)
    int wabort;            // workers: uniform abort decision
    int dig_newp[TC_SD];   // sub-chunk starts a new period
    int growth;            // some column scale grew in this sub-chunk
    int E_cur[64];         // scale of the running period
    int E_pend[64];        // largest scale seen so far
    int E_old[64];         // scale of the period being drained
    int E_acc[64];         // scale of the fixed-point accumulators
    int e_sub[64];
};

// Drain one finished period from TMEM into the caller's fixed-point
// accumulators (E_acc -> E_old re-grid first).  All 512 workers call it.
__device__ __forceinline__ void tc_drain(TcShared& S, uint32_t tmem, int wt, int quad, int lane, int J0,
                                         long long (&hi)[16], int (&lo)[16]) {
    const int lanei = quad * 32 + lane;
    const int h = lanei >> 6, i = lanei & 63;
    const int Ei = S.E_old[i], Eai = S.E_acc[i];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int Ej = S.E_old[J0 + k], Eaj = S.E_acc[J0 + k];
        const int sh = (Eai == EXP_EMPTY || Eaj == EXP_EMPTY) ? 64 : (Ei - Eai) + (Ej - Eaj);
        if (sh > 0) {
            hi[k] = sh >= 63 ? 0 : hi[k] >> sh;
            lo[k] = sh >= 31 ? 0 : lo[k] >> sh;
        }
    }
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + J0;
    uint32_t r[16];
    // exact integers |v| <= 2^24: the 1.5 * 2^23 bias converts |v| <= 2^22, F2I the rest
#define TC_CVT(V)                                                                              \
    ((fabsf(V) <= 4194304.0f) ? (__float_as_int((V) + 12582912.0f) - 0x4B400000) : __float2int_rn(V))
#define TC_FOLD(CB, SH)                                                                        \
    {                                                                                          \
        tmem_ld16(trow + (CB) * 64, r);                                                        \
        _Pragma("unroll") for (int k = 0; k < 16; ++k) {                                       \
            const long long iv = (long long)TC_CVT(__uint_as_float(r[k]));                      \
            hi[k] += (long long)((unsigned long long)iv << (SH));                              \
        }                                                                                      \
    }
#define TC_FOLD_LO(CB, RS)                                                                     \
    {                                                                                          \
        tmem_ld16(trow + (CB) * 64, r);                                                        \
        _Pragma("unroll") for (int k = 0; k < 16; ++k) {                                       \
            const int iv = TC_CVT(__uint_as_float(r[k]));                                      \
            lo[k] += (RS) == 0 ? iv : ((iv + (1 << ((RS) > 0 ? (RS) - 1 : 0))) >> (RS));        \
        }                                                                                      \
    }
    if (h == 0) {
        TC_FOLD(0, 25)      // (0,1)
        TC_FOLD(1, 1)       // (0,4)
        TC_FOLD(2, 17)      // (0,2)
        TC_FOLD(3, 9)       // (0,3)
        TC_FOLD_LO(4, 0)    // (0,5)
        TC_FOLD_LO(5, 8)    // (6,0)
        TC_FOLD_LO(6, 8)    // (4,2)
        TC_FOLD_LO(7, 0)    // (2,3)
    } else {
        TC_FOLD(0, 16)      // (1,1) diagonal: 1/2
        TC_FOLD_LO(1, 0)    // (1,4)
        TC_FOLD(2, 9)       // (1,2)
        TC_FOLD(3, 1)       // (1,3)
        TC_FOLD_LO(4, 8)    // (1,5)
        TC_FOLD(5, 32)      // (0,0) diagonal: 1/2
        TC_FOLD(6, 0)       // (2,2) diagonal: 1/2
        TC_FOLD_LO(7, 9)    // (3,3) diagonal: 1/2
    }
#undef TC_FOLD_LO
#undef TC_FOLD
#undef TC_CVT
    tc_fence_before();
    named_bar(1, TC_WORKERS);
    if (wt < 64) S.E_acc[wt] = S.E_old[wt];
    named_bar(1, TC_WORKERS);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmapA, int64_t m, int n, int64_t rows_per_cta,
                   long long* __restrict__ part_hi, long long* __restrict__ part_lo, int* __restrict__ part_E,
                   DevInfo* info) {
    extern __shared__ unsigned char tc_dyn[];
    // 1024-byte alignment for the swizzled operand atoms
    unsigned char* base = tc_dyn + ((1024 - (smem_addr(tc_dyn) & 1023)) & 1023);
    unsigned char* dig = base;                                           // [SD][7*64 rows][128 B]
    float* fpb = reinterpret_cast<float*>(base + TC_SD * TC_DIG_BYTES);  // [SF][64][64]
    __shared__ TcShared S;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r_end = min(m, r_begin + rows_per_cta);
    const int G = r_end > r_begin ? (int)((r_end - r_begin + TC_SUB - 1) / TC_SUB) : 0;

    if (tid == 0) {
        for (int s = 0; s < TC_SF; ++s) { mbar_init(&S.fp_full[s], 1); mbar_init(&S.fp_empty[s], 1); }
        for (int s = 0; s < TC_SD; ++s) { mbar_init(&S.dig_full[s], 1); mbar_init(&S.dig_empty[s], 1); }
        mbar_init(&S.acc_full, 1);
        mbar_init(&S.acc_empty, 1);
        mbar_fence_init();
        S.abort = 0;
        S.wabort = 0;
    }
    if (tid < 64) {
        S.E_cur[tid] = EXP_EMPTY;
        S.E_pend[tid] = EXP_EMPTY;
        S.E_old[tid] = EXP_EMPTY;
        S.E_acc[tid] = EXP_EMPTY;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            smem_addr(&S.tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    int tma_issued = 0;

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 40;");
        if (warp == 0 && lane == 0) {
            // ---------------- TMA producer
            tma_prefetch_desc(&tmapA);
            const unsigned bytes = (unsigned)(TC_SUB * n * 4);
            int issued = 0;
            for (int g = 0; g < G; ++g) {
                const int f = g % TC_SF;
                if (g >= TC_SF && !mbar_wait(&S.fp_empty[f], ((g / TC_SF) - 1) & 1)) {
                    atomicExch(&S.abort, 1);
                    break;
                }
                if (S.abort) break;
                mbar_expect_tx(&S.fp_full[f], bytes);
                tma_load_2d(fpb + (size_t)f * 64 * TC_SUB, &tmapA, (int)(r_begin + (int64_t)g * TC_SUB), 0,
                            &S.fp_full[f]);
                issued = g + 1;
            }
            tma_issued = issued;
        } else if (warp == 1 && lane == 0) {
            // ---------------- MMA issuer
            const uint32_t id256 = idesc_bf16(128, 256), id64 = idesc_bf16(128, 64);
            int period = 0;
            for (int g = 0; g < G; ++g) {
                const int d = g % TC_SD;
                if (!mbar_wait(&S.dig_full[d], (g / TC_SD) & 1) || S.abort) { atomicExch(&S.abort, 1); break; }
                const int newp = S.dig_newp[d];
                if (newp && g > 0) {
                    // close the running period: the workers drain it before it is overwritten
                    mma_commit(&S.acc_full);
                    if (!mbar_wait(&S.acc_empty, period & 1)) { atomicExch(&S.abort, 1); break; }
                    tc_fence_after();
                    ++period;
                }
                const uint32_t sb = smem_addr(dig + (size_t)d * TC_DIG_BYTES);
#pragma unroll
                for (int kk = 0; kk < TC_SUB / 16; ++kk) {
                    const uint32_t acc = (newp && kk == 0) ? 0u : 1u;
                    const uint32_t ko = kk * 32;
                    mma_bf16(tmem + 0, desc_sw128(sb + 1 * 8192 + ko), desc_sw128(sb + 2 * 8192 + ko), id256, acc);
                    mma_bf16(tmem + 256, desc_sw128(sb + 1 * 8192 + ko), desc_sw128(sb + 6 * 8192 + ko), id64, acc);
                    mma_bf16(tmem + 320, desc_sw128(sb + 0 * 8192 + ko), desc_sw128(sb + 1 * 8192 + ko), id64, acc);
                    mma_bf16(tmem + 384, desc_sw128(sb + 3 * 8192 + ko), desc_sw128(sb + 4 * 8192 + ko), id64, acc);
                    mma_bf16(tmem + 448, desc_sw128(sb + 4 * 8192 + ko), desc_sw128(sb + 5 * 8192 + ko), id64, acc);
                }
                mma_commit(&S.dig_empty[d]);
            }
            // the last period (or, after a failure, whatever was accumulated) goes to the workers;
            // every MMA issued by this thread has completed once that phase completes
            mma_commit(&S.acc_full);
            (void)mbar_wait(&S.acc_full, period & 1);
        }
    } else {
        // ---------------- 16 worker warps: split every sub-chunk, drain every period
        asm volatile("setmaxnreg.inc.sync.aligned.u32 104;");
        const int wt = tid - 128;                  // worker thread 0..511
        const int quad = warp & 3;                 // TMEM lane quadrant of this warp
        const int J0 = 16 * ((warp - 4) >> 2);     // columns J0..J0+15 of the drain
        const int half = lane >> 4, q = lane & 15; // split item: column half of the warp, row quad
        const unsigned long long MAGIC = f2_pack(12582912.0f, 12582912.0f);  // 1.5 * 2^23
        const unsigned long long S256 = f2_pack(256.0f, 256.0f);
        long long hi[16];
        int lo[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) { hi[k] = 0; lo[k] = 0; }
        int period_len = 0, drained = 0;
        bool bad = false, aborted = false;
        for (int g = 0; g < G && !aborted; ++g) {
            const int f = g % TC_SF, d = g % TC_SD;
            if (!mbar_wait(&S.fp_full[f], (g / TC_SF) & 1)) atomicOr(&S.wabort, 1);
            if (wt == 0 && S.abort) atomicOr(&S.wabort, 1);
            named_bar(1, TC_WORKERS);
            if (S.wabort) { aborted = true; break; }
            // two items (column j, rows 4q..4q+3) per thread; a half-warp covers one column
            const float* fp = fpb + (size_t)f * 64 * TC_SUB;
            float v[2][4];
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int j = 2 * ((wt >> 5) + 16 * it) + half;
                float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < n) a4 = *reinterpret_cast<const float4*>(fp + j * TC_SUB + 4 * q);
                v[it][0] = a4.x; v[it][1] = a4.y; v[it][2] = a4.z; v[it][3] = a4.w;
                // max |a| on the bit patterns (also exposes Inf / NaN, whose patterns are the largest)
                unsigned mb = max(max(__float_as_uint(a4.x) & 0x7fffffffu, __float_as_uint(a4.y) & 0x7fffffffu),
                                  max(__float_as_uint(a4.z) & 0x7fffffffu, __float_as_uint(a4.w) & 0x7fffffffu));
                mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 1));
                mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 2));
                mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 4));
                mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 8));
                if (mb >= 0x7f800000u) bad = true;
                if (q == 0) S.e_sub[j] = (mb == 0u || mb >= 0x7f800000u) ? EXP_EMPTY : tc_exp_above(__uint_as_float(mb));
            }
            if (wt == 0) S.growth = 0;
            named_bar(1, TC_WORKERS);
            if (wt < 64) {
                // E_pend: largest scale seen; E_cur: scale of the running period.  One binade
                // above E_cur is "soft" (top digit in [-256, 256], still exact in bf16); more,
                // or a first non-zero entry, is "hard" and needs a new period.
                const int e = S.e_sub[wt], cur = S.E_cur[wt];
                S.E_pend[wt] = max(S.E_pend[wt], e);
                if (e != EXP_EMPTY) {
                    if (cur == EXP_EMPTY || e > cur + 1) atomicOr(&S.growth, 2);
                    else if (e == cur + 1) atomicOr(&S.growth, 1);
                }
            }
            named_bar(1, TC_WORKERS);
            // exactness budget of a period: sum |q_s q_t| <= 2^24 per block and (i, j);
            // a normal sub-chunk may add 64 * 128^2 = 2^20 (1 unit), a soft one 2^22 (4 units)
            const int cost = (S.growth & 1) ? 4 : 1;
            const bool newp = (g == 0) || (S.growth & 2) || (period_len + cost > TC_PERIOD);
            if (newp) {
                named_bar(1, TC_WORKERS);  // every worker has read S.growth
                if (wt < 64) {
                    S.E_old[wt] = S.E_cur[wt];    // scale of the period that ends here
                    S.E_cur[wt] = S.E_pend[wt];   // the new period starts on every grown scale
                }
                named_bar(1, TC_WORKERS);
                period_len = 0;
            }
            period_len += newp ? 1 : cost;
            // free digit stage?
            if (g >= TC_SD && !mbar_wait(&S.dig_empty[d], ((g / TC_SD) - 1) & 1)) atomicOr(&S.wabort, 1);
            named_bar(1, TC_WORKERS);
            if (S.wabort) { aborted = true; break; }
            unsigned char* ds = dig + (size_t)d * TC_DIG_BYTES;
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int j = 2 * ((wt >> 5) + 16 * it) + half;
                const int E = S.E_cur[j];
                // y = 128 a 2^-E (|y| < 256); digit q = RN(y) by the 1.5*2^23 bias; y <- 256 (y - q)
                unsigned long long y01 = 0ull, y23 = 0ull;
                if (E != EXP_EMPTY) {
                    const int k = 7 - E;
                    y01 = f2_pack(tc_scale_pow2(v[it][0], k), tc_scale_pow2(v[it][1], k));
                    y23 = f2_pack(tc_scale_pow2(v[it][2], k), tc_scale_pow2(v[it][3], k));
                }
#pragma unroll
                for (int sdig = 0; sdig < 7; ++sdig) {
                    const unsigned long long q01 = f2_sub(f2_add(y01, MAGIC), MAGIC);
                    const unsigned long long q23 = f2_sub(f2_add(y23, MAGIC), MAGIC);
                    float a0, a1, a2, a3;
                    f2_unpack(q01, a0, a1);
                    f2_unpack(q23, a2, a3);
                    const __nv_bfloat162 b01 = __floats2bfloat162_rn(a0, a1);
                    const __nv_bfloat162 b23 = __floats2bfloat162_rn(a2, a3);
                    y01 = f2_mul(f2_sub(y01, q01), S256);
                    y23 = f2_mul(f2_sub(y23, q23), S256);
                    const int row = c_pos_of_digit[sdig] * 64 + j;
                    uint2* dst = reinterpret_cast<uint2*>(ds + row * 128 + (((q >> 1) ^ (row & 7)) << 4) + ((q & 1) << 3));
                    *dst = make_uint2(*reinterpret_cast<const uint32_t*>(&b01), *reinterpret_cast<const uint32_t*>(&b23));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            named_bar(1, TC_WORKERS);
            if (wt == 0) {
                S.dig_newp[d] = newp ? 1 : 0;
                mbar_arrive(&S.dig_full[d]);
                mbar_arrive(&S.fp_empty[f]);
            }
            if (newp && g > 0) {
                // the MMA issuer closes the previous period on seeing this stage; drain it
                if (!mbar_wait(&S.acc_full, drained & 1)) atomicOr(&S.wabort, 1);
                tc_fence_after();
                named_bar(1, TC_WORKERS);
                if (S.wabort) { aborted = true; break; }
                tc_drain(S, tmem, wt, quad, lane, J0, hi, lo);
                if (wt == 0) mbar_arrive(&S.acc_empty);
                ++drained;
            }
        }
        // the last period
        if (!aborted && G > 0) {
            if (wt < 64) S.E_old[wt] = S.E_cur[wt];
            if (!mbar_wait(&S.acc_full, drained & 1)) atomicOr(&S.wabort, 1);
            tc_fence_after();
            named_bar(1, TC_WORKERS);
            if (!S.wabort) tc_drain(S, tmem, wt, quad, lane, J0, hi, lo);
        }
        if (bad) atomicOr(&info->flags, FLAG_NONFINITE);
        // partials of this CTA: W = sum over blocks (s < t) + 1/2 (s = s); G = W + W^T later.
        // The two digit halves of row i add into the same W(i, j): half 0 first, then half 1.
        const int lanei = quad * 32 + lane, h = lanei >> 6, i = lanei & 63;
        long long* ph = part_hi + (size_t)blockIdx.x * 64 * 64;
        long long* pl = part_lo + (size_t)blockIdx.x * 64 * 64;
        for (int hh = 0; hh < 2; ++hh) {
            if (h == hh) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const long long l63 = (long long)((unsigned long long)(long long)lo[k] << 9);
                    if (hh == 0) { ph[i * 64 + J0 + k] = hi[k]; pl[i * 64 + J0 + k] = l63; }
                    else { ph[i * 64 + J0 + k] += hi[k]; pl[i * 64 + J0 + k] += l63; }
                }
            }
            __threadfence_block();
            named_bar(1, TC_WORKERS);
        }
        if (wt < 64) part_E[(size_t)blockIdx.x * 64 + wt] = S.E_acc[wt];
        if (wt == 0 && S.wabort) atomicExch(&S.abort, 1);
    }
    // teardown: every tcgen05 access is complete before the TMEM is freed
    tc_fence_before();
    __syncthreads();
    if (S.abort && tid == 0) {
        atomicOr(&info->flags, FLAG_TIMEOUT);
        // no TMA write may land after the CTA exits: wait (bounded) for the last loads
        for (int g = (tma_issued > TC_SF ? tma_issued - TC_SF : 0); g < tma_issued; ++g)
            (void)mbar_wait(&S.fp_full[g % TC_SF], (g / TC_SF) & 1);
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

}  // namespace

bool gram_tc_ok(const void* A, int working, int n, int64_t lda) {
    return working == 0 && n >= 1 && n <= 64 && ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
}

GramPlan gram_tc_plan(int64_t m, int n, int sm_count, int split_k_opt) {
    GramPlan p;
    p.NP = 64;
    const int64_t subs = (m + TC_SUB - 1) / TC_SUB;
    int64_t P = split_k_opt > 0 ? split_k_opt : sm_count;
    const int64_t min_P = (m + GRAM_MAX_ROWS_PER_CTA - 1) / GRAM_MAX_ROWS_PER_CTA;
    if (P < min_P) P = min_P;
    if (P > subs) P = subs;
    if (P < 1) P = 1;
    p.rows_per_cta = (subs + P - 1) / P * TC_SUB;
    p.P = (int)((m + p.rows_per_cta - 1) / p.rows_per_cta);
    if (p.P < 1) p.P = 1;
    (void)n;
    return p;
}

cudaError_t launch_gram_tc(const void* A, int64_t m, int n, int64_t lda, const GramPlan& plan, void* part,
                           DevInfo* info, cudaStream_t s) {
    CUtensorMap tmap;
    cudaError_t e = make_tmap_2d(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), A, (uint64_t)m, (uint64_t)n,
                                 (uint64_t)lda, TC_SUB, (uint32_t)n, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (e != cudaSuccess) return e;
    long long* ph = reinterpret_cast<long long*>(part);
    long long* pl = ph + (size_t)plan.P * 64 * 64;
    int* pE = reinterpret_cast<int*>(pl + (size_t)plan.P * 64 * 64);
    e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    gram_tc_kernel<<<plan.P, TC_THREADS, TC_SMEM, s>>>(tmap, m, n, plan.rows_per_cta, ph, pl, pE, info);
    return cudaGetLastError();
}

}  // namespace tsvd
