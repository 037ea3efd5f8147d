// gram_tc.cu -- the higher-precision Gram matrix on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators, TMA), n <= 64, FP32 working precision.
// Alg. 1 lines 1-2, same arithmetic as gram_ozaki.cu (see there for the
// digit split and the error analysis); this file only changes where the
// exact integer sums are formed and how long they accumulate.
//
// Per CTA (one per SM, a contiguous range of rows, 4 warpgroups):
//   WG0  warp 0: TMA producer -- 64-row x n FP32 sub-chunks into a 4-stage ring.
//        warp 1: TMEM owner (512 columns) and, on one lane, the MMA issuer.
//   WG1  digit split -- per sub-chunk: column maxima -> running power-of-two
//        scale E_j, then 7 signed 8-bit digits per entry (|q| <= 128, exact in
//        bf16) written as the K-major, 128-byte-swizzled MMA operand.
//   WG2, WG3  drain -- per accumulation period: TMEM -> registers -> fixed
//        point: hi (int64, units 2^(E_i+E_j-47)) takes the digit pairs with
//        s + t <= 4 exactly; lo (int32, units 2^(E_i+E_j-54)) takes s + t = 5
//        exactly and s + t = 6 (weight <= 2^-62) rounded to its grid, at most
//        2 roundings of 2^-55 per (i, j) per 1024 rows.  Over <= 32 periods
//        |lo| < 2^31; the partial is written in units 2^-63 like gram_ozaki.cu.
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
// 2^24: with |q| <= 128 that is 1024 rows.  A period therefore spans at most
// 16 sub-chunks, and ends early when some column's scale E_j grows (the
// digits of the new period are relative to the new scale; the drain shifts
// the int64 accumulators onto the coarser grid first).  Every wait on an
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
constexpr int TC_THREADS = 512;
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
    uint64_t rec_full[2], rec_empty[2];
    uint32_t tmem_base;
    int abort;             // any role gave up (bounded wait expired)
    int sabort;            // split group: uniform abort decision
    int dabort;            // drain group: uniform abort decision
    int dig_newp[TC_SD];   // sub-chunk starts a new period
    int acc_last;          // the period being drained is the last one
    int growth;            // split: some column scale grew in this sub-chunk
    int E_cur[64];         // split: running scales
    int e_sub[64];
    int rec_E[2][64];      // scale of each period (ring of 2)
    int E_last[64];        // drain: scale of the accumulators
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmapA, int64_t m, int n, int64_t rows_per_cta,
                   long long* __restrict__ part_hi, long long* __restrict__ part_lo, int* __restrict__ part_E,
                   DevInfo* info) {
    extern __shared__ unsigned char tc_dyn[];
    // 1024-byte alignment for the swizzled operand atoms
    unsigned char* base = tc_dyn + ((1024 - (smem_addr(tc_dyn) & 1023)) & 1023);
    unsigned char* dig = base;                              // [SD][7*64 rows][128 B]
    float* fpb = reinterpret_cast<float*>(base + TC_SD * TC_DIG_BYTES);  // [SF][64][64]
    __shared__ TcShared S;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, wg = warp >> 2;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r_end = min(m, r_begin + rows_per_cta);
    const int G = r_end > r_begin ? (int)((r_end - r_begin + TC_SUB - 1) / TC_SUB) : 0;

    if (tid == 0) {
        for (int s = 0; s < TC_SF; ++s) { mbar_init(&S.fp_full[s], 1); mbar_init(&S.fp_empty[s], 1); }
        for (int s = 0; s < TC_SD; ++s) { mbar_init(&S.dig_full[s], 1); mbar_init(&S.dig_empty[s], 1); }
        mbar_init(&S.acc_full, 2);  // tcgen05.commit + the MMA thread's own arrive
        mbar_init(&S.acc_empty, 1);
        for (int s = 0; s < 2; ++s) { mbar_init(&S.rec_full[s], 1); mbar_init(&S.rec_empty[s], 1); }
        mbar_fence_init();
        S.abort = 0;
        S.sabort = 0;
        S.dabort = 0;
        S.acc_last = 0;
    }
    if (tid < 64) { S.E_cur[tid] = EXP_EMPTY; S.E_last[tid] = EXP_EMPTY; }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            smem_addr(&S.tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    if (wg == 0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 56;");
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
            if (S.abort) {
                // no TMA write may land after the CTA exits: wait (bounded) for the last loads
                for (int g = (issued > TC_SF ? issued - TC_SF : 0); g < issued; ++g)
                    (void)mbar_wait(&S.fp_full[g % TC_SF], (g / TC_SF) & 1);
            }
        } else if (warp == 1 && lane == 0) {
            // ---------------- MMA issuer
            const uint32_t id256 = idesc_bf16(128, 256), id64 = idesc_bf16(128, 64);
            int period = 0;
            for (int g = 0; g < G; ++g) {
                const int d = g % TC_SD;
                if (!mbar_wait(&S.dig_full[d], (g / TC_SD) & 1) || S.abort) { atomicExch(&S.abort, 1); break; }
                const int newp = S.dig_newp[d];
                if (newp && g > 0) {
                    // close the running period: drain it before overwriting the accumulators
                    S.acc_last = 0;
                    mma_commit(&S.acc_full);
                    mbar_arrive(&S.acc_full);
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
            // the last period (or, after a failure, whatever was accumulated) goes to the drain
            S.acc_last = 1;
            if (S.abort || G == 0) atomicExch(&S.abort, 1);
            mma_commit(&S.acc_full);
            mbar_arrive(&S.acc_full);
            // every MMA issued by this thread has completed once acc_full's phase completes
            (void)mbar_wait(&S.acc_full, period & 1);
        }
    } else if (wg == 1) {
        // ---------------- digit split (128 threads)
        asm volatile("setmaxnreg.dec.sync.aligned.u32 112;");
        const int st = tid - 128, sw = st >> 5;  // split thread / warp
        const int colsub = lane >> 3, oct = lane & 7;  // 4 columns x 8 row-octets per warp pass
        int period_len = 0, period = 0;
        bool bad = false;
        for (int g = 0; g < G; ++g) {
            const int f = g % TC_SF, d = g % TC_SD;
            if (!mbar_wait(&S.fp_full[f], (g / TC_SF) & 1)) atomicOr(&S.sabort, 1);
            if (st == 0 && S.abort) atomicOr(&S.sabort, 1);
            named_bar(1, 128);
            if (S.sabort) break;
            const float* fp = fpb + (size_t)f * 64 * TC_SUB;
            float v[4][8];
#pragma unroll
            for (int ps = 0; ps < 4; ++ps) {
                const int j = 16 * ps + 4 * sw + colsub;
                const float4* src = reinterpret_cast<const float4*>(fp + j * TC_SUB + 8 * oct);
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                if (j < n) { a = src[0]; b = src[1]; }
                v[ps][0] = a.x; v[ps][1] = a.y; v[ps][2] = a.z; v[ps][3] = a.w;
                v[ps][4] = b.x; v[ps][5] = b.y; v[ps][6] = b.z; v[ps][7] = b.w;
                float mx = 0.f;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if (!isfinite(v[ps][e])) { bad = true; v[ps][e] = 0.f; }
                    mx = fmaxf(mx, fabsf(v[ps][e]));
                }
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
                if (oct == 0) S.e_sub[j] = (mx == 0.f) ? EXP_EMPTY : tc_exp_above(mx);
            }
            if (st == 0) S.growth = 0;
            named_bar(1, 128);
            if (st < 64) {
                const int old = S.E_cur[st], nw = max(old, S.e_sub[st]);
                if (nw != old) { S.E_cur[st] = nw; atomicOr(&S.growth, 1); }
            }
            named_bar(1, 128);
            const bool newp = (g == 0) || (S.growth != 0) || (period_len == TC_PERIOD);
            if (newp) {
                // publish the scale of the new period (ring of 2 records)
                if (st == 0 && period >= 2 && !mbar_wait(&S.rec_empty[period & 1], ((period >> 1) - 1) & 1))
                    atomicOr(&S.sabort, 1);
                named_bar(1, 128);
                if (S.sabort) break;
                if (st < 64) S.rec_E[period & 1][st] = S.E_cur[st];
                named_bar(1, 128);
                if (st == 0) mbar_arrive(&S.rec_full[period & 1]);
                period_len = 0;
                ++period;
            }
            ++period_len;
            // free digit stage?
            if (g >= TC_SD && !mbar_wait(&S.dig_empty[d], ((g / TC_SD) - 1) & 1)) atomicOr(&S.sabort, 1);
            named_bar(1, 128);
            if (S.sabort) break;
            unsigned char* ds = dig + (size_t)d * TC_DIG_BYTES;
#pragma unroll
            for (int ps = 0; ps < 4; ++ps) {
                const int j = 16 * ps + 4 * sw + colsub;
                const int E = S.E_cur[j];
                float y[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) y[e] = (E == EXP_EMPTY) ? 0.f : tc_scale_pow2(v[ps][e], 7 - E);
#pragma unroll
                for (int s = 0; s < 7; ++s) {
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float q0 = rintf(y[2 * e]), q1 = rintf(y[2 * e + 1]);
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(q0, q1);
                        w[e] = *reinterpret_cast<const uint32_t*>(&b2);
                        y[2 * e] = (y[2 * e] - q0) * 256.f;
                        y[2 * e + 1] = (y[2 * e + 1] - q1) * 256.f;
                    }
                    const int row = c_pos_of_digit[s] * 64 + j;
                    uint4* dst = reinterpret_cast<uint4*>(ds + row * 128 + ((oct ^ (row & 7)) << 4));
                    *dst = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            named_bar(1, 128);
            if (st == 0) {
                S.dig_newp[d] = newp ? 1 : 0;
                mbar_arrive(&S.dig_full[d]);
                mbar_arrive(&S.fp_empty[f]);
            }
        }
        if (bad) atomicOr(&info->flags, FLAG_NONFINITE);
        if (st == 0 && S.sabort) atomicExch(&S.abort, 1);
    } else {
        // ---------------- drain (256 threads): TMEM -> exact int64 fixed point
        asm volatile("setmaxnreg.inc.sync.aligned.u32 168;");
        const int quad = warp & 3;
        const int lanei = quad * 32 + lane;        // TMEM lane
        const int h = lanei >> 6, i = lanei & 63;  // digit half of A, row i of the Gram
        const int J0 = (wg == 2) ? 0 : 32;
        long long hi[32];
        int lo[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) { hi[k] = 0; lo[k] = 0; }
        const int dt = tid - 256;  // drain thread 0..255
        for (int p = 0;; ++p) {
            if (!mbar_wait(&S.acc_full, p & 1)) atomicOr(&S.dabort, 1);
            tc_fence_after();
            const bool last = S.acc_last != 0;
            if (dt == 0 && S.abort) atomicOr(&S.dabort, 1);
            named_bar(2, 256);
            if (S.dabort) break;
            if (!mbar_wait(&S.rec_full[p & 1], (p >> 1) & 1)) atomicOr(&S.dabort, 1);
            named_bar(2, 256);
            if (S.dabort) break;
            // re-grid the accumulators if the scales grew
            const int Ei = S.rec_E[p & 1][i], Eli = S.E_last[i];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int Ej = S.rec_E[p & 1][J0 + k], Elj = S.E_last[J0 + k];
                const int sh = (Eli == EXP_EMPTY || Elj == EXP_EMPTY) ? 64 : (Ei - Eli) + (Ej - Elj);
                if (sh > 0) {
                    hi[k] = sh >= 63 ? 0 : hi[k] >> sh;
                    lo[k] = sh >= 31 ? 0 : lo[k] >> sh;
                }
            }
            const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + J0;
            uint32_t r[16];
            // fold: (column block, half) -> (accumulator, shift); values are exact integers < 2^24
#define TC_FOLD(CB, ACC, SH)                                                                   \
    _Pragma("unroll") for (int half = 0; half < 2; ++half) {                                  \
        tmem_ld16(trow + (CB) * 64 + 16 * half, r);                                           \
        _Pragma("unroll") for (int k = 0; k < 16; ++k) {                                      \
            const long long iv = (long long)__float2int_rn(__uint_as_float(r[k]));             \
            ACC[16 * half + k] += (long long)((unsigned long long)iv << (SH));                 \
        }                                                                                     \
    }
// lo: exact (SH = 0) or rounded right shift by RS
#define TC_FOLD_LO(CB, RS)                                                                     \
    _Pragma("unroll") for (int half = 0; half < 2; ++half) {                                  \
        tmem_ld16(trow + (CB) * 64 + 16 * half, r);                                           \
        _Pragma("unroll") for (int k = 0; k < 16; ++k) {                                      \
            const int iv = __float2int_rn(__uint_as_float(r[k]));                              \
            lo[16 * half + k] += (RS) == 0 ? iv : ((iv + (1 << ((RS) > 0 ? (RS) - 1 : 0))) >> (RS)); \
        }                                                                                     \
    }
            if (h == 0) {
                TC_FOLD(0, hi, 25)   // (0,1)
                TC_FOLD(1, hi, 1)    // (0,4)
                TC_FOLD(2, hi, 17)   // (0,2)
                TC_FOLD(3, hi, 9)    // (0,3)
                TC_FOLD_LO(4, 0)     // (0,5)
                TC_FOLD_LO(5, 8)     // (6,0)
                TC_FOLD_LO(6, 8)     // (4,2)
                TC_FOLD_LO(7, 0)     // (2,3)
            } else {
                TC_FOLD(0, hi, 16)   // (1,1) diagonal: 1/2
                TC_FOLD_LO(1, 0)     // (1,4)
                TC_FOLD(2, hi, 9)    // (1,2)
                TC_FOLD(3, hi, 1)    // (1,3)
                TC_FOLD_LO(4, 8)     // (1,5)
                TC_FOLD(5, hi, 32)   // (0,0) diagonal: 1/2
                TC_FOLD(6, hi, 0)    // (2,2) diagonal: 1/2
                TC_FOLD_LO(7, 9)     // (3,3) diagonal: 1/2
            }
#undef TC_FOLD_LO
#undef TC_FOLD
            tc_fence_before();
            named_bar(2, 256);
            if (dt < 64) S.E_last[dt] = S.rec_E[p & 1][dt];
            named_bar(2, 256);
            if (dt == 0) {
                mbar_arrive(&S.rec_empty[p & 1]);
                mbar_arrive(&S.acc_empty);
            }
            if (last) break;
        }
        // partials of this CTA: W = sum over blocks (s < t) + 1/2 (s = s); G = W + W^T later
        long long* ph = part_hi + (size_t)blockIdx.x * 64 * 64;
        long long* pl = part_lo + (size_t)blockIdx.x * 64 * 64;
        // the two digit halves of row i add into the same W(i, j): half 0 first, then half 1
        for (int hh = 0; hh < 2; ++hh) {
            if (h == hh) {
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const long long l63 = (long long)((unsigned long long)(long long)lo[k] << 9);
                    if (hh == 0) { ph[i * 64 + J0 + k] = hi[k]; pl[i * 64 + J0 + k] = l63; }
                    else { ph[i * 64 + J0 + k] += hi[k]; pl[i * 64 + J0 + k] += l63; }
                }
            }
            __threadfence_block();
            named_bar(2, 256);
        }
        if (dt < 64) part_E[(size_t)blockIdx.x * 64 + dt] = S.E_last[dt];
        if (dt == 0 && S.dabort) atomicExch(&S.abort, 1);
    }
    // teardown: every tcgen05 access is complete before the TMEM is freed
    tc_fence_before();
    __syncthreads();
    if (S.abort && tid == 0) atomicOr(&info->flags, FLAG_TIMEOUT);
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
