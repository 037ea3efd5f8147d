// gram_tc.cu -- the higher-precision Gram matrix on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators, TMA), n <= 64, FP32 working precision.
// Alg. 1 lines 1-2, same arithmetic as gram_ozaki.cu (see there for the
// digit split and the error analysis); this file only changes where the
// exact integer sums are formed and how long they accumulate.
//
// Per CTA (one per SM, every P-th 64-row sub-chunk, 640 threads):
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

#include <cstring>

#include "internal.cuh"
#include "tma_util.cuh"

namespace tsvd {
namespace {

constexpr int TC_SUB = 64;           // rows per sub-chunk (= MMA K of one digit stage)
constexpr int TC_PERIOD = 16;        // sub-chunks per exact accumulation period (1024 rows)
constexpr int TC_SF = 6;             // FP32 stages
constexpr int TC_SD = 2;             // digit stages
constexpr int TC_MX = 4;             // column-maxima slots (the workers publish two sub-chunks ahead)
constexpr int TC_THREADS = 640;   // 4 control warps + 16 workers
constexpr int TC_WORKERS = 512;
constexpr int TC_RD = 8;              // decision records
constexpr int BAR_DEC = 1, BAR_WORK = 2;  // named barrier ids: the two decider warps, the workers
constexpr int TC_FP_BYTES = 64 * TC_SUB * 4;       // [64 cols][64 rows] FP32
constexpr int TC_DIG_BYTES = 7 * 64 * 128;         // 7 slices x 64 rows x 128 B
constexpr int TC_SMEM = TC_SD * TC_DIG_BYTES + TC_SF * TC_FP_BYTES + 1024;  // + alignment slack

// slot position of each digit (0-based digit index -> position)
__host__ __device__ constexpr int tc_pos_of_digit(int s) {
    return s == 0 ? 1 : s == 1 ? 2 : s == 2 ? 4 : s == 3 ? 5 : s == 4 ? 3 : s == 5 ? 6 : 0;
}

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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
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
__device__ __forceinline__ int tc_exp_above(float mx) {
    const unsigned b = __float_as_uint(mx);
    const int be = (b >> 23) & 0xff;
    return be == 0 ? -126 : be - 126;
}

// The deciders' decision on one sub-chunk, read by the workers and the MMA issuer.
struct TcRecord {
    int newp;      // the sub-chunk opens a new period (the previous one is drained first)
    int regrid[2]; // per decider warp: some dsh of its columns is non-zero
    int pad;
    int E[64];     // scale of each column for this sub-chunk's digits
    int dsh[64];   // when newp: E_old - E_acc of the period that ends (0 while nothing was accumulated)
};

struct TcShared {
    uint64_t fp_full[TC_SF], fp_empty[TC_SF];
    uint64_t dig_full[TC_SD], dig_empty[TC_SD];
    uint64_t dec_full[TC_RD], dec_empty[TC_RD];
    uint64_t max_full[TC_MX];  // per sub-chunk (mod TC_MX): the workers have published its column maxima
    uint64_t acc_full, acc_empty;
    TcRecord rec[TC_RD];
    int dflags[2][2];      // decider warps: growth (soft 1, hard 2) and abort (4) bits, double-buffered
    uint32_t tmem_base;
    int abort;             // some role gave up (bounded wait expired)
    int dig_newp[TC_SD];   // the sub-chunk in this digit stage opens a new period
    unsigned colmax[TC_MX][64];  // per sub-chunk (mod TC_MX): max |a| of each column (float bit pattern)
};

// Bit pattern of the float 1.5 * 2^e.  Adding it to a float x with |x| <= 2^(e-1)
// rounds x to the grid 2^(e-23); the low mantissa bits of the sum then hold that
// integer, offset by the pattern itself.
__host__ __device__ constexpr uint32_t tc_magic(int e) { return ((uint32_t)(e + 127) << 23) | 0x400000u; }
// the same constant in both halves of an f32x2 pair
__host__ __device__ constexpr unsigned long long tc_magic2(int e) {
    return ((unsigned long long)tc_magic(e) << 32) | tc_magic(e);
}

// Fold rules of one TMEM column block (digit pair (s, t), w = 8 (s + t)): the
// block holds P * 2^-w, P the exact integer sum of the digit products.
//   kind 0: hi += P * 2^SH       (P split into RN(P / 2^G) * 2^G + rest, both exact)
//   kind 1: lo += P              (same split)
//   kind 2: lo += RN(P / 2^RS)   (s + t = 6 only)
// Every magic add leaves its constant's pattern in the sum; those offsets are
// constants per block and are removed once per drain (modular arithmetic).
struct TcFold { int kind, w, sh, g; };
__host__ __device__ constexpr TcFold tc_fold(int h, int cb) {
    // h = 0: A holds digit 0; h = 1: digit 1 (cover: B = [1, 4, 2, 3], then [5], and
    // the three 64-wide MMAs [6;0]x[0], [4;2]x[2], [2;3]x[3])
    return h == 0 ? (cb == 0 ? TcFold{0, 8, 25, 6}      // (0,1)
                   : cb == 1 ? TcFold{0, 32, 1, 12}    // (0,4)
                   : cb == 2 ? TcFold{0, 16, 17, 12}   // (0,2)
                   : cb == 3 ? TcFold{0, 24, 9, 12}    // (0,3)
                   : cb == 4 ? TcFold{1, 40, 0, 12}    // (0,5)
                   : cb == 5 ? TcFold{2, 48, 8, 0}     // (6,0)
                   : cb == 6 ? TcFold{2, 48, 8, 0}     // (4,2)
                             : TcFold{1, 40, 0, 12})   // (2,3)
                  : (cb == 0 ? TcFold{0, 16, 16, 12}   // (1,1) diagonal: 1/2
                   : cb == 1 ? TcFold{1, 40, 0, 12}    // (1,4)
                   : cb == 2 ? TcFold{0, 24, 9, 12}    // (1,2)
                   : cb == 3 ? TcFold{0, 32, 1, 12}    // (1,3)
                   : cb == 4 ? TcFold{2, 48, 8, 0}     // (1,5)
                   : cb == 5 ? TcFold{0, 0, 32, 12}    // (0,0) diagonal: 1/2
                   : cb == 6 ? TcFold{0, 32, 0, 12}    // (2,2) diagonal: 1/2
                             : TcFold{2, 48, 9, 0});   // (3,3) diagonal: 1/2
}
// A block of kind 0 adds y = (a << g) + b (mod 2^32) to hi, shifted by sh: a and b are the
// bit patterns of 1.5 2^(23+g-w) + a' 2^(g-w) and 1.5 2^(23-w) + b' 2^-w, so y is the block's
// value P = a' 2^g + b' (|P| <= 2^24) plus a constant bias that keeps y inside [0, 2^32)
// (no data-dependent wrap), and hi gets P 2^sh plus the bias 2^sh.
__host__ __device__ constexpr uint32_t tc_fold_bias(TcFold f) {
    return (uint32_t)((tc_magic(23 + f.g - f.w) << f.g) + tc_magic(23 - f.w));
}
__host__ __device__ constexpr bool tc_fold_nowrap(TcFold f) {
    return tc_fold_bias(f) >= (1u << 24) && tc_fold_bias(f) <= 0xffffffffu - (1u << 24);
}
__host__ __device__ constexpr unsigned long long tc_hi_offset(int h) {
    unsigned long long o = 0;
    for (int cb = 0; cb < 8; ++cb) {
        const TcFold f = tc_fold(h, cb);
        if (f.kind == 0) o += (unsigned long long)tc_fold_bias(f) << f.sh;
    }
    return o;
}
__host__ __device__ constexpr uint32_t tc_lo_offset(int h) {
    uint32_t o = 0;
    for (int cb = 0; cb < 8; ++cb) {
        const TcFold f = tc_fold(h, cb);
        if (f.kind == 1) o += (tc_magic(23 + f.g - f.w) << f.g) + tc_magic(23 - f.w);
        if (f.kind == 2) o += tc_magic(23 + f.sh - f.w);
    }
    return o;
}

// Residuals of the s + t = 6 blocks: kind 2 adds RN(P / 2^RS) to lo and keeps the exact
// remainder P - RN(P / 2^RS) 2^RS (|.| <= 2^(RS - 1)) in units of 2^-9 of lo's unit (an
// off-diagonal block's remainder counts twice, the diagonal (3,3) block's once): two 16-bit
// sums per 32-bit register, columns k and k + 8 (|sum| < 2^15 for R <= 2^15 rows: two blocks
// of at most 2^9 per 1024-row period).  With them every digit-pair product is accumulated
// exactly.
__device__ __forceinline__ void tc_res_add(uint32_t (&res)[8], int kk, int r) {
    res[kk & 7] += (kk < 8) ? (uint32_t)r : ((uint32_t)r << 16);
}
__device__ __forceinline__ int tc_res_get(const uint32_t (&res)[8], int kk) {
    const int v = (int)res[kk & 7];
    const int low = (int)(short)(v & 0xffff);
    return kk < 8 ? low : ((v - low) >> 16);
}

template <int H, int CB>
__device__ __forceinline__ void tc_fold_block(uint32_t trow, unsigned long long (&hi)[16], uint32_t (&lo)[16],
                                              uint32_t (&res)[8]) {
    constexpr TcFold F = tc_fold(H, CB);
    // two halves of 8 columns keep the temporaries few (the accumulators use 56 registers)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
        uint32_t r[8];
        tmem_ld8(trow + CB * 64 + 8 * hf, r);
        if constexpr (F.kind == 2) {
            constexpr unsigned long long C = tc_magic2(23 + F.sh - F.w), CR = tc_magic2(23 - F.w);
            constexpr uint32_t PR = tc_magic(23 - F.w);
            constexpr int RW = F.sh == 8 ? 2 : 1;  // remainder weight in units 2^-9 of lo's unit
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const unsigned long long v = f2_pack(__uint_as_float(r[k]), __uint_as_float(r[k + 1]));
                const unsigned long long t = f2_add(v, C);                  // RN(P / 2^RS) in the low bits
                const unsigned long long u = f2_add(f2_sub(v, f2_sub(t, C)), CR);  // the exact remainder
                float t0, t1, u0, u1;
                f2_unpack(t, t0, t1);
                f2_unpack(u, u0, u1);
                lo[8 * hf + k] += __float_as_uint(t0);
                lo[8 * hf + k + 1] += __float_as_uint(t1);
                tc_res_add(res, 8 * hf + k, RW * (int)(__float_as_uint(u0) - PR));
                tc_res_add(res, 8 * hf + k + 1, RW * (int)(__float_as_uint(u1) - PR));
            }
        } else {
            constexpr unsigned long long C1 = tc_magic2(23 + F.g - F.w), C2 = tc_magic2(23 - F.w);
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const int kk = 8 * hf + k;
                const unsigned long long v = f2_pack(__uint_as_float(r[k]), __uint_as_float(r[k + 1]));
                const unsigned long long t1 = f2_add(v, C1);                 // RN(P / 2^G) in the low bits
                const unsigned long long t2 = f2_add(f2_sub(v, f2_sub(t1, C1)), C2);  // P - RN(P / 2^G) 2^G
                float x0, x1, y0, y1;
                f2_unpack(t1, x0, x1);
                f2_unpack(t2, y0, y1);
                const uint32_t a0 = __float_as_uint(x0), a1 = __float_as_uint(x1);
                const uint32_t b0 = __float_as_uint(y0), b1 = __float_as_uint(y1);
                if constexpr (F.kind == 1) {
                    lo[kk] += (a0 << F.g) + b0;
                    lo[kk + 1] += (a1 << F.g) + b1;
                } else {
                    static_assert(tc_fold_nowrap(F), "the combined pattern must not wrap");
                    hi[kk] += (unsigned long long)((a0 << F.g) + b0) << F.sh;
                    hi[kk + 1] += (unsigned long long)((a1 << F.g) + b1) << F.sh;
                }
            }
        }
    }
}
template <int H>
__device__ __forceinline__ void tc_fold_all(uint32_t trow, unsigned long long (&hi)[16], uint32_t (&lo)[16],
                                            uint32_t (&res)[8]) {
    tc_fold_block<H, 0>(trow, hi, lo, res);
    tc_fold_block<H, 1>(trow, hi, lo, res);
    tc_fold_block<H, 2>(trow, hi, lo, res);
    tc_fold_block<H, 3>(trow, hi, lo, res);
    tc_fold_block<H, 4>(trow, hi, lo, res);
    tc_fold_block<H, 5>(trow, hi, lo, res);
    tc_fold_block<H, 6>(trow, hi, lo, res);
    tc_fold_block<H, 7>(trow, hi, lo, res);
    constexpr unsigned long long OH = tc_hi_offset(H);
    constexpr uint32_t OL = tc_lo_offset(H);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        hi[k] -= OH;
        lo[k] -= OL;
    }
}

// Drain one finished period from TMEM into the calling warp's fixed-point
// accumulators, after moving them onto the period's (coarser or equal) grid: dsh
// holds E_old - E_acc per column.  Each warp works alone: its lane quadrant
// `quad` is fixed by the warp (a warp may only read its own 32 TMEM lanes),
// columns J0..J0+15.
__device__ __forceinline__ void tc_drain(const TcRecord& R, uint32_t tmem, int quad, int lane, int J0,
                                         unsigned long long (&hi)[16], uint32_t (&lo)[16], uint32_t (&res)[8]) {
    if (R.regrid[0] | R.regrid[1]) {
        // truncating shift onto the grid of the grown scales (the residuals are first rounded
        // into lo: a re-grid truncates anyway)
        const int di = R.dsh[(quad * 32 + lane) & 63];
#pragma unroll
        for (int k = 0; k < 16; ++k) lo[k] += (uint32_t)((tc_res_get(res, k) + 256) >> 9);
#pragma unroll
        for (int k = 0; k < 8; ++k) res[k] = 0u;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int sh = di + R.dsh[J0 + k];
            if (sh > 0) {
                hi[k] = sh >= 63 ? 0ull : (unsigned long long)((long long)hi[k] >> sh);
                lo[k] = sh >= 31 ? 0u : (uint32_t)((int)lo[k] >> sh);
            }
        }
    }
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + J0;
    if (quad < 2) tc_fold_all<0>(trow, hi, lo, res);   // TMEM lanes 0..63: first digit of A
    else tc_fold_all<1>(trow, hi, lo, res);            // lanes 64..127: second digit
}

// The workers publish the column maxima of sub-chunk h for the deciders: lane l takes rows
// 4 (l % 8) .. + 3 and 32 + 4 (l % 8) .. + 3 of column 4 w + l / 8 (the digits' layout: 8 lanes
// read 128 contiguous bytes per 16-byte load, no bank conflict), the column's 8 lanes combine
// theirs by shuffles.  max |a| is taken on the bit patterns (Inf and NaN order above every
// finite value).  False if the stage did not land (it is then not read).
__device__ __forceinline__ bool tc_publish_max(TcShared& S, const float* fpb, int h, int n, int wq, int lane,
                                               long long wait_limit) {
    const int f = h % TC_SF;
    bool ok = mbar_wait_susp(&S.fp_full[f], (h / TC_SF) & 1, wait_limit) && !S.abort;
    if (!__all_sync(0xffffffffu, ok)) return false;
    const int jj = 4 * wq + (lane >> 3), rb = lane & 7;
    unsigned mx = 0u;
    if (jj < n) {
        const float4* src =
            reinterpret_cast<const float4*>(fpb + (size_t)f * 64 * TC_SUB + (size_t)jj * TC_SUB + 4 * rb);
        const float4 a = src[0], b = src[8];
        mx = max(max(max(__float_as_uint(a.x) & 0x7fffffffu, __float_as_uint(a.y) & 0x7fffffffu),
                     max(__float_as_uint(a.z) & 0x7fffffffu, __float_as_uint(a.w) & 0x7fffffffu)),
                 max(max(__float_as_uint(b.x) & 0x7fffffffu, __float_as_uint(b.y) & 0x7fffffffu),
                     max(__float_as_uint(b.z) & 0x7fffffffu, __float_as_uint(b.w) & 0x7fffffffu)));
    }
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
    if (rb == 0) S.colmax[h % TC_MX][jj] = mx;
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.max_full[h % TC_MX]);
    return true;
}

// partial slot and status block of this CTA (batched use: those of its item)
template <bool BATCH>
__device__ __forceinline__ int64_t tc_slot(const TcBatchItem* items) {
    return BATCH ? (int64_t)items[blockIdx.x].slot : (int64_t)blockIdx.x;
}
template <bool BATCH>
__device__ __forceinline__ DevInfo* tc_info(DevInfo* info, const TcBatchItem* items) {
    return BATCH ? info + items[blockIdx.x].inst : info;
}

template <bool BATCH>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapB, int64_t m,
                   int n, int split, int64_t rows_per_cta,
                   long long* __restrict__ part_hi, long long* __restrict__ part_lo, int* __restrict__ part_E,
                   DevInfo* info, const TcBatchItem* __restrict__ items, long long wait_limit,
                   const int* __restrict__ E_fixed) {
    extern __shared__ unsigned char tc_dyn[];
    // 1024-byte alignment for the swizzled operand atoms
    unsigned char* base = tc_dyn + ((1024 - (smem_addr(tc_dyn) & 1023)) & 1023);
    unsigned char* dig = base;                                           // [SD][7*64 rows][128 B]
    float* fpb = reinterpret_cast<float*>(base + TC_SD * TC_DIG_BYTES);  // [SF][64][64]
    __shared__ TcShared S;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // sub-chunks are dealt round-robin (CTA b takes b, b + P, b + 2P, ...): at any time the
    // CTAs stream neighbouring 256-byte pieces of every column.  A CTA takes at most
    // rows_per_cta rows (the fixed-point bounds need <= 2^15).
    // Batched use (items != null): CTA b streams the rows [r0, r1) of one instance alone
    // (a multiple of 64 rows apart from the instance's last row), through that instance's
    // tensor map in global memory, into partial slot items[b].slot.
    // (The slot and the status block are re-read where they are used, so that they hold no
    // registers through the main loop.)
    // An item with a second map (n <= 32) packs two consecutive 64-row blocks side by side as
    // the two 32-column groups: sub-chunk g covers rows r0 + 128 g .. + 127, and the instance's
    // Gram is the sum of the two diagonal 32 x 32 tiles.
    const CUtensorMap* mapA = &tmapA;
    const CUtensorMap* mapB = &tmapB;
    int64_t first = blockIdx.x, P = gridDim.x;
    int G;
    if (BATCH) {
        const TcBatchItem it = items[blockIdx.x];
        mapA = static_cast<const CUtensorMap*>(it.tmap);
        first = it.r0 / TC_SUB;
        if (it.tmap2 != nullptr) {
            mapB = static_cast<const CUtensorMap*>(it.tmap2);
            n = 64;
            split = 1;
            P = 2;
            G = (int)((it.r1 - it.r0 + 2 * TC_SUB - 1) / (2 * TC_SUB));
        } else {
            n = it.n;
            split = 0;
            P = 1;
            G = (int)((it.r1 - it.r0 + TC_SUB - 1) / TC_SUB);
        }
    } else {
        const int64_t subs = (m + TC_SUB - 1) / TC_SUB;
        G = (int64_t)blockIdx.x < subs ? (int)((subs - 1 - blockIdx.x) / P + 1) : 0;
    }
    (void)rows_per_cta;

    if (tid == 0) {
        // an FP32 stage is free once the MMA issuer has seen every worker's digits of that
        // sub-chunk (the workers read it for its maxima and its digits only)
        for (int s = 0; s < TC_SF; ++s) { mbar_init(&S.fp_full[s], 1); mbar_init(&S.fp_empty[s], 1); }
        for (int s = 0; s < TC_MX; ++s) mbar_init(&S.max_full[s], 16);
        for (int s = 0; s < TC_SD; ++s) { mbar_init(&S.dig_full[s], 16); mbar_init(&S.dig_empty[s], 1); }
        for (int s = 0; s < TC_RD; ++s) { mbar_init(&S.dec_full[s], 2); mbar_init(&S.dec_empty[s], 16); }
        mbar_init(&S.acc_full, 1);
        mbar_init(&S.acc_empty, 16);
        mbar_fence_init();
        S.abort = 0;
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
        asm volatile("setmaxnreg.dec.sync.aligned.u32 32;");
        if (warp == 0 && lane == 0) {
            // ---------------- TMA producer
            tma_prefetch_desc(mapA);
            if (split) tma_prefetch_desc(mapB);
            // split: two 32-column groups (FP columns 0..31 and 32..63) from two maps
            const unsigned bytes = (unsigned)(TC_SUB * (split ? 64 : n) * 4);
            int issued = 0;
            for (int g = 0; g < G; ++g) {
                const int f = g % TC_SF;
                if (g >= TC_SF && !mbar_wait_susp(&S.fp_empty[f], ((g / TC_SF) - 1) & 1, wait_limit)) {
                    atomicExch(&S.abort, 1);
                    break;
                }
                if (S.abort) break;
                mbar_expect_tx(&S.fp_full[f], bytes);
                const int row0 = (int)((first + (int64_t)g * P) * TC_SUB);
                tma_load_2d(fpb + (size_t)f * 64 * TC_SUB, mapA, row0, 0, &S.fp_full[f]);
                if (split) tma_load_2d(fpb + (size_t)f * 64 * TC_SUB + 32 * TC_SUB, mapB, row0, 0, &S.fp_full[f]);
                issued = g + 1;
            }
            tma_issued = issued;
        } else if (warp == 1 && lane == 0) {
            // ---------------- MMA issuer
            const uint32_t id256 = idesc_bf16(128, 256), id64 = idesc_bf16(128, 64);
            int period = 0;
            for (int g = 0; g < G; ++g) {
                const int d = g % TC_SD;
                if (!mbar_wait_susp(&S.dig_full[d], (g / TC_SD) & 1, wait_limit) || S.abort) {
                    atomicExch(&S.abort, 1);
                    break;
                }
                mbar_arrive(&S.fp_empty[g % TC_SF]);  // every worker has read this FP32 stage
                const int newp = S.dig_newp[d];
                if (newp && g > 0) {
                    // close the running period: the workers drain it before it is overwritten
                    mma_commit(&S.acc_full);
                    if (!mbar_wait_susp(&S.acc_empty, period & 1, wait_limit)) { atomicExch(&S.abort, 1); break; }
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
            (void)mbar_wait_susp(&S.acc_full, period & 1);
        } else if (warp >= 2) {
            // ---------------- deciders (warps 2, 3; lane l owns column j = 32 (warp - 2) + l).
            // For each sub-chunk, from the column maxima the workers publish: growth class; the
            // two warps agree on whether a new period starts (an entry needs more than one binade
            // above the running scale, or the exactness budget is spent) and publish a record.
            const int dw = warp - 2, j = 32 * dw + lane;
            int Ecur = EXP_EMPTY, Epend = EXP_EMPTY, Eacc = EXP_EMPTY, period_len = 0;
            bool bad = false, over = false;
            // fixed scales (E_fixed): every sub-chunk's digits are relative to the given column
            // exponent, so nothing grows and no period is re-gridded; an entry at or above 2^E
            // is an argument error (the exponents must bound the whole column)
            const int Efix = (E_fixed != nullptr && j < n) ? E_fixed[j] : EXP_EMPTY;
            for (int g = 0; g <= G; ++g) {
                const int r = g % TC_RD;
                int fl = 0;
                if (g < G) {
                    // the column maxima of sub-chunk g, found by the workers (8 lanes per column)
                    const bool got = mbar_wait_susp(&S.max_full[g % TC_MX], (g / TC_MX) & 1, wait_limit);
                    if (!got) fl |= 4;
                    const unsigned mine = got ? S.colmax[g % TC_MX][j] : 0u;
                    if (mine >= 0x7f800000u) bad = true;
                    const int e = (mine == 0u || mine >= 0x7f800000u) ? EXP_EMPTY : tc_exp_above(__uint_as_float(mine));
                    // one binade above the running scale is "soft" (top digit in [-256, 256], still
                    // exact in bf16); more, or a first non-zero entry, is "hard"
                    if (E_fixed != nullptr) {
                        if (e != EXP_EMPTY && e > Efix) over = true;
                        Epend = Efix;
                    } else {
                        if (e != EXP_EMPTY) {
                            if (Ecur == EXP_EMPTY || e > Ecur + 1) fl |= 2;
                            else if (e == Ecur + 1) fl |= 1;
                        }
                        Epend = max(Epend, e);
                    }
                }
                if (g >= TC_RD && !mbar_wait_susp(&S.dec_empty[r], ((g / TC_RD) - 1) & 1, wait_limit)) fl |= 4;
                if (S.abort) fl |= 4;
                fl = __reduce_or_sync(0xffffffffu, fl);
                if (lane == 0) S.dflags[g & 1][dw] = fl;
                named_bar(BAR_DEC, 64);
                const int F = S.dflags[g & 1][0] | S.dflags[g & 1][1];
                if (F & 4) {
                    atomicExch(&S.abort, 1);
                    break;
                }
                // exactness budget of a period: sum |q_s q_t| <= 2^24 grid units per block and
                // (i, j); a normal sub-chunk adds at most 64 * 128^2 = 2^20 (1 unit), one with a
                // soft growth 64 * 256^2 = 2^22 (4 units).  g == G closes the last period.
                const int cost = (F & 1) ? 4 : 1;
                const bool newp = g == 0 || g == G || (F & 2) || period_len + cost > TC_PERIOD;
                int dsh = 0;
                if (newp) {
                    if (g > 0) {
                        // re-grid of the accumulators.  A column whose grid is still EXP_EMPTY has
                        // accumulated only zeros (its scale never shrinks): nothing to move, and no
                        // re-grid is flagged for it (a flagged re-grid rounds the residuals away)
                        dsh = Eacc == EXP_EMPTY ? 0 : Ecur - Eacc;
                        Eacc = Ecur;
                    }
                    Ecur = Epend;  // the new period starts on every grown scale
                    period_len = 1;
                } else {
                    period_len += cost;
                }
                TcRecord& R = S.rec[r];
                R.E[j] = Ecur;
                R.dsh[j] = dsh;
                const bool rg = __any_sync(0xffffffffu, dsh != 0);
                if (lane == 0) R.regrid[dw] = rg ? 1 : 0;
                if (j == 0) R.newp = newp ? 1 : 0;
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.dec_full[r]);
            }
            if (bad) atomicOr(&tc_info<BATCH>(info, items)->flags, FLAG_NONFINITE);
            if (over) atomicOr(&tc_info<BATCH>(info, items)->flags, FLAG_BAD_SCALE);
            part_E[(size_t)tc_slot<BATCH>(items) * 64 + j] = Eacc;
        }
    } else {
        // ---------------- 16 worker warps.  Per sub-chunk: take the record, write the 7 digit
        // slices of columns 4w .. 4w+3 (lane l: 8 rows of one column), hand the stage to
        // the MMA; when a period closes, drain TMEM lanes 32 (w % 4).. x columns 16 (w / 4)...
        // Warps only meet on mbarriers: no CTA-wide barrier until the partials are written.
        asm volatile("setmaxnreg.inc.sync.aligned.u32 112;");
        const int wq = warp - 4;                   // worker warp 0..15
        const int quad = warp & 3;                 // TMEM lane quadrant of this warp
        const int J0 = 16 * (wq >> 2);             // drain columns J0..J0+15
        unsigned long long hi[16];
        uint32_t lo[16];
        uint32_t res[8];
#pragma unroll
        for (int k = 0; k < 16; ++k) { hi[k] = 0; lo[k] = 0; }
#pragma unroll
        for (int k = 0; k < 8; ++k) res[k] = 0u;
        int drained = 0, res_periods = 0;
        bool failed = false;
        // the maxima of sub-chunk g + 2 are published right after the digits of sub-chunk g, so
        // the deciders have a whole sub-chunk's time for each record
        for (int h = 0; h < 2 && h < G && !failed; ++h) {
            if (!tc_publish_max(S, fpb, h, n, wq, lane, wait_limit)) {
                failed = true;
                if (lane == 0) atomicExch(&S.abort, 1);
            }
        }
        for (int g = 0; g <= G && !failed; ++g) {
            const int r = g % TC_RD;
            bool ok = mbar_wait_susp(&S.dec_full[r], (g / TC_RD) & 1, wait_limit) && !S.abort;
            if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
            const TcRecord& R = S.rec[r];
            const int newp = R.newp;
            if (g < G) {
                const int d = g % TC_SD, f = g % TC_SF;
                // the FP32 stage has landed: the deciders waited for it before publishing the record
                // (their release on dec_full orders it before this warp's acquire)
                ok = g < TC_SD || mbar_wait_susp(&S.dig_empty[d], ((g / TC_SD) - 1) & 1, wait_limit);
                if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
                // digits of sub-chunk g: y = 128 a 2^-E (|y| < 128, < 256 after a soft growth);
                // digit s is y's remainder rounded to the grid 2^-8s (|digit| <= 128 grid units,
                // exact in bf16: 8 significant bits); the MMA sees digit s scaled by 2^-8s.
                // Lane l takes rows 4 (l % 8) .. + 3 and 32 + 4 (l % 8) .. + 3 of column
                // j = 4 w + l / 8 and writes them as K positions 8 (l % 8) .. + 7: one 16-byte chunk
                // of a digit slice per digit (a quarter-warp writes one slice row, 128 bytes).  Every
                // slice holds the rows in the same order, so each block's sum over K is unchanged.
                const int jj = 4 * wq + (lane >> 3), rb = lane & 7;
                const int E = R.E[jj];
                unsigned long long y[4] = {0ull, 0ull, 0ull, 0ull};
                if (E != EXP_EMPTY) {
                    const float4* src =
                        reinterpret_cast<const float4*>(fpb + (size_t)f * 64 * TC_SUB + (size_t)jj * TC_SUB + 4 * rb);
                    const float4 a = src[0], b = src[8];
                    const int k = 7 - E, k1 = k / 2, k2 = k - k1;
                    const float s1 = __int_as_float((k1 + 127) << 23), s2 = __int_as_float((k2 + 127) << 23);
                    const unsigned long long S1 = f2_pack(s1, s1), S2 = f2_pack(s2, s2);
                    y[0] = f2_mul(f2_mul(f2_pack(a.x, a.y), S1), S2);
                    y[1] = f2_mul(f2_mul(f2_pack(a.z, a.w), S1), S2);
                    y[2] = f2_mul(f2_mul(f2_pack(b.x, b.y), S1), S2);
                    y[3] = f2_mul(f2_mul(f2_pack(b.z, b.w), S1), S2);
                }
                unsigned char* drow = dig + (size_t)d * TC_DIG_BYTES + jj * 128 + ((rb ^ (jj & 7)) << 4);
#pragma unroll
                for (int sdig = 0; sdig < 7; ++sdig) {
                    // when no row of the warp has a remainder left after five digits, the last two
                    // are +0 (what the split would give): store them without the arithmetic.  Only
                    // an entry about 2^16 or more below its column's largest (|y| < 2^-9) has bits
                    // below 2^-32 left, so most warps skip.
                    if (sdig == 5 &&
                        !__any_sync(0xffffffffu, ((y[0] | y[1] | y[2] | y[3]) & 0x7fffffff7fffffffull) != 0ull)) {
#pragma unroll
                        for (int z = sdig; z < 7; ++z)
                            *reinterpret_cast<uint4*>(drow + tc_pos_of_digit(z) * 8192) = make_uint4(0u, 0u, 0u, 0u);
                        break;
                    }
                    const unsigned long long M2 = tc_magic2(23 - 8 * sdig);
                    uint32_t bq[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const unsigned long long qd = f2_sub(f2_add(y[c], M2), M2);
                        if (sdig < 6) y[c] = f2_sub(y[c], qd);
                        float a0, a1;
                        f2_unpack(qd, a0, a1);
                        // the digit has at most 8 significant bits: its bf16 is the top half
                        bq[c] = __byte_perm(__float_as_uint(a0), __float_as_uint(a1), 0x7632);
                    }
                    // slice position of digit s: 64 rows (columns j) of 128 bytes, 16-byte chunks
                    // swizzled by row
                    *reinterpret_cast<uint4*>(drow + tc_pos_of_digit(sdig) * 8192) =
                        make_uint4(bq[0], bq[1], bq[2], bq[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    S.dig_newp[d] = newp;  // every warp writes the same value
                    mbar_arrive(&S.dig_full[d]);
                }
                if (g + 2 < G && !tc_publish_max(S, fpb, g + 2, n, wq, lane, wait_limit)) {
                    failed = true;
                    if (lane == 0) atomicExch(&S.abort, 1);
                    break;
                }
            }
            if (((newp && g > 0) || g == G) && G > 0) {
                // the MMA issuer closes a period on seeing the first stage of the next one
                // (or after the last sub-chunk); drain it
                ok = mbar_wait_susp(&S.acc_full, drained & 1, wait_limit);
                if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
                tc_fence_after();
                if (res_periods == 32) {
                    // the 16-bit residual sums hold 32 periods; more (scale growths shorten
                    // periods) are first rounded into lo.  A CTA of fixed scales (at most 2^15
                    // rows, 1024-row periods) never gets here.
#pragma unroll
                    for (int k = 0; k < 16; ++k) lo[k] += (uint32_t)((tc_res_get(res, k) + 256) >> 9);
#pragma unroll
                    for (int k = 0; k < 8; ++k) res[k] = 0u;
                    res_periods = 0;
                }
                tc_drain(R, tmem, quad, lane, J0, hi, lo, res);
                ++res_periods;
                tc_fence_before();
                __syncwarp();
                if (lane == 0 && g < G) mbar_arrive(&S.acc_empty);
                ++drained;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.dec_empty[r]);
        }
        if (failed && lane == 0) atomicExch(&S.abort, 1);
        // partials of this CTA: W = sum over blocks (s < t) + 1/2 (s = s); G = W + W^T later.
        // The two digit halves of row i add into the same W(i, j): half 0 first, then half 1.
        const int lanei = quad * 32 + lane, h = lanei >> 6, i = lanei & 63;
        long long* ph = part_hi + (size_t)tc_slot<BATCH>(items) * 64 * 64;
        long long* pl = part_lo + (size_t)tc_slot<BATCH>(items) * 64 * 64;
        for (int hh = 0; hh < 2; ++hh) {
            if (h == hh) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const long long l63 =
                        (long long)((unsigned long long)(long long)(int)lo[k] << 9) + (long long)tc_res_get(res, k);
                    if (hh == 0) { ph[i * 64 + J0 + k] = (long long)hi[k]; pl[i * 64 + J0 + k] = l63; }
                    else { ph[i * 64 + J0 + k] += (long long)hi[k]; pl[i * 64 + J0 + k] += l63; }
                }
            }
            __threadfence_block();
            named_bar(BAR_WORK, TC_WORKERS);
        }
    }
    // teardown: every tcgen05 access is complete before the TMEM is freed
    tc_fence_before();
    __syncthreads();
    if (S.abort && tid == 0) {
        atomicOr(&tc_info<BATCH>(info, items)->flags, FLAG_TIMEOUT);
        // no TMA write may land after the CTA exits: wait (bounded) for the last loads
        for (int g = (tma_issued > TC_SF ? tma_issued - TC_SF : 0); g < tma_issued; ++g)
            (void)mbar_wait_susp(&S.fp_full[g % TC_SF], (g / TC_SF) & 1);
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

}  // namespace

bool gram_tc_ok(const void* A, int working, int n, int64_t lda) {
    return working == 0 && n >= 1 && n <= 256 && ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
}

GramPlan gram_tc_plan(int64_t m, int n, int sm_count, int split_k_opt) {
    GramPlan p;
    p.NP = 64;
    const int64_t subs = (m + TC_SUB - 1) / TC_SUB;
    int64_t P = split_k_opt > 0 ? split_k_opt : sm_count;
    const int64_t min_P = (m + GRAM_MAX_ROWS_PER_CTA - 1) / GRAM_MAX_ROWS_PER_CTA;
    // more CTAs than SMs (one CTA per SM at a time): whole waves of equal row counts
    if (P < min_P) P = split_k_opt > 0 ? min_P : (min_P + sm_count - 1) / sm_count * sm_count;
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
    return launch_gram_tc2(A, m, n, lda, -1, -1, plan, part, info, s);
}

// c1 < 0: columns 0..n-1 (n <= 64).  Otherwise the virtual 64 columns are the
// 32-column groups starting at c1 and c2 of A (columns >= n read as zero).
cudaError_t launch_gram_tc2(const void* A, int64_t m, int n, int64_t lda, int c1, int c2, const GramPlan& plan,
                            void* part, DevInfo* info, cudaStream_t s) {
    CUtensorMap tmapA, tmapB;
    const bool split = c1 >= 0;
    const float* Af = static_cast<const float*>(A);
    cudaError_t e;
    if (!split) {
        e = make_tmap_2d(&tmapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), A, (uint64_t)m, (uint64_t)n,
                         (uint64_t)lda, TC_SUB, (uint32_t)n, CU_TENSOR_MAP_SWIZZLE_NONE);
        tmapB = tmapA;
    } else {
        e = make_tmap_2d(&tmapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), Af + (size_t)c1 * lda, (uint64_t)m,
                         (uint64_t)(n - c1), (uint64_t)lda, TC_SUB, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
        if (e == cudaSuccess)
            e = make_tmap_2d(&tmapB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), Af + (size_t)c2 * lda,
                             (uint64_t)m, (uint64_t)(n - c2), (uint64_t)lda, TC_SUB, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
    }
    if (e != cudaSuccess) return e;
    long long* ph = reinterpret_cast<long long*>(part);
    long long* pl = ph + (size_t)plan.P * 64 * 64;
    int* pE = reinterpret_cast<int*>(pl + (size_t)plan.P * 64 * 64);
    e = cudaFuncSetAttribute(gram_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    gram_tc_kernel<false><<<plan.P, TC_THREADS, TC_SMEM, s>>>(tmapA, tmapB, m, split ? 64 : n, split ? 1 : 0,
                                                              plan.rows_per_cta, ph, pl, pE, info, nullptr,
                                                              wait_limit_of(plan.wait_cycles), plan.E_fixed);
    return cudaGetLastError();
}

bool gram_tc_batch_ok(const void* A, int64_t lda) { return ((uintptr_t)A % 16 == 0) && (lda % 4 == 0); }

size_t tc_tmap_bytes() { return sizeof(CUtensorMap); }

cudaError_t make_tc_batch_tmap(void* map, const float* A, int64_t m, int n, int64_t lda, int box_cols) {
    return make_tmap_2d(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), A,
                        (uint64_t)m, (uint64_t)n, (uint64_t)lda, TC_SUB, (uint32_t)box_cols,
                        CU_TENSOR_MAP_SWIZZLE_NONE);
}

cudaError_t launch_gram_tc_batch(const TcBatchItem* items, int nitems, void* part, int total_slots, DevInfo* infos,
                                 cudaStream_t s, long long wait_cycles) {
    if (nitems == 0) return cudaSuccess;
    long long* ph = reinterpret_cast<long long*>(part);
    long long* pl = ph + (size_t)total_slots * 64 * 64;
    int* pE = reinterpret_cast<int*>(pl + (size_t)total_slots * 64 * 64);
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    CUtensorMap unused;
    std::memset(&unused, 0, sizeof(unused));
    gram_tc_kernel<true><<<nitems, TC_THREADS, TC_SMEM, s>>>(unused, unused, 0, 64, 0, 0, ph, pl, pE, infos, items,
                                                             wait_limit_of(wait_cycles), nullptr);
    return cudaGetLastError();
}

}  // namespace tsvd
