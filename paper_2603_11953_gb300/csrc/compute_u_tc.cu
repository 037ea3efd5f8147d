// compute_u_tc.cu -- U = A W on the 5th-generation tensor cores (Alg. 1 line 6,
// eq. (AV-0)), FP32 working precision, n <= 64.
//
// A dense m x n by n x n product in FP32 costs 2 n^2 FP32 flops per row: at
// n = 64 the FP32 FMA units, not HBM, bound a CUDA-core kernel.  Here the
// contraction runs on tcgen05 in TF32 with a three-term split that keeps FP32
// accuracy: x = x_hi + x_lo with x_hi = RN_tf32(x) and x_lo = RN_tf32(x - x_hi)
// (x - x_hi is exact in FP32, |x_lo| <= 2^-11 |x|), and
//     A W ~ A_hi W_hi + A_hi W_lo + A_lo W_hi,
// accumulated in FP32 in TMEM.  Per product the representation error is at
// most 2^-22 |a| |w| from each rounded low part and from the dropped
// A_lo W_lo, i.e. 3 * 2^-22 = 12 u_32 |a||w| in all, on top of the FP32
// accumulation: |U - AW| <= (n + 12) u_32 (|A||W|) + O(u^2), the same order as
// the FP32 dot products the paper's error model assumes.  (Rounding ties away
// from zero instead of to even changes none of these bounds.)
//
// One persistent CTA per SM (384 threads), 128-row tiles of A dealt
// round-robin over the CTAs:
//   warp 0      TMA producer: one 2-D load (128 rows x n FP32) per tile into a
//               4-stage ring (the operand stage is single: the MMAs of a tile
//               take a fraction of the time its bytes take to stream).
//   warp 1      TMEM owner (128 columns: two 64-column accumulators) and MMA
//               issuer: 3 x 8 tcgen05.mma.kind::tf32 (M = 128, N = 64, K = 8)
//               per tile.
//   warps 4-11  convert each tile into the K-major, 128-byte-swizzled hi and
//               lo operands (thread t: row t % 128, columns 32 (t / 128)..+31),
//               and write the previous tile's U from TMEM (lane = row, 32
//               columns per thread): into a shared output tile that warp 2
//               sends to U with one TMA store (a 16-byte-aligned U), else
//               straight to U (each warp store covers 32 consecutive rows of
//               one column, 128 bytes).
// With the TMA store the ring has 3 A stages, the fourth 32 KB going to the
// output tile: loads and stores both stay in flight, as in a TMA copy.
// W^T (the B operand, rows = columns of U) is split once per CTA.  Every
// mbarrier wait is bounded; on timeout the kernel records TSVD_ERR_TIMEOUT,
// waits for its own TMA loads and frees its TMEM.
#include "internal.cuh"
#include "tma_util.cuh"

namespace tsvd {
namespace {

constexpr int UT_ROWS = 128;
constexpr int UT_THREADS = 384;
constexpr int UT_FP_BYTES = 64 * UT_ROWS * 4;      // one A tile: [64 cols][128 rows] FP32
constexpr int UT_OP_BYTES = 2 * UT_ROWS * 128;     // one K-major tf32 operand: [2 atoms][128 rows][128 B]
constexpr int UT_W_BYTES = 2 * 64 * 128;           // W^T operand: [2 atoms][64 rows][128 B]
constexpr int UT_SO = 1;
// A stages: 4 (~96 KB of loads outstanding per SM) with plain stores, 3 beside the output tile
template <bool TS> __host__ __device__ constexpr int ut_sf() { return TS ? 3 : 4; }
template <bool TS> __host__ __device__ constexpr int ut_smem() {
    return ut_sf<TS>() * UT_FP_BYTES + UT_SO * 2 * UT_OP_BYTES + 2 * UT_W_BYTES + (TS ? UT_FP_BYTES : 0) + 1024;
}

struct UtShared {
    uint64_t fp_full[4], fp_empty[4];
    uint64_t op_full[UT_SO], op_empty[UT_SO];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t out_full, out_free;  // output tile written by the 8 epilogue warps / read by its TMA store
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint64_t ut_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused: swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8-row groups 1024 B apart
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}
// kind::tf32, D = F32, A = B = TF32, K-major both, M = 128, N = 64
constexpr uint32_t UT_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);
__device__ __forceinline__ void ut_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(UT_IDESC), "r"(acc));
}
__device__ __forceinline__ void ut_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void ut_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void ut_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void ut_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Round to TF32 (10 explicit significand bits, to nearest, ties away from zero):
// half a TF32 ulp (2^12 in the bit pattern) is added to the magnitude bits and
// the 13 low bits are cleared, the rounding cvt.rna.tf32.f32 does, in two
// integer operations (the conversion instruction made the kernel issue-bound).
// A carry into the exponent is the correct round-up; the MMA ignores the low
// 13 bits, so a rounded value is used exactly.
__device__ __forceinline__ float ut_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}
// byte offset of element (row, k) in a [2 atoms][rows][128 B] K-major SW128 operand
__device__ __forceinline__ uint32_t ut_off(int row, int k, int rows) {
    return (uint32_t)((k >> 5) * rows * 128 + row * 128 + ((((k & 31) >> 2) ^ (row & 7)) << 4) + ((k & 3) << 2));
}

// TMA store of the output tile (box = 128 rows x n columns) to rows x0.. of U
__device__ __forceinline__ void ut_tma_store(const CUtensorMap* map, const void* src, int x0) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x0), "r"(0), "r"(smem_addr(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

template <bool TS>
__global__ void __launch_bounds__(UT_THREADS, 1)
    compute_u_tc_kernel(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapU, int64_t m,
                        int n, const float* __restrict__ W, float* __restrict__ U, int64_t ldu, DevInfo* info) {
    constexpr int SF = ut_sf<TS>();
    extern __shared__ unsigned char ut_dyn[];
    unsigned char* base = ut_dyn + ((1024 - (smem_addr(ut_dyn) & 1023)) & 1023);
    unsigned char* ops = base;                                        // [SO][hi, lo][UT_OP_BYTES]
    unsigned char* wop = base + UT_SO * 2 * UT_OP_BYTES;              // [hi, lo][UT_W_BYTES]
    float* fpb = reinterpret_cast<float*>(wop + 2 * UT_W_BYTES);      // [SF][64][128]
    float* outb = fpb + (size_t)SF * 64 * UT_ROWS;                    // TS: [n][128] output tile
    __shared__ UtShared S;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tiles = (m + UT_ROWS - 1) / UT_ROWS;
    const int64_t P = gridDim.x;
    const int T = (int64_t)blockIdx.x < tiles ? (int)((tiles - 1 - blockIdx.x) / P + 1) : 0;

    if (tid == 0) {
        for (int s = 0; s < SF; ++s) { mbar_init(&S.fp_full[s], 1); mbar_init(&S.fp_empty[s], 8); }
        for (int s = 0; s < UT_SO; ++s) { mbar_init(&S.op_full[s], 8); mbar_init(&S.op_empty[s], 1); }
        for (int s = 0; s < 2; ++s) { mbar_init(&S.acc_full[s], 1); mbar_init(&S.acc_empty[s], 8); }
        mbar_init(&S.out_full, 8);
        mbar_init(&S.out_free, 1);
        mbar_fence_init();
        S.abort = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
            smem_addr(&S.tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // W^T split into hi / lo (rows j = columns of U, K = rows of W); zero padding past n
    for (int idx = tid; idx < 64 * 64; idx += UT_THREADS) {
        const int j = idx >> 6, k = idx & 63;
        const float w = (j < n && k < n) ? W[k + (size_t)j * n] : 0.0f;
        const float wh = ut_tf32(w), wl = ut_tf32(w - wh);
        *reinterpret_cast<float*>(wop + ut_off(j, k, 64)) = wh;
        *reinterpret_cast<float*>(wop + UT_W_BYTES + ut_off(j, k, 64)) = wl;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ut_fence_before();
    __syncthreads();
    ut_fence_after();
    const uint32_t tmem = S.tmem_base;
    int tma_issued = 0;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            tma_prefetch_desc(&tmapA);
            const unsigned bytes = (unsigned)(UT_ROWS * n * 4);
            for (int j = 0; j < T; ++j) {
                const int f = j % SF;
                if (j >= SF && !mbar_wait(&S.fp_empty[f], ((j / SF) - 1) & 1)) { atomicExch(&S.abort, 1); break; }
                if (S.abort) break;
                mbar_expect_tx(&S.fp_full[f], bytes);
                tma_load_2d(fpb + (size_t)f * 64 * UT_ROWS, &tmapA, (int)(((int64_t)blockIdx.x + (int64_t)j * P) * UT_ROWS),
                            0, &S.fp_full[f]);
                tma_issued = j + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            const uint32_t wh = smem_addr(wop), wl = smem_addr(wop + UT_W_BYTES);
            for (int j = 0; j < T; ++j) {
                const int o = j % UT_SO, b = j & 1;
                if (!mbar_wait(&S.op_full[o], (j / UT_SO) & 1) || S.abort) { atomicExch(&S.abort, 1); break; }
                if (j >= 2 && !mbar_wait(&S.acc_empty[b], ((j / 2) - 1) & 1)) { atomicExch(&S.abort, 1); break; }
                ut_fence_after();
                const uint32_t ah = smem_addr(ops + (size_t)o * 2 * UT_OP_BYTES), al = ah + UT_OP_BYTES;
                const uint32_t d = tmem + (uint32_t)(b * 64);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const uint32_t oa = (uint32_t)((kk >> 2) * UT_ROWS * 128 + (kk & 3) * 32);
                    const uint32_t ob = (uint32_t)((kk >> 2) * 64 * 128 + (kk & 3) * 32);
                    ut_mma(d, ut_desc(ah + oa), ut_desc(wh + ob), kk > 0 ? 1u : 0u);
                    ut_mma(d, ut_desc(ah + oa), ut_desc(wl + ob), 1u);
                    ut_mma(d, ut_desc(al + oa), ut_desc(wh + ob), 1u);
                }
                ut_commit(&S.op_empty[o]);
                ut_commit(&S.acc_full[b]);
            }
        }
    } else if (warp == 2) {
        if (TS && lane == 0) {
            // ---------------- output tile -> U (TMA store), then hand the tile back
            tma_prefetch_desc(&tmapU);
            for (int j = 0; j < T; ++j) {
                if (!mbar_wait(&S.out_full, j & 1) || S.abort) { atomicExch(&S.abort, 1); break; }
                ut_tma_store(&tmapU, outb, (int)(((int64_t)blockIdx.x + (int64_t)j * P) * UT_ROWS));
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                mbar_arrive(&S.out_free);
            }
            // the stores have left shared memory; wait for their writes too before the CTA exits
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
    } else if (warp >= 4) {
        // ---------------- converters and epilogue
        const int t = tid - 128;
        const int row = t & 127, kbase = 32 * (t >> 7);
        const int q = warp & 3, colh = (warp - 4) >> 2;  // TMEM lane quadrant, column half
        const int rowoff = (kbase >> 5) * UT_ROWS * 128 + row * 128;
        bool ok = true;
        auto epilogue = [&](int jj) {
            const int b = jj & 1;
            if (!mbar_wait(&S.acc_full[b], (jj / 2) & 1)) ok = false;
            // TS: the previous tile's store has read the output tile
            if (TS && jj >= 1 && !mbar_wait(&S.out_free, (jj - 1) & 1)) ok = false;
            ut_fence_after();
            const int64_t r0 = ((int64_t)blockIdx.x + (int64_t)jj * P) * UT_ROWS + 32 * q + lane;
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 64 + 32 * colh);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t r[16];
                ut_ld16(ta + 16 * hh, r);
                if (TS) {
                    // [column][128 rows]: a warp writes 32 consecutive rows of one column
                    float* oc = outb + (size_t)(32 * colh + 16 * hh) * UT_ROWS + 32 * q + lane;
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (n == 64 || 32 * colh + 16 * hh + c < n) oc[c * UT_ROWS] = __uint_as_float(r[c]);
                } else if (r0 < m) {
                    float* ur = U + r0 + (size_t)(32 * colh + 16 * hh) * ldu;
                    if (n == 64) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) ur[(size_t)c * ldu] = __uint_as_float(r[c]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (32 * colh + 16 * hh + c < n) ur[(size_t)c * ldu] = __uint_as_float(r[c]);
                    }
                }
            }
            ut_fence_before();
            if (TS) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&S.acc_empty[b]);
                if (TS) mbar_arrive(&S.out_full);
            }
        };
        for (int j = 0; j < T && ok; ++j) {
            const int f = j % SF, o = j % UT_SO;
            if (!mbar_wait(&S.fp_full[f], (j / SF) & 1)) { ok = false; break; }
            if (j >= UT_SO && !mbar_wait(&S.op_empty[o], ((j / UT_SO) - 1) & 1)) { ok = false; break; }
            const float* fp = fpb + (size_t)f * 64 * UT_ROWS + row;
            unsigned char* oh = ops + (size_t)o * 2 * UT_OP_BYTES;
            unsigned char* ol = oh + UT_OP_BYTES;
#pragma unroll
            for (int g4 = 0; g4 < 8; ++g4) {
                float4 hi4, lo4;
                float* h = &hi4.x;
                float* l = &lo4.x;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kbase + 4 * g4 + u;
                    const float a = (n == 64 || k < n) ? fp[k * UT_ROWS] : 0.0f;
                    const float ah = ut_tf32(a);
                    h[u] = ah;
                    l[u] = ut_tf32(a - ah);
                }
                // row of the K-major operand: atom kbase / 32, 16-byte chunk g4 swizzled by row
                const uint32_t off = (uint32_t)(rowoff + ((g4 ^ (row & 7)) << 4));
                *reinterpret_cast<float4*>(oh + off) = hi4;
                *reinterpret_cast<float4*>(ol + off) = lo4;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&S.op_full[o]);
                mbar_arrive(&S.fp_empty[f]);
            }
            if (j >= 1) epilogue(j - 1);
        }
        if (ok && T > 0) epilogue(T - 1);
        if (!ok) atomicExch(&S.abort, 1);
    }
    // teardown: every tcgen05 access is complete before the TMEM is freed
    ut_fence_before();
    __syncthreads();
    if (S.abort && tid == 0) {
        atomicOr(&info->flags, FLAG_TIMEOUT);
        for (int j = (tma_issued > SF ? tma_issued - SF : 0); j < tma_issued; ++j)
            (void)mbar_wait(&S.fp_full[j % SF], (j / SF) & 1);
    }
    if (warp == 1) {
        __syncwarp();
        ut_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
    }
}

}  // namespace

bool compute_u_tc_ok(const void* A, int working, int64_t m, int n, int64_t lda) {
    // TMA: 16-byte aligned base and column stride
    return working == 0 && n >= 1 && n <= 64 && m >= 1 && ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
}

cudaError_t launch_compute_u_tc(const float* A, int64_t m, int n, int64_t lda, const float* W, float* U,
                                int64_t ldu, int sm_count, DevInfo* info, cudaStream_t s) {
    CUtensorMap tmap, tmapU;
    cudaError_t e = make_tmap_2d(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), A, (uint64_t)m,
                                 (uint64_t)n, (uint64_t)lda, UT_ROWS, (uint32_t)n, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (e != cudaSuccess) return e;
    // U written by TMA stores when its base and column stride are 16-byte aligned
    const bool ts = ((uintptr_t)U % 16 == 0) && (ldu % 4 == 0) &&
                    make_tmap_2d(&tmapU, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), U, (uint64_t)m, (uint64_t)n,
                                 (uint64_t)ldu, UT_ROWS, (uint32_t)n, CU_TENSOR_MAP_SWIZZLE_NONE) == cudaSuccess;
    if (!ts) tmapU = tmap;  // unused
    const int64_t tiles = (m + UT_ROWS - 1) / UT_ROWS;
    int64_t grid = sm_count;
    if (grid > tiles) grid = tiles;
    if (ts) {
        e = cudaFuncSetAttribute(compute_u_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ut_smem<true>());
        if (e != cudaSuccess) return e;
        compute_u_tc_kernel<true><<<(unsigned)grid, UT_THREADS, ut_smem<true>(), s>>>(tmap, tmapU, m, n, W, U, ldu, info);
    } else {
        e = cudaFuncSetAttribute(compute_u_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ut_smem<false>());
        if (e != cudaSuccess) return e;
        compute_u_tc_kernel<false><<<(unsigned)grid, UT_THREADS, ut_smem<false>(), s>>>(tmap, tmapU, m, n, W, U, ldu, info);
    }
    return cudaGetLastError();
}

}  // namespace tsvd
