// tma_util.cuh -- tensor-map (TMA) creation on the host and the mbarrier /
// bulk-tensor PTX helpers shared by the streaming kernels.  Every wait on an
// mbarrier is bounded: after about a second of GPU clock it reports failure and the
// caller records TSVD_ERR_TIMEOUT instead of spinning forever.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tsvd {

// Give up on an mbarrier after about one second of GPU clock (2^31 cycles).
constexpr long long TMA_WAIT_CYCLES = 1ll << 31;

// Host: encode a 2-D tiled tensor map over a column-major matrix
// (inner dimension = rows, contiguous; outer = columns, stride ld elements).
// Returns cudaErrorNotSupported when the driver entry point is unavailable
// or the map is rejected (alignment, box size).
cudaError_t make_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, size_t elem_bytes,
                         const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                         uint32_t box_rows, uint32_t box_cols, CUtensorMapSwizzle swizzle);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Wait for the phase with parity `parity` to complete; false when `limit`
// cycles (default about a second of GPU clock) have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = TMA_WAIT_CYCLES) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}
// As mbar_wait, with a suspend-time hint: a warp whose phase is not complete is descheduled
// until it completes or hint_ns nanoseconds pass, and does not take issue slots meanwhile.
__device__ __forceinline__ bool mbar_wait_susp(uint64_t* bar, unsigned parity, long long limit = TMA_WAIT_CYCLES,
                                               unsigned hint_ns = 2000) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}
// 2-D tiled TMA load of the box at (x = row, y = column) into dst.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace tsvd
