// gram_static.cu -- tsvd_gram_static: the Gram matrix without any allocation.
//
// Some callers cannot call cudaMalloc: services that reserve all device
// memory up front and forbid allocation on the request path, plug-ins that
// must not own device memory of their own, and code that may not risk the
// implicit device synchronisation of cudaMalloc / cudaFree.  tsvd_gram
// needs a handle, and a handle allocates its workspace; this entry point
// needs neither.  The split-K partials of the Gram and the small status block
// live instead in one file-scope device array of fixed size
// (TSVD_GRAM_STATIC_SCRATCH_BYTES), which every GPU that loads this part of
// the library holds until the process exits.
//
// The kernels are those tsvd_gram runs with default options: input that TMA
// can load (16-byte aligned A, lda a multiple of 4) goes to the tcgen05 Gram
// with the same split-K plan, so the result is bitwise that of tsvd_gram;
// other input goes to the mma.sync Ozaki Gram, whose split-K may be capped by
// the array size (same error bound, possibly other bits).
//
// Set-up: host code cannot use the array's name as a device address (on the
// host it only names a stand-in), so the first call on each device (and the
// first after that device's context changed, e.g. after cudaDeviceReset)
// asks the runtime for the real address with cudaGetSymbolAddress, with that
// device current, and caches it with the context it belongs to.  That first
// call per device should come before any stream capture.
//
// All calls share the one array and each call leaves its contents behind:
// the status block is cleared at the start of every call and every partial
// is overwritten by the Gram kernel before it is read.  Calls that overlap
// on the GPU (for example on two streams at once) race on the array.
#include <cuda.h>

#include <mutex>

#include "internal.cuh"

using namespace tsvd;

namespace {

constexpr size_t kScratchBytes = TSVD_GRAM_STATIC_SCRATCH_BYTES;
constexpr size_t kInfoBytes = 256;  // DevInfo block at the start of the array
static_assert(sizeof(DevInfo) <= kInfoBytes, "status block does not fit");

static __device__ __align__(256) unsigned char g_gram_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_looked_up = false;

// The current driver context (null when none is current or the driver entry
// point is unavailable).
CUcontext current_context() {
    if (!g_ctx_looked_up) {
        g_ctx_looked_up = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
        else
            cudaGetLastError();
    }
    CUcontext c = nullptr;
    if (g_ctx_get == nullptr || g_ctx_get(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of g_gram_scratch on `dev` (which must be current).  The
// cached address is only reused while the context it was taken in is still
// the current one; a new context (after a device reset) loads the module
// again, at a new address.
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    const CUcontext ctx = current_context();
    if (g_scratch_addr[dev] == nullptr || ctx == nullptr || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context();  // the runtime has made its context current by now
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

tsvd_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return TSVD_OK;
    if (e == cudaErrorNotSupported) return TSVD_ERR_UNSUPPORTED;
    return TSVD_ERR_CUDA;
}

}  // namespace

extern "C" tsvd_status tsvd_gram_static(const void* A, int64_t m, int64_t n, int64_t lda,
                                        tsvd_prec working, tsvd_prec higher, double* G, int64_t ldg,
                                        tsvd_info* info, void* stream) {
    if (!A || !G || m < 1 || n < 1 || lda < m || ldg < n ||
        (working != TSVD_FP32 && working != TSVD_FP64) || (higher != TSVD_FP64 && higher != TSVD_DD))
        return TSVD_ERR_ARG;
    if (working != TSVD_FP32 || n > 64) return TSVD_ERR_UNSUPPORTED;
    int dev = -1, sm_count = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices ||
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TSVD_ERR_CUDA;
    }
    // The plan tsvd_gram would use; when its partials do not fit the array, the
    // largest split-K the array holds for this n, unless that leaves more rows
    // per CTA than the int64 accumulators allow (then m is refused).
    const bool tc = gram_tc_ok(A, 0, (int)n, lda);
    GramPlan plan = tc ? gram_tc_plan(m, (int)n, sm_count, 0) : gram_plan(m, (int)n, sm_count, 0);
    const size_t per_cta = (size_t)plan.NP * plan.NP * sizeof(long long) * 2 + (size_t)plan.NP * sizeof(int);
    const int64_t cap_ctas = (int64_t)((kScratchBytes - kInfoBytes - 256) / per_cta);
    if (plan.P > cap_ctas)
        plan = tc ? gram_tc_plan(m, (int)n, sm_count, (int)cap_ctas) : gram_plan(m, (int)n, sm_count, (int)cap_ctas);
    if (plan.P > cap_ctas || plan.rows_per_cta > GRAM_MAX_ROWS_PER_CTA ||
        gram_partials_bytes(plan) > kScratchBytes - kInfoBytes)
        return TSVD_ERR_UNSUPPORTED;  // m too large for the static scratch array

    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess) return status_of(e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base);
    void* part = base + kInfoBytes;
    e = cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s);
    if (e == cudaSuccess)
        e = tc ? launch_gram_tc(A, m, (int)n, lda, plan, part, dinfo, s)
               : launch_gram_ozaki(A, 0, m, (int)n, lda, plan, part, dinfo, s);
    if (e == cudaSuccess)
        e = launch_gram_combine(plan, part, (int)n, G, higher == TSVD_DD ? G + ldg * n : nullptr, ldg, s);
    if (e == cudaSuccess) e = launch_finalize_info(dinfo, s);
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, dinfo, sizeof(DevInfo), cudaMemcpyDefault, s);
    return status_of(e);
}
