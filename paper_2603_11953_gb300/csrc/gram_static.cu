// gram_static.cu -- tsvd_gram_static: the Gram matrix without any allocation.
//
// Some callers cannot call cudaMalloc: services that reserve all device
// memory up front and forbid allocation on the request path, plug-ins that
// must not own device memory of their own, and code that may not risk the
// implicit device synchronisation of cudaMalloc / cudaFree.  tsvd_gram
// needs a handle, and a handle allocates its workspace; this entry point
// needs neither.  The split-K partials of the tensor-core Gram and the small
// status block live instead in one file-scope device array of fixed size
// (TSVD_GRAM_STATIC_SCRATCH_BYTES), which every GPU that loads this part of
// the library holds until the process exits.
//
// Set-up: host code cannot use the array's name as a device address (on the
// host it only names a stand-in), so the first call on each device asks the
// runtime for the real address with cudaGetSymbolAddress, with that device
// current, and caches it.  That first call per device should come before any
// stream capture.
//
// All calls share the one array and each call leaves its contents behind:
// the status block is cleared at the start of every call and every partial
// is overwritten by the Gram kernel before it is read.  Calls that overlap
// on the GPU (for example on two streams at once) race on the array.
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

// Device address of g_gram_scratch on `dev` (which must be current).
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
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
    // Largest split-K the array can hold for this n; beyond it the rows per
    // CTA would exceed the int64 accumulator range, so larger m is refused.
    GramPlan plan = gram_plan(m, (int)n, sm_count, 0);
    const size_t per_cta = (size_t)plan.NP * plan.NP * sizeof(long long) * 2 + (size_t)plan.NP * sizeof(int);
    const int64_t cap_ctas = (int64_t)((kScratchBytes - kInfoBytes - 256) / per_cta);
    if (plan.P > cap_ctas) plan = gram_plan(m, (int)n, sm_count, (int)cap_ctas);
    if (plan.P > cap_ctas || gram_partials_bytes(plan) > kScratchBytes - kInfoBytes)
        return TSVD_ERR_UNSUPPORTED;  // m too large for the static scratch array

    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess) return status_of(e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base);
    void* part = base + kInfoBytes;
    e = cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s);
    if (e == cudaSuccess) e = launch_gram_ozaki(A, 0, m, (int)n, lda, plan, part, dinfo, s);
    if (e == cudaSuccess)
        e = launch_gram_combine(plan, part, (int)n, G, higher == TSVD_DD ? G + ldg * n : nullptr, ldg, s);
    if (e == cudaSuccess) e = launch_finalize_info(dinfo, s);
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, dinfo, sizeof(DevInfo), cudaMemcpyDefault, s);
    return status_of(e);
}
