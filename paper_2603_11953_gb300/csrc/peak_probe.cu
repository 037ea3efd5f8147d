// peak_probe.cu -- arithmetic peaks of the GPU the library runs on, measured
// with the library's own small kernels (libtsvd_probe.so, separate from
// libtsvd.so).  bench.py uses these as the denominators of the FP64, FP32 and
// integer-tensor roofline terms; the HBM and BF16 tensor denominators are
// measured elsewhere (a device copy and a cuBLAS GEMM).
//
// Each throughput kernel keeps 8 independent dependency chains per thread and
// runs one CTA of 512 threads per SM slot (4 per SM), so the pipe, not the
// latency, limits it.  Kinds:
//   0  FP64 fma.rn.f64                    2 flops per lane-op
//   1  FP32 fma.rn.f32                    2 flops per lane-op
//   2  FP32 fma.rn.f32x2 (packed pairs)   4 flops per lane-op
//   3  INT8 mma.sync m16n8k32 s8 -> s32   8192 ops per warp-op
//   4  BF16 mma.sync m16n8k16 -> f32      4096 flops per warp-op
//   5  dependent FP64 fma latency (one thread): cycles per operation in *ops
//   6  dependent FP32 fma latency (one thread): cycles per operation in *ops
//   7, 8, 9  FP64 fma stream with only 1, 8 or 16 lanes of each warp active
//            (does the narrow FP64 pipe charge for idle lanes?)
#include <cuda_runtime.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PROBE_API __attribute__((visibility("default")))
#else
#define PROBE_API
#endif

namespace {

constexpr int kThreads = 512;
constexpr int kCtasPerSm = 4;

__global__ void __launch_bounds__(kThreads) fp64_fma_kernel(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 123.456) out[blockIdx.x] = s;  // never true: keeps the chains alive
}

// kind 0 with only the first `active` lanes of every warp doing the work
__global__ void __launch_bounds__(kThreads) fp64_fma_partial_kernel(double* out, int iters, double a, double b,
                                                                    int active) {
    if ((threadIdx.x & 31) >= active) return;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 123.456) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fp32_fma_kernel(float* out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 123.456f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fp32x2_fma_kernel(float* out, int iters, float a, float b) {
    unsigned long long x[8], av, bv;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b), "f"(b));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float v0 = threadIdx.x * 1e-3f + k, v1 = v0 + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(v0), "f"(v1));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
    }
    float s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
        s += lo + hi;
    }
    if (s == 123.456f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) i8_mma_kernel(int* out, int iters) {
    uint32_t a[4], b[2];
    int c[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = 0x01020304u * (threadIdx.x + k);
    b[0] = 0x05060708u + threadIdx.x;
    b[1] = 0x0102fffeu;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) c[j][k] = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) s += c[j][k];
    if (s == 123456789) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) bf16_mma_kernel(float* out, int iters) {
    uint32_t a[4], b[2];
    float c[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = 0x3f803f80u;  // (1.0, 1.0) in bf16
    b[0] = b[1] = 0x3c003c00u;                       // small values, keeps the sums finite
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) c[j][k] = 0.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) s += c[j][k];
    if (s == 123.456f) out[blockIdx.x] = s;
}

__global__ void fp64_latency_kernel(double* out, long long* cycles, int iters, double a, double b) {
    double x = threadIdx.x + 1.0;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) x = fma(x, a, b);
    const long long t1 = clock64();
    out[0] = x;
    cycles[0] = t1 - t0;
}

__global__ void fp32_latency_kernel(float* out, long long* cycles, int iters, float a, float b) {
    float x = threadIdx.x + 1.0f;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) x = fmaf(x, a, b);
    const long long t1 = clock64();
    out[0] = x;
    cycles[0] = t1 - t0;
}

}  // namespace

// Run probe `kind` with `iters` iterations per thread.  *ops: operations
// performed (flops or integer ops; for kinds 5 and 6 the cycles per dependent
// operation); *ms: device time of the timed launch (after one warm-up
// launch).  Returns 0, or the CUDA error code.
extern "C" PROBE_API int tsvd_probe(int kind, int iters, double* ops, float* ms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || !ops || !ms || iters < 1) return e != cudaSuccess ? (int)e : -1;
    void* buf = nullptr;
    long long* cyc = nullptr;
    if ((e = cudaMalloc(&buf, 1 << 16)) != cudaSuccess) return (int)e;
    if ((e = cudaMalloc(&cyc, sizeof(long long))) != cudaSuccess) {
        cudaFree(buf);
        return (int)e;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sms * kCtasPerSm;
    const double lanes = (double)grid * kThreads;
    double count = 0;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        switch (kind) {
            case 0: fp64_fma_kernel<<<grid, kThreads>>>((double*)buf, iters, 0.999999, 1e-6); count = lanes * iters * 8 * 2; break;
            case 1: fp32_fma_kernel<<<grid, kThreads>>>((float*)buf, iters, 0.9999f, 1e-4f); count = lanes * iters * 8 * 2; break;
            case 2: fp32x2_fma_kernel<<<grid, kThreads>>>((float*)buf, iters, 0.9999f, 1e-4f); count = lanes * iters * 8 * 4; break;
            case 3: i8_mma_kernel<<<grid, kThreads>>>((int*)buf, iters); count = lanes / 32 * iters * 4 * 8192.0; break;
            case 4: bf16_mma_kernel<<<grid, kThreads>>>((float*)buf, iters); count = lanes / 32 * iters * 4 * 4096.0; break;
            case 5: fp64_latency_kernel<<<1, 1>>>((double*)buf, cyc, iters, 0.999999, 1e-6); break;
            case 6: fp32_latency_kernel<<<1, 1>>>((float*)buf, cyc, iters, 0.9999f, 1e-4f); break;
            case 7: case 8: case 9: {
                const int act = kind == 7 ? 1 : kind == 8 ? 8 : 16;
                fp64_fma_partial_kernel<<<grid, kThreads>>>((double*)buf, iters, 0.999999, 1e-6, act);
                count = lanes / 32 * act * iters * 8 * 2;
                break;
            }
            default: rep = 2; e = cudaErrorInvalidValue; break;
        }
        cudaEventRecord(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && (kind == 5 || kind == 6)) {
        long long c = 0;
        e = cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
        count = (double)c / iters;
    }
    *ops = count;
    *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(cyc);
    return (int)e;
}
