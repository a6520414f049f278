// sbr_probe.cu -- measured peaks for the traversal's roofline: the L2 read
// bandwidth (a buffer that fits in L2, read again and again with loads that
// bypass L1) and the FP32 fused multiply-add throughput (independent FMA
// chains on every lane of every SM). Both are timed with CUDA events on a
// stream of their own after a warm-up launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "sbr.h"

namespace {

__global__ void __launch_bounds__(256) k_probe_fill(float4* buf, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        buf[i] = make_float4((float)(i & 1023), 1.f, 2.f, 3.f);
}

// every thread reads float4s at a stride of the grid size, `passes` times over
// the buffer; the bit-xor of what it read is written, so no load is dropped
__global__ void __launch_bounds__(256) k_probe_l2(const float4* __restrict__ buf, long long n, int passes,
                                                  unsigned* out)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x, s = (long long)gridDim.x * blockDim.x;
    unsigned acc = 0;
    for (int p = 0; p < passes; ++p)
        for (long long i = g; i < n; i += s) {
            const float4 v = __ldcg(buf + i);
            acc ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^ __float_as_uint(v.w);
        }
    out[g] = acc;
}

// 8 independent FMA chains per thread, `iters` rounds of 8 FMAs each
__global__ void __launch_bounds__(256) k_probe_fma(int iters, float a, float b, float* out)
{
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f, x4 = x0 + 4.f, x5 = x0 + 5.f,
          x6 = x0 + 6.f, x7 = x0 + 7.f;
    for (int k = 0; k < iters; ++k) {
        x0 = __fmaf_rn(x0, a, b);
        x1 = __fmaf_rn(x1, a, b);
        x2 = __fmaf_rn(x2, a, b);
        x3 = __fmaf_rn(x3, a, b);
        x4 = __fmaf_rn(x4, a, b);
        x5 = __fmaf_rn(x5, a, b);
        x6 = __fmaf_rn(x6, a, b);
        x7 = __fmaf_rn(x7, a, b);
    }
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

struct ProbeRes {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* p = nullptr;
    void* q = nullptr;
    ~ProbeRes()
    {
        if (st) cudaStreamSynchronize(st);
        if (p) cudaFree(p);
        if (q) cudaFree(q);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    }
};

int probe_setup(int device, ProbeRes& r, int& n_sms)
{
    if (cudaSetDevice(device) != cudaSuccess) return SBR_ERR_CUDA;
    if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SBR_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&r.st, cudaStreamNonBlocking) != cudaSuccess) return SBR_ERR_CUDA;
    if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) return SBR_ERR_CUDA;
    return SBR_OK;
}

}  // namespace

extern "C" int sbr_probe_l2_bandwidth(int device, int64_t bytes, int passes, double* gb_per_s)
{
    if (!gb_per_s || bytes < (1 << 20) || passes < 1 || passes > 1000) return SBR_ERR_ARG;
    ProbeRes r;
    int n_sms = 0;
    int rc = probe_setup(device, r, n_sms);
    if (rc != SBR_OK) return rc;
    const long long n = bytes / (long long)sizeof(float4);
    const int blocks = n_sms * 8, threads = 256;
    if (cudaMalloc(&r.p, (size_t)n * sizeof(float4)) != cudaSuccess) return SBR_ERR_OOM;
    if (cudaMalloc(&r.q, sizeof(unsigned) * (size_t)blocks * threads) != cudaSuccess) return SBR_ERR_OOM;
    k_probe_fill<<<blocks, threads, 0, r.st>>>((float4*)r.p, n);
    k_probe_l2<<<blocks, threads, 0, r.st>>>((const float4*)r.p, n, 2, (unsigned*)r.q);  // warm-up: brings the buffer into L2
    cudaEventRecord(r.e0, r.st);
    k_probe_l2<<<blocks, threads, 0, r.st>>>((const float4*)r.p, n, passes, (unsigned*)r.q);
    cudaEventRecord(r.e1, r.st);
    if (cudaStreamSynchronize(r.st) != cudaSuccess) return SBR_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess || !(ms > 0.f)) return SBR_ERR_CUDA;
    *gb_per_s = (double)n * sizeof(float4) * passes / (ms * 1e-3) / 1e9;
    return SBR_OK;
}

extern "C" int sbr_probe_fp32_fma(int device, double* tflops)
{
    if (!tflops) return SBR_ERR_ARG;
    ProbeRes r;
    int n_sms = 0;
    int rc = probe_setup(device, r, n_sms);
    if (rc != SBR_OK) return rc;
    const int blocks = n_sms * 8, threads = 256, iters = 1 << 15;
    if (cudaMalloc(&r.q, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) return SBR_ERR_OOM;
    k_probe_fma<<<blocks, threads, 0, r.st>>>(256, 0.999f, 1e-3f, (float*)r.q);  // warm-up
    cudaEventRecord(r.e0, r.st);
    k_probe_fma<<<blocks, threads, 0, r.st>>>(iters, 0.999f, 1e-3f, (float*)r.q);
    cudaEventRecord(r.e1, r.st);
    if (cudaStreamSynchronize(r.st) != cudaSuccess) return SBR_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess || !(ms > 0.f)) return SBR_ERR_CUDA;
    // two floating-point operations per fused multiply-add
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    return SBR_OK;
}
