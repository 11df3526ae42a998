// vbgs_probe.cu -- arithmetic peak probes for the ALU rooflines.
//
// The CUDA-core E-step kernels are bound by FP64 FMA, FP32 FMA or MUFU ex2
// throughput, none of which the copy/GEMM peaks describe.  Each probe runs
// 8 independent dependency chains per thread on every SM, calibrates its
// iteration count to a few milliseconds, and reports operations per second
// measured with CUDA events.
#include "vbgs_internal.cuh"
#include <algorithm>

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T *out, int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = T(threadIdx.x + i);
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < kChains; i++) a[i] = fma(a[i], b, c);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    if (s == T(-1.2345)) out[0] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(256) k_ex2(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) x[i] = 0.1f * (float)(i + 1) + 1e-6f * threadIdx.x;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < kChains; i++) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[i]) : "f"(-x[i]));
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += x[i];
    if (s == -1.2345f) out[0] = s;
}

template <typename F>
double time_ms(F launch, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    launch();
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

} // namespace

extern "C" int vbgs_probe_peaks(int device, double *out)
{
    if (!out) return VBGS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return VBGS_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st;
    cudaEvent_t e0, e1;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return VBGS_ECUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    void *buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) return VBGS_ENOMEM;
    const int blocks = sms * 8, threads = 256;
    const double work_per_iter = (double)blocks * threads * kChains;
    auto calibrated = [&](auto launcher) {
        int iters = 64;
        double ms = time_ms([&] { launcher(iters); }, st, e0, e1);
        for (int r = 0; r < 12 && ms < 4.0; r++) {
            iters = (int)std::min<double>(iters * std::max(2.0, 5.0 / std::max(ms, 1e-3)), 1 << 24);
            ms = time_ms([&] { launcher(iters); }, st, e0, e1);
        }
        return work_per_iter * iters / (ms * 1e-3);   // operations per second
    };
    double f64 = calibrated([&](int it) { k_fma<double><<<blocks, threads, 0, st>>>((double *)buf, it, 0.999, 1e-3); });
    double f32 = calibrated([&](int it) { k_fma<float><<<blocks, threads, 0, st>>>((float *)buf, it, 0.999f, 1e-3f); });
    double ex2 = calibrated([&](int it) { k_ex2<<<blocks, threads, 0, st>>>((float *)buf, it); });
    out[0] = 2.0 * f64 / 1e12;
    out[1] = 2.0 * f32 / 1e12;
    out[2] = ex2 / 1e9;
    out[3] = sms;
    cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    return e == cudaSuccess ? VBGS_OK : VBGS_ECUDA;
}
