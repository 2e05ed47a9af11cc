// sg_measure_peak: the arithmetic throughput of the current device, measured
// with register-resident multiply-add loops on every SM.  It supplies the
// denominators of the roofline fractions the benchmark reports (the FP32 and
// FP64 CUDA-core rates); it is not part of the method of the paper.
//
// Each thread runs kChains independent chains a_i <- a_i * b + c, so every
// multiply-add depends only on its own chain's previous value; with 32 warps
// per SM the schedulers always have independent instructions to issue.  The
// loop count is calibrated by a short launch, then one launch of about the
// requested duration is timed with CUDA events on the caller's stream.
#include <algorithm>
#include <string>

#include "sg_internal.h"

namespace {

#ifndef SG_PEAK_CHAINS
#define SG_PEAK_CHAINS 16
#endif
constexpr int kChains = SG_PEAK_CHAINS;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 4;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(T *out, T b, T c, long long iters)
{
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = (T)(threadIdx.x + i);
    for (long long n = 0; n < iters; n++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32: one fma.rn.f32x2 instruction does two single-precision
// multiply-adds (sm_100 family and later).
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma2(float *out, float b, float c, long long iters)
{
    unsigned long long a[kChains], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        const float lo = (float)(threadIdx.x + i), hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(lo), "f"(hi));
    }
    for (long long n = 0; n < iters; n++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) a[i] = fma2(a[i], bb, cc);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One timed launch: returns its duration in ms (or a negative value on error).
float timed_launch(int kind, void *buf, unsigned blocks, long long iters, cudaStream_t s, cudaError_t *err)
{
    cudaEvent_t e0, e1;
    *err = cudaEventCreate(&e0);
    if (*err != cudaSuccess) return -1.0f;
    *err = cudaEventCreate(&e1);
    if (*err != cudaSuccess) { cudaEventDestroy(e0); return -1.0f; }
    // b slightly below 1 and c small keep every chain finite for any length
    cudaEventRecord(e0, s);
    if (kind == SG_PEAK_FP32)
        k_peak_fma<float><<<blocks, kPeakThreads, 0, s>>>(static_cast<float *>(buf), 0.999999f, 1e-7f, iters);
    else if (kind == SG_PEAK_FP32X2)
        k_peak_fma2<<<blocks, kPeakThreads, 0, s>>>(static_cast<float *>(buf), 0.999999f, 1e-7f, iters);
    else
        k_peak_fma<double><<<blocks, kPeakThreads, 0, s>>>(static_cast<double *>(buf), 0.999999, 1e-7, iters);
    *err = cudaGetLastError();
    cudaEventRecord(e1, s);
    float ms = -1.0f;
    if (*err == cudaSuccess) *err = cudaEventSynchronize(e1);
    if (*err == cudaSuccess) *err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return *err == cudaSuccess ? ms : -1.0f;
}

}  // namespace

extern "C" sg_status sg_measure_peak(int kind, double seconds, double *flops_per_s, int *sms, void *stream)
{
    if (kind != SG_PEAK_FP32 && kind != SG_PEAK_FP32X2 && kind != SG_PEAK_FP64) return SG_EINVAL;
    if (!(seconds > 0.0) || seconds > 60.0 || !flops_per_s) return SG_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SG_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return SG_ECUDA;
    if (sms) *sms = nsm;
    const unsigned blocks = (unsigned)nsm * kPeakBlocksPerSM;
    const size_t threads = (size_t)blocks * kPeakThreads;
    void *buf = nullptr;
    if (cudaMalloc(&buf, threads * sizeof(double)) != cudaSuccess) return SG_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaSuccess;
    // calibration: a short launch, then one of about `seconds`
    long long iters = 1 << 14;
    float ms = timed_launch(kind, buf, blocks, iters, s, &err);
    if (ms > 0.0f) {
        const double scale = seconds * 1e3 / std::max(ms, 1e-3f);
        iters = std::max<long long>(1, (long long)((double)iters * scale));
        ms = timed_launch(kind, buf, blocks, iters, s, &err);
    }
    cudaFree(buf);
    if (err != cudaSuccess || ms <= 0.0f) return SG_ECUDA;
    const double fma_per_chain = kind == SG_PEAK_FP32X2 ? 2.0 : 1.0;
    *flops_per_s = 2.0 * fma_per_chain * kChains * (double)iters * (double)threads / (ms * 1e-3);
    return SG_OK;
}
