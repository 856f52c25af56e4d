// peaks.cu -- CUDA-core arithmetic peaks of the device, measured: the
// ceilings that bound the sweeps when they are not memory-bound (the FP64
// path, and K1, whose recurrences issue mostly FMAs and shared loads).
//
// One kernel per kind keeps kChains independent FMA chains per thread in
// registers and runs them for `iters` rounds; the grid holds enough warps
// per SM to cover the FMA latency.  FLOPs = 2 per FMA (4 per packed FFMA2).
#include <cuda_runtime.h>

#include <string>

#include "ads.h"
#include "internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// out is written only when the accumulated value equals `never` (it does not
// for the inputs used), which keeps the chains live without a store per thread
__global__ void __launch_bounds__(kThreads) k_dfma(double a, double b, int iters, double never, double *out)
{
    double c[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) c[k] = fma(c[k], a, b);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += c[k];
    if (s == never) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_ffma(float a, float b, int iters, float never, float *out)
{
    float c[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) c[k] = fmaf(c[k], a, b);
    }
    float s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += c[k];
    if (s == never) out[0] = s;
}

// packed FP32: one FFMA2 instruction is two FMAs on a pair of registers
__global__ void __launch_bounds__(kThreads) k_ffma2(float a, float b, int iters, float never, float *out)
{
    float2 c[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) c[k] = __ffma2_rn(c[k], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += c[k].x + c[k].y;
    if (s == never) out[0] = s;
}

}  // namespace

extern "C" int ads_measure_fma_peak(int device, int kind, int iters, double *tflops, double *ms_out)
{
    if (!tflops || kind < 0 || kind > 2 || iters < 1 || iters > (1 << 24))
        return ads_internal_fail(ADS_ERR_INVALID_ARG, "ads_measure_fma_peak: arguments");
    int dev0 = 0;
    if (cudaGetDevice(&dev0) != cudaSuccess) {
        cudaGetLastError();
        return ads_internal_fail(ADS_ERR_CUDA, "ads_measure_fma_peak: no CUDA device");
    }
    const int dev = device < 0 ? dev0 : device;
    if (dev != dev0 && cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return ads_internal_fail(ADS_ERR_CUDA, "ads_measure_fma_peak: cannot select the device");
    }
    int rc = ADS_OK;
    int sms = 0;
    void *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && rc == ADS_OK) {
            cudaGetLastError();
            rc = ads_internal_fail(ADS_ERR_CUDA, (std::string("ads_measure_fma_peak: ") + what + ": " +
                                                  cudaGetErrorString(e)).c_str());
        }
        return rc == ADS_OK;
    };
    if (ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count") &&
        ck(cudaMalloc(&sink, 64), "sink") && ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream") &&
        ck(cudaEventCreate(&e0), "event") && ck(cudaEventCreate(&e1), "event")) {
        // 8 CTAs of 256 threads per SM: 64 warps, 16 per scheduler
        const dim3 grid((unsigned)(sms * 8)), block(kThreads);
        auto launch = [&]() {
            if (kind == 0) k_dfma<<<grid, block, 0, st>>>(1.0000001, 1e-9, iters, -1.0, (double *)sink);
            else if (kind == 1) k_ffma<<<grid, block, 0, st>>>(1.0000001f, 1e-9f, iters, -1.0f, (float *)sink);
            else k_ffma2<<<grid, block, 0, st>>>(1.0000001f, 1e-9f, iters, -1.0f, (float *)sink);
            return cudaGetLastError();
        };
        if (ck(launch(), "warm-up launch") && ck(cudaEventRecord(e0, st), "record") && ck(launch(), "launch") &&
            ck(cudaEventRecord(e1, st), "record") && ck(cudaEventSynchronize(e1), "sync")) {
            float ms = 0;
            if (ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed")) {
                const double fma_per_thread = (double)iters * kChains * (kind == 2 ? 2 : 1);
                const double flops = 2.0 * fma_per_thread * grid.x * kThreads;
                *tflops = flops / (ms * 1e-3) / 1e12;
                if (ms_out) *ms_out = ms;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (dev != dev0) cudaSetDevice(dev0);
    return rc;
}
