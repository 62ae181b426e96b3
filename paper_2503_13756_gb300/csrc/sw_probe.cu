// sw_probe.cu -- measured FP32 fused multiply-add throughput of the current
// GPU (not part of the method: it is the denominator of the ALU-bound
// rooflines that the benchmark reports for the projection and the CUDA-core
// correlation).
//
// Every thread runs kChains independent FFMA chains x <- x a + b for `iters`
// rounds, so each SM sub-partition always has independent FFMAs to issue;
// the grid fills every SM with 2048 resident threads.  The result of every
// chain feeds one store that the compiler cannot drop (it depends on a value
// only known at run time), so no chain is eliminated.  The kernel is timed
// with CUDA events after warm-up launches; the best of several timed launches
// is reported (the probe changes no clock or other setting of the GPU).
#include <cuda_runtime.h>

#include "swalign.h"

namespace {

constexpr int kChains = 16;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_ffma_probe(float *out, int iters, float a,
                                                               float b, float sentinel)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == sentinel) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" sw_status sw_measure_fp32_fma(int device, double *tflops, double *ms_per_launch)
{
    if (!tflops) return SW_ERR_INVALID_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SW_ERR_CUDA;
    }
    sw_status result = SW_OK;
    int sms = 0;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int iters = 8192;
    do {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
            sms <= 0) {
            result = SW_ERR_CUDA;
            break;
        }
        const int blocks = sms * (2048 / kProbeThreads);
        if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * kProbeThreads) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            result = SW_ERR_CUDA;
            break;
        }
        const float a = 0.99990f, b = 1e-4f, sentinel = -1.2345e30f;
        for (int w = 0; w < 3; ++w) k_ffma_probe<<<blocks, kProbeThreads>>>(out, iters, a, b, sentinel);
        float best = 1e30f;
        for (int r = 0; r < 10 && result == SW_OK; ++r) {
            cudaEventRecord(e0);
            k_ffma_probe<<<blocks, kProbeThreads>>>(out, iters, a, b, sentinel);
            cudaEventRecord(e1);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                result = SW_ERR_CUDA;
            else if (ms < best)
                best = ms;
        }
        if (result != SW_OK) break;
        const double flops = 2.0 * kChains * (double)iters * blocks * kProbeThreads;
        *tflops = flops / (best * 1e-3) / 1e12;
        if (ms_per_launch) *ms_per_launch = best;
    } while (false);
    if (result != SW_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    cudaSetDevice(prev);
    return result;
}
