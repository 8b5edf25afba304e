// Throughput microbenchmarks for the blend kernels' rooflines (sm_103a): FP32 FMA and exp2f.
//
// Each thread runs kChains independent dependency chains, so every SM sub-partition has enough
// independent work in flight to keep its pipe busy; the grid fills every SM several times. The
// chains' values are stored at the end, so the compiler keeps the arithmetic.
#include <cuda_runtime.h>

#include "odgs.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- exp2f(-x) stays in [2^-1, 1] for x in [0, 1], so every evaluation is an ordinary one.
__global__ void __launch_bounds__(kThreads) k_peak_ex2(float* out, int iters) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = exp2f(-x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Milliseconds of the second of two launches (the first warms up clocks and caches).
template <typename Launch>
cudaError_t time_launch(Launch launch, cudaStream_t st, float* ms) {
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    launch();
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" odgs_status odgs_measure_peaks(odgs_peaks* out, void* stream) {
    if (!out) return ODGS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ODGS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return ODGS_ERR_CUDA;
    const int blocks = sms * kBlocksPerSm;
    const double threads = (double)blocks * kThreads;
    float* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess) return ODGS_ERR_CUDA;
    const int it_fma = 1 << 14, it_ex2 = 1 << 12;
    float ms_fma = 0.f, ms_ex2 = 0.f;
    cudaError_t e = time_launch([&] { k_peak_ffma<<<blocks, kThreads, 0, st>>>(buf, it_fma, 0.999999f, 1e-6f); },
                                st, &ms_fma);
    if (e == cudaSuccess)
        e = time_launch([&] { k_peak_ex2<<<blocks, kThreads, 0, st>>>(buf, it_ex2); }, st, &ms_ex2);
    cudaFree(buf);
    if (e != cudaSuccess || ms_fma <= 0.f || ms_ex2 <= 0.f) return ODGS_ERR_CUDA;
    const double fmas = threads * it_fma * 4.0 * kChains;
    const double ex2s = threads * it_ex2 * 4.0 * kChains;
    out->ffma_tflops = 2.0 * fmas / (ms_fma * 1e-3) / 1e12;
    out->ex2_gops = ex2s / (ms_ex2 * 1e-3) / 1e9;
    out->sms = sms;
    return ODGS_OK;
}
