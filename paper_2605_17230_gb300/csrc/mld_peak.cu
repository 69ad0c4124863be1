// Measurement helper: the FP32 FFMA rate this GPU sustains, for the roofline
// of the FP32 sweep kernels (the method itself does not use it).
//
// Every thread runs kChains independent FMA chains (enough in flight to cover
// the pipe latency) for `iters` iterations on registers; the result is
// folded into one store per thread so that no chain is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mld_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_peak_kernel(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" mld_status mld_measure_fp32_peak(double seconds, double* tflops, int* sm_count) {
    if (!tflops || !(seconds > 0.0)) return MLD_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    if (sm_count) *sm_count = sms;
    const int threads = 256, blocks = sms * 8;     // 64 warps per SM
    float* out = nullptr;
    if (cudaMalloc(&out, (size_t)threads * blocks * sizeof(float)) != cudaSuccess) return MLD_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    mld_status st = MLD_OK;
    // a = 1, b = 0 keeps every value finite (x stays x); the compiler cannot
    // know that, a and b are kernel arguments
    int iters = 1024;
    ffma_peak_kernel<<<blocks, threads>>>(out, iters, 1.f, 0.f);   // warm-up
    float ms = 0.f;
    for (int rep = 0; rep < 12; ++rep) {          // grow the launch to the requested duration
        cudaEventRecord(e0);
        ffma_peak_kernel<<<blocks, threads>>>(out, iters, 1.f, 0.f);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = MLD_ERR_CUDA; break; }
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms * 1e-3 >= seconds || iters >= (1 << 24)) break;
        iters *= 2;
    }
    if (st == MLD_OK) {
        const double fl = 2.0 * kChains * 16.0 * iters * (double)threads * blocks;
        *tflops = fl / (ms * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
