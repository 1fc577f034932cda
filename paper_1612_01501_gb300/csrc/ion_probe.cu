// ion_probe.cu -- throughput probes of the units the kernels depend on: the SFU
// (ex2.approx; tanh.approx.bf16x2 for the surrogate's activations) and the FP32 FMA pipe.
// They give the measured denominators of the rooflines at the clock the GPU runs at.
//
// Each thread runs 8 independent dependency chains so that latency is hidden; the
// chains feed back into themselves so nothing can be hoisted or removed.  The ex2 chain
// is x <- 2^(-x), which stays in [0.5, 1] for x in [0, 1].
#include <cuda_runtime.h>

#include "ion.h"
#include "ion_kernels.cuh"
#include "ion_sim.h"

namespace ion {

__global__ void probe_ex2_kernel(float *out, int iters) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 0.1f * k + 1e-3f * (threadIdx.x & 7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = ex2_approx(-x[k]);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.0f) out[threadIdx.x] = s;   // never true; keeps the chains alive
}

__global__ void probe_ffma_kernel(float *out, int iters) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 0.1f * k;
    const float a = 0.999f, b = 1e-4f * (threadIdx.x & 3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.0f) out[threadIdx.x] = s;
}

// tanh.approx.bf16x2 (the surrogate's activation): x <- tanh(x + 0.5) on packed pairs
__global__ void probe_tanh_kernel(float *out, int iters) {
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 0x3E003E00u + (uint32_t)k + (threadIdx.x & 7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm("tanh.approx.bf16x2 %0, %1;" : "=r"(x[k]) : "r"(x[k]));
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= x[k];
    if (s == 0x12345678u) out[threadIdx.x] = (float)s;
}

}  // namespace ion

// rate_out: operations per second (ex2 results, or FMAs) over the whole GPU.
extern "C" ion_status ion_probe_peak(int32_t what, int32_t iters, void *stream, double *rate_out) {
    if (!rate_out || iters < 1 || what < 0 || what > 2)
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_probe_peak: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = sms * 8;
    float *d = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&d, threads * sizeof(float)) != cudaSuccess)
        return ion_fail(nullptr, ION_ERR_OOM, "ion_probe_peak: allocation failed");
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int rep = 0; rep < 2; ++rep) {   // first pass warms up
        cudaEventRecord(e0, st);
        if (what == 0) ion::probe_ex2_kernel<<<blocks, threads, 0, st>>>(d, iters);
        else if (what == 1) ion::probe_ffma_kernel<<<blocks, threads, 0, st>>>(d, iters);
        else ion::probe_tanh_kernel<<<blocks, threads, 0, st>>>(d, iters);
        cudaEventRecord(e1, st);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_probe_peak: %s", cudaGetErrorString(e));
    *rate_out = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    return ION_OK;
}
