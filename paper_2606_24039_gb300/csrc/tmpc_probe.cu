// Measurement helper: the FP32 FMA throughput of the device, the denominator
// of the roofline of the FMA-issue-bound solve kernels.  Every thread runs
// eight independent FMA chains (no dependency stall at full occupancy), eight
// CTAs of 256 threads per SM.
#include <cuda_runtime.h>

#include "tmpc.h"

namespace {

__global__ void fma_chains(float* out, int iters, float a, float b) {
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
    float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
            x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

extern "C" tmpc_status tmpc_fp32_fma_probe(float* tflops, float* ms) {
    if (!tflops) return TMPC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TMPC_ERR_CUDA;
    const int threads = 256, blocks = sms * 8, iters = 4096;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * threads * blocks) != cudaSuccess) return TMPC_ERR_OOM;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tmpc_status st = TMPC_OK;
    float best = 1e30f;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        st = TMPC_ERR_CUDA;
    } else {
        for (int r = 0; r < 8 && st == TMPC_OK; ++r) {   // 3 warm-up launches, then the fastest of 5
            cudaEventRecord(e0, s);
            fma_chains<<<blocks, threads, 0, s>>>(out, iters, 0.999f, 0.001f);
            cudaEventRecord(e1, s);
            float t = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                st = TMPC_ERR_CUDA;
            else if (r >= 3 && t < best)
                best = t;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    if (st != TMPC_OK) return st;
    const double flops = 2.0 * 8 * 16 * (double)iters * threads * blocks;
    *tflops = (float)(flops / (best * 1e-3) / 1e12);
    if (ms) *ms = best;
    return TMPC_OK;
}
