// hcg_peaks.cu -- a measurement helper outside the gridding path: the FP32
// fused multiply-add throughput of the device, the denominator of the
// arithmetic roofline of the CUDA-core gathers (one FMA per contribution).
#include <algorithm>

#include "hcg_internal.h"

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread (hides the FMA latency)
constexpr int kUnroll = 16;

// Every thread runs kChains dependent chains of `iters` x kUnroll FMAs; the
// sums are stored only when a thread's result hits an impossible value, so
// the work cannot be removed but nothing is written.
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float a, float b, float *sink) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    if (s == -1.2345e30f) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" hcg_status hcg_measure_fp32_peak(int device, double *tflops) {
    if (!tflops) { hcg_set_error("null output"); return HCG_ERR_INVALID_ARG; }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaSetDevice");
    int nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, 256, 0);
    const int blocks = nsm * std::max(1, per_sm);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    hcg_status s = HCG_OK;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = cudaMalloc((void **)&sink, 256 * sizeof(float))) != cudaSuccess) {
        s = hcg_cuda_fail(e, "peak measurement set-up");
    } else {
        const int iters = 4096;
        const float a = 0.999999f, b = 1e-7f;
        for (int w = 0; w < 3; w++) k_fma_peak<<<blocks, 256, 0, st>>>(iters, a, b, sink);   // warm-up, clocks up
        double best = 0;
        for (int r = 0; r < 5 && s == HCG_OK; r++) {
            cudaEventRecord(e0, st);
            k_fma_peak<<<blocks, 256, 0, st>>>(iters, a, b, sink);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { s = hcg_cuda_fail(e, "peak kernel"); break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            const double flops = 2.0 * blocks * 256.0 * (double)iters * kUnroll * kChains;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
        *tflops = best;
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return s;
}
