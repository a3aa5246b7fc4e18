// Measured FP64 fused multiply-add rate of the device: the denominator of
// the FP64 step's roofline.  On this GPU the FP64 units, not HBM, bound the
// FP64 step, and the vendor's nominal FP64 figure is no substitute for a
// measurement on the part at hand.  The paper has no counterpart (it
// measures the machine, not the method).
//
// Every thread runs eight independent FMA chains a <- a * b + c with
// |b| < 1, so the values stay bounded and no chain waits on another; the
// grid fills every SM with 2048 resident threads.  The chains' sum is
// compared with a value it never takes, which keeps the compiler from
// removing them; nothing is written in practice.
#include "ddcc.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma_rate(double* __restrict__ sink, int iters, double seed) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + 1e-3 * k + 1e-7 * threadIdx.x;
    const double b = 1.0 - 1e-9, c = 1e-9;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) sink[blockIdx.x] = s;   // never true: a[k] stays in (0, 2)
}

}  // namespace

extern "C" int ddcc_measure_fp64_peak(void* cuda_stream, double* dev_sink, double* tflops_out) {
    if (!tflops_out) return DDCC_ERR_PARAM;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return DDCC_ERR_CUDA;
    const int blocks = 8 * sms, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return DDCC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DDCC_ERR_CUDA;
    }
    int st = DDCC_OK;
    float best = 0.0f;
    for (int rep = 0; rep < 4 && st == DDCC_OK; ++rep) {   // the first run warms up
        cudaEventRecord(e0, s);
        k_dfma_rate<<<blocks, threads, 0, s>>>(dev_sink, iters, 0.5);
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = DDCC_ERR_CUDA;
        else if (rep > 0 && (best == 0.0f || ms < best))
            best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != DDCC_OK) return st;
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    return DDCC_OK;
}
