// Instrumentation: the FP64 fused multiply-add rate of the current GPU,
// the ALU roofline of the FP64 hop (GB300 has a reduced FP64 rate and no
// measured FP64 peak).  Every thread runs 8 independent dependency
// chains of a = a * b + c, so the FP64 pipe, not latency, sets the time.
#include "api_util.h"

namespace {

__global__ void __launch_bounds__(256) dfma_kernel(int iters, double b, double c, double* out) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
    if (s == 12345.678) out[0] = s;  // keeps the chains live; never true in practice
}

}  // namespace

extern "C" int eofa_probe_fp64_fma(double* tflops) {
    if (!tflops) return EOFA_EINVAL;
    try {
        int dev = 0, sms = 0;
        EOFA_CUDA(cudaGetDevice(&dev));
        EOFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        double* out = nullptr;
        EOFA_CUDA(cudaMalloc(&out, sizeof(double)));
        cudaEvent_t e0, e1;
        EOFA_CUDA(cudaEventCreate(&e0));
        EOFA_CUDA(cudaEventCreate(&e1));
        const int blocks = sms * 8, threads = 256, iters = 1 << 14;
        dfma_kernel<<<blocks, threads>>>(64, 0.999999, 1e-7, out);  // warm-up
        EOFA_LAUNCHED();
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            EOFA_CUDA(cudaEventRecord(e0));
            dfma_kernel<<<blocks, threads>>>(iters, 0.999999, 1e-7, out);
            EOFA_LAUNCHED();
            EOFA_CUDA(cudaEventRecord(e1));
            EOFA_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            EOFA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) best = ms;
        }
        EOFA_CUDA(cudaEventDestroy(e0));
        EOFA_CUDA(cudaEventDestroy(e1));
        EOFA_CUDA(cudaFree(out));
        const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
        *tflops = flops / (best * 1e-3) / 1e12;
    } catch (const eofa_error& e) {
        return e.code;
    }
    return EOFA_OK;
}
