// Peak probes for the rooflines of the CUDA-core kernels: FP32 FMA rate (one-
// lane fma and two-lane fma.rn.f32x2) and MUFU ex2 rate, measured with CUDA
// events on the caller's stream.  Each thread runs 8 independent dependency
// chains so that latency is hidden; the grid is 8 x the SM count x 1024
// threads.  Results are written to a device buffer the caller reads back.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024) fma_probe(int iters, float a, float b, float *sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) *sink = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(1024) fma2_probe(int iters, float a, float b, float *sink) {
    unsigned long long x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) {
        const float lo = threadIdx.x * 1e-3f + 2 * c, hi = lo + 1.f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    unsigned long long av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 1234.5f) *sink = s;
}

// y <- 2^(-y) stays in [0.5, 1) for y in (0, 1]
__global__ void __launch_bounds__(1024) ex2_probe(int iters, float *sink) {
    float y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) y[c] = 0.5f + 0.01f * c + threadIdx.x * 1e-6f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) y[c] = ex2_approx(-y[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += y[c];
    if (s == 1234.5f) *sink = s;
}

}  // namespace

cudaError_t measure_alu_peaks(double *out3, cudaStream_t st) {
    int dev = 0, sms = 148;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *sink = nullptr;
    e = cudaMallocAsync(&sink, sizeof(float), st);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 8 * sms, threads = 1024;
    const int iters_fma = 4096, iters_ex2 = 1024;
    double res[3] = {0, 0, 0};
    for (int which = 0; which < 3 && e == cudaSuccess; ++which) {
        for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
            cudaEventRecord(e0, st);
            if (which == 0)
                fma_probe<<<blocks, threads, 0, st>>>(iters_fma, 0.999f, 1e-3f, sink);
            else if (which == 1)
                fma2_probe<<<blocks, threads, 0, st>>>(iters_fma, 0.999f, 1e-3f, sink);
            else
                ex2_probe<<<blocks, threads, 0, st>>>(iters_ex2, sink);
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double lanes = static_cast<double>(blocks) * threads * kChains;
            if (which < 2)  // FLOP/s: 2 per FMA
                res[which] = lanes * iters_fma * 2.0 / (ms * 1e-3);
            else            // ex2 per second
                res[which] = lanes * iters_ex2 / (ms * 1e-3);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    for (int i = 0; i < 3; ++i) out3[i] = res[i];
    return e;
}

}  // namespace wrf
