// Measured arithmetic peaks of the current GPU (FMA throughput), used as the
// roofline denominator of the SIMT kernels: every thread runs 8 independent
// FMA chains; FLOP/s = 2 * FMAs / (CUDA-event time of the kernel).
#include <cuda_runtime.h>

#include "../../include/sc.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *sink, int iters, T seed) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = seed + (T)(threadIdx.x + i);
    const T b = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = a[i] * b + c;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += a[i];
    if (s == (T)-12345.0) sink[blockIdx.x] = s;  // keeps the chains alive
}

template <typename T>
int probe(cudaStream_t st, int iters, double *out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SC_ERR_CUDA;
    T *sink = nullptr;
    int blocks = sms * 8;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return SC_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 3; rep++) {
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<blocks, 256, 0, st>>>(sink, iters, (T)1.0);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaFree(sink);
            return SC_ERR_CUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double f = 2.0 * 8.0 * (double)iters * blocks * 256 / (ms * 1e-3);
        if (f > best) best = f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    *out = best;
    return SC_OK;
}

}  // namespace

extern "C" int sc_probe_fma_peak(int kind, void *cuda_stream, double *flops_per_s) {
    if (kind != 0 && kind != 1) return -1;
    if (!flops_per_s) return -3;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return kind == 0 ? probe<double>(st, 20000, flops_per_s) : probe<float>(st, 400000, flops_per_s);
}
