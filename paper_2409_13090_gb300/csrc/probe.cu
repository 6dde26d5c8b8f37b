// Measured arithmetic peaks of the current GPU (FMA throughput), used as the
// roofline denominator of the SIMT kernels. The timed body is the inner step
// of an outer-product tile: every thread keeps NA x NB accumulators acc[i][j]
// and adds a[i] * b[j] into them, 16 independent FMAs per loop trip. Three
// shapes (4 x 4, 2 x 8, 1 x 8 with 8 per trip) are timed at the occupancy the
// compiler's register use allows (whole waves), each best of three CUDA-event
// timings of about 0.1 s; FLOP/s = 2 * FMAs / time, the best value is
// reported. The register allocation of a given body can cost a sixth of the
// FP64 rate, which is why several bodies are tried.
#include <cuda_runtime.h>

#include "../../include/sc.h"

namespace {

template <typename T, int NA, int NB>
__global__ void __launch_bounds__(256) k_fma_tile(T *sink, int iters) {
    T a[NA], b[NB], acc[NA][NB];
#pragma unroll
    for (int i = 0; i < NA; i++) a[i] = (T)1e-3 * (T)(1 + i + threadIdx.x % 5);
#pragma unroll
    for (int j = 0; j < NB; j++) b[j] = (T)1e-3 * (T)(2 + j + threadIdx.x % 7);
#pragma unroll
    for (int i = 0; i < NA; i++)
#pragma unroll
        for (int j = 0; j < NB; j++) acc[i][j] = (T)0;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < NA; i++)
#pragma unroll
            for (int j = 0; j < NB; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < NA; i++)
#pragma unroll
        for (int j = 0; j < NB; j++) s += acc[i][j];
    if (s == (T)-12345.0) sink[blockIdx.x] = s;  // keeps the accumulators alive
}

// best FLOP/s of one body at its full occupancy (at most 8 CTAs per SM)
template <typename T, int NA, int NB>
int time_body(cudaStream_t st, int sms, T *sink, double fmas_per_thread, double *best) {
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_tile<T, NA, NB>, 256, 0) != cudaSuccess ||
        occ < 1)
        return SC_ERR_CUDA;
    occ = occ > 8 ? 8 : occ;
    const int blocks = sms * occ;
    // the same number of FMAs per SM at every occupancy: about the same time
    const int iters = (int)(fmas_per_thread * 8 / occ / (NA * NB));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SC_OK;
    k_fma_tile<T, NA, NB><<<blocks, 256, 0, st>>>(sink, iters / 8);  // untimed: clocks leave idle
    for (int rep = 0; rep < 3; rep++) {
        cudaEventRecord(e0, st);
        k_fma_tile<T, NA, NB><<<blocks, 256, 0, st>>>(sink, iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = SC_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double f = 2.0 * NA * NB * (double)iters * blocks * 256 / (ms * 1e-3);
        if (f > *best) *best = f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

template <typename T>
int probe(cudaStream_t st, double fmas_per_thread, double *out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SC_ERR_CUDA;
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * sms * 8) != cudaSuccess) return SC_ERR_OOM;
    double best = 0.0;
    int rc = time_body<T, 4, 4>(st, sms, sink, fmas_per_thread, &best);
    if (!rc) rc = time_body<T, 2, 8>(st, sms, sink, fmas_per_thread, &best);
    if (!rc) rc = time_body<T, 1, 8>(st, sms, sink, fmas_per_thread, &best);
    cudaFree(sink);
    if (rc) return rc;
    *out = best;
    return SC_OK;
}

}  // namespace

extern "C" int sc_probe_fma_peak(int kind, void *cuda_stream, double *flops_per_s) {
    if (kind != 0 && kind != 1) return -1;
    if (!flops_per_s) return -3;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // FMAs per thread at 8 CTAs of 256 threads per SM (scaled to the occupancy): FP64 2e5 x 311,296
    // threads = 6e10 FMAs, ~0.1 s at ~1.25 TFLOP/s; FP32 1e7 x 311,296 = 3e12 FMAs, ~0.08 s
    return kind == 0 ? probe<double>(st, 2.0e5, flops_per_s) : probe<float>(st, 1.0e7, flops_per_s);
}
