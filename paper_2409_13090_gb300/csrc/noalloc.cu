// Allocation-free residual and backward error.
//
// Some applications cannot let a library allocate device memory at the time
// of a call: they hand all device memory to their own pool up front, or they
// run latency-critical loops in which a cudaMalloc (which may synchronise the
// whole device) is not acceptable. sc_residual_eta_noalloc serves them: it
// computes R = B - A X and the backward error of each column with the same
// arithmetic as the check inside sc_solve, but the only working memory it uses
// is the fixed-size array below, which every GPU that loads this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/sc.h"

namespace {

// Working memory: per right-hand side the maxima |r|, |x|, |b|, then ||A||_inf.
// 3 * SC_NOALLOC_MAX_RHS + 1 doubles (about 24 KB).
static __device__ __align__(256) double g_noalloc_scratch[3 * SC_NOALLOC_MAX_RHS + 1];

// max of two non-negative values or NaNs (a NaN wins)
__device__ inline double nan_max(double a, double b) { return (a != a || a > b) ? a : b; }

// atomic maximum of non-negative doubles (and NaNs with the sign bit clear) by
// their bit patterns, which order like the values
__device__ inline void atomic_max_nonneg(double *addr, double v) {
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_na_clear(double *scratch, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) scratch[i] = 0.0;
}

__global__ void k_na_anorm(const int64_t *__restrict__ ptr, const double *__restrict__ val, int64_t n,
                           double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t p = ptr[i]; p < ptr[i + 1]; p++) s += fabs(val[p]);
    atomic_max_nonneg(out, s);
}

__global__ void k_na_residual(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const double *__restrict__ val, int64_t n, const double *__restrict__ B, int64_t ldb,
                              const double *__restrict__ X, int64_t ldx, double *__restrict__ R, int64_t ldr,
                              double *__restrict__ red) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    const double *x = X + (int64_t)c * ldx;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    if (i < n) {  // every lane stays for the warp-wide reduction below
        double b = B[(int64_t)c * ldb + i];
        double s = b;
        for (int64_t p = ptr[i]; p < ptr[i + 1]; p++) s -= val[p] * x[col[p]];
        R[(int64_t)c * ldr + i] = s;
        m0 = fabs(s);
        m1 = fabs(x[i]);
        m2 = fabs(b);
    }
    // maxima over the warp first (one atomic per warp and value, not per row);
    // fmax would drop a NaN, so a NaN is carried as itself: its bit pattern with
    // the sign cleared is above every finite value and +inf in atomicMax's order
    for (int o = 16; o > 0; o >>= 1) {
        m0 = nan_max(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = nan_max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = nan_max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(red + 3 * c, m0);
        atomic_max_nonneg(red + 3 * c + 1, m1);
        atomic_max_nonneg(red + 3 * c + 2, m2);
    }
}

// eta per column; not finite (NaN) when a residual, an entry of X or B, or
// ||A|| is not finite, so a caller's "eta <= tol" test never passes on it
__global__ void k_na_eta(const double *__restrict__ red, int nrhs, double *__restrict__ eta) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    const double anorm = red[3 * SC_NOALLOC_MAX_RHS];
    const double r = red[3 * c], den = anorm * red[3 * c + 1] + red[3 * c + 2];
    if (!isfinite(r) || !isfinite(den)) eta[c] = NAN;
    else eta[c] = den > 0.0 ? r / den : (r == 0.0 ? 0.0 : INFINITY);
}

// Device address of the scratch array for the current device, looked up on
// every call with the device current (a module reloaded after a device reset
// is found at its new address), except while the stream is being captured:
// then the address of the last lookup on this device is reused, so the first
// call on a device has to come before any capture.
constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(cudaStream_t st, double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SC_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SC_ERR_CUDA;
        g_scratch_addr[dev] = (double *)p;
    } else if (!g_scratch_addr[dev]) {
        return SC_ERR_CUDA;  // first call on this device inside a capture: no address known yet
    }
    *out = g_scratch_addr[dev];
    return SC_OK;
}

}  // namespace

extern "C" int sc_residual_eta_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                                       int64_t nrhs, const double *B, int64_t ldb, const double *X, int64_t ldx,
                                       double *R, int64_t ldr, double *eta, void *cuda_stream) {
    if (n < 1) return -1;
    if (!row_ptr) return -2;
    if (!col) return -3;
    if (!val) return -4;
    if (nrhs < 1 || nrhs > SC_NOALLOC_MAX_RHS) return -5;
    if (!B) return -6;
    if (ldb < n) return -7;
    if (!X) return -8;
    if (ldx < n) return -9;
    if (!R) return -10;
    if (ldr < n) return -11;
    if (!eta) return -12;
    double *scratch = nullptr;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = scratch_for_current_device(st, &scratch);
    if (rc) return rc;
    // every call starts from zeroed maxima: the array keeps the previous call's values
    k_na_clear<<<(3 * SC_NOALLOC_MAX_RHS + 1 + 255) / 256, 256, 0, st>>>(scratch, 3 * SC_NOALLOC_MAX_RHS + 1);
    k_na_anorm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(row_ptr, val, n, scratch + 3 * SC_NOALLOC_MAX_RHS);
    k_na_residual<<<dim3((unsigned)((n + 255) / 256), (unsigned)nrhs), 256, 0, st>>>(row_ptr, col, val, n, B, ldb, X,
                                                                                      ldx, R, ldr, scratch);
    k_na_eta<<<(unsigned)((nrhs + 255) / 256), 256, 0, st>>>(scratch, (int)nrhs, eta);
    return cudaGetLastError() == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}
