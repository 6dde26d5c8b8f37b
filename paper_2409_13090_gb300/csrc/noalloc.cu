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
    if (i >= n) return;
    const double *x = X + (int64_t)c * ldx;
    double b = B[(int64_t)c * ldb + i];
    double s = b;
    for (int64_t p = ptr[i]; p < ptr[i + 1]; p++) s -= val[p] * x[col[p]];
    R[(int64_t)c * ldr + i] = s;
    atomic_max_nonneg(red + 3 * c, fabs(s));
    atomic_max_nonneg(red + 3 * c + 1, fabs(x[i]));
    atomic_max_nonneg(red + 3 * c + 2, fabs(b));
}

__global__ void k_na_eta(const double *__restrict__ red, int nrhs, double *__restrict__ eta) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double anorm = red[3 * SC_NOALLOC_MAX_RHS];
    double den = anorm * red[3 * c + 1] + red[3 * c + 2];
    eta[c] = den > 0.0 ? red[3 * c] / den : 0.0;
}

// Device address of the scratch array, looked up once per device (with that
// device current) and kept for the life of the process.
constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SC_ERR_CUDA;
        g_scratch_addr[dev] = (double *)p;
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
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // every call starts from zeroed maxima: the array keeps the previous call's values
    k_na_clear<<<(3 * SC_NOALLOC_MAX_RHS + 1 + 255) / 256, 256, 0, st>>>(scratch, 3 * SC_NOALLOC_MAX_RHS + 1);
    k_na_anorm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(row_ptr, val, n, scratch + 3 * SC_NOALLOC_MAX_RHS);
    k_na_residual<<<dim3((unsigned)((n + 255) / 256), (unsigned)nrhs), 256, 0, st>>>(row_ptr, col, val, n, B, ldb, X,
                                                                                      ldx, R, ldr, scratch);
    k_na_eta<<<(unsigned)((nrhs + 255) / 256), 256, 0, st>>>(scratch, (int)nrhs, eta);
    return cudaGetLastError() == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}
