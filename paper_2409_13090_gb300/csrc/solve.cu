// Triangular solves and iterative refinement of libsc (Sec. 1 step 4).
//
// Work vectors are kept in the final ordering, row-major n x nb (nb right-hand
// sides of one block), in the storage precision of the factor.
//   forward  (levels ascending):  y_c = L_cc^{-1} x_c ; x_rows -= L_{rows,c} y_c
//   backward (levels descending): z_c = L_cc^{-T} (y_c - L_{rows,c}^T z_rows)
// where c runs over the chunks of a level and rows over the panel rows below
// the chunk (global row = glbind(J)[row]). Each sweep is one persistent launch:
// CTAs take row tiles in level order (reverse order backward) and wait on
// per-chunk counters instead of a barrier per level. The backward gather of a
// chunk is spread over row tiles; the last tile to finish (per-chunk counter
// after a memory fence) applies the diagonal solve and marks the chunk done.
// Refinement: r = b - A x in FP64 on the caller's matrix (CSR), then
//   eta = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) per column, and
//   x += solve(r) until eta <= ir_tol.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "numeric.h"

namespace sc {

#define SC_CUDA(x)                                  \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return SC_ERR_CUDA;  \
    } while (0)

namespace {

constexpr int kRhsBlk = 64;  // right-hand sides of one block: one sweep unit covers all of them
constexpr int kSolveRows = 64;
// one synchronisation word per 128-byte line: the CTAs that poll one chunk's
// word do not contend with arrivals at its neighbours
constexpr int kSyncStride = 32;
// synchronisation words per chunk and block of right-hand sides: forward
// arrivals, forward "y_c published", backward tile count, backward "z_c done"
constexpr int kSyncWords = 4;

// row stride (elements) of the shared-memory right-hand-side tiles of a block
// of nb right-hand sides: a multiple of 4, so 16-byte vector loads stay aligned
__host__ __device__ constexpr int rhs_ld(int nb) { return (nb + 3) / 4 * 4; }

// right-hand sides per thread in the block products (four thread groups share
// the block's right-hand sides): 1, 2, 4, 8 or 16
inline int rhs_per_thread(int nb) {
    const int q = (nb + 3) / 4;
    return q <= 1 ? 1 : q <= 2 ? 2 : q <= 4 ? 4 : q <= 8 ? 8 : 16;
}

// dynamic shared memory of a sweep CTA for blocks of nb right-hand sides: the
// diagonal block (or its inverse) and the tile's rows of L (64 x 65 each), then
// two 64 x rhs_ld(nb) right-hand-side tiles (also the per-warp slices of the
// narrow-tile path: 8 warps x kSmallW rows)
template <typename T>
size_t solve_smem(int nb) {
    // + 16 elements: a product thread's 16-byte loads of b may run up to 15
    // elements past its row's last right-hand side (those values are not used)
    return sizeof(T) * (2 * (size_t)kMaxChunk * (kMaxChunk + 1) + 2 * (size_t)kMaxChunk * rhs_ld(nb) + 16);
}

// Loads a rows x w block (row stride ld) into shared memory dst[r][c] with a
// fixed trip count per thread, so every thread keeps all of its loads in flight.
template <typename T>
__device__ __forceinline__ void stage_block(T (*dst)[kMaxChunk + 1], const T *__restrict__ src, int64_t ld, int rows,
                                            int w) {
    constexpr int kIters = kMaxChunk * kMaxChunk / 256;
    T tmp[kIters];
#pragma unroll
    for (int it = 0; it < kIters; it++) {
        const int idx = threadIdx.x + it * 256;
        const int r = idx / kMaxChunk, c = idx % kMaxChunk;
        tmp[it] = (r < rows && c < w) ? src[(int64_t)r * ld + c] : T(0);
    }
#pragma unroll
    for (int it = 0; it < kIters; it++) {
        const int idx = threadIdx.x + it * 256;
        dst[idx / kMaxChunk][idx % kMaxChunk] = tmp[it];
    }
}

// Loads rows x nb values of a row-major vector block (row r at src + row(r) * nb,
// read through L2: other CTAs wrote them) into dst[r][0..nb) (row stride ldv).
// Rows of a whole number of 16-byte pieces go through cp.async.cg (L2 only,
// every copy in flight at once, no registers); each thread waits for its own
// copies and the caller's __syncthreads() makes them visible to the CTA. Other
// widths are loaded directly.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void stage_rhs_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T, typename RowOf>
__device__ __forceinline__ void stage_rhs(T *__restrict__ dst, int ldv, const T *src, int nb, int rows,
                                          RowOf row_of) {
    if ((nb * (int)sizeof(T)) % 16 == 0) {
        const int per_row = nb * (int)sizeof(T) / 16, total = rows * per_row;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = idx / per_row, q = idx % per_row;
            cp_async16(reinterpret_cast<unsigned char *>(dst + r * ldv) + 16 * q,
                       reinterpret_cast<const unsigned char *>(src + (int64_t)row_of(r) * nb) + 16 * q);
        }
        stage_rhs_wait();
        return;
    }
    for (int idx = threadIdx.x; idx < rows * nb; idx += blockDim.x) {
        const int r = idx / nb, c = idx % nb;
        dst[r * ldv + c] = __ldcg(src + (int64_t)row_of(r) * nb + c);
    }
}

// x_perm[k][r] = B[perm[k]][r0 + r]
template <typename T>
__global__ void k_perm_in(T *__restrict__ x, const double *__restrict__ B, int64_t ldb, const int32_t *__restrict__ perm,
                          int64_t n, int nb, int r0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nb) return;
    int64_t k = i / nb;
    int r = (int)(i % nb);
    x[i] = (T)B[(int64_t)(r0 + r) * ldb + perm[k]];
}

// X[perm[k]][r0 + r] (+)= z_perm[k][r]
template <typename T>
__global__ void k_perm_out(double *__restrict__ X, int64_t ldx, const T *__restrict__ z, const int32_t *__restrict__ perm,
                           int64_t n, int nb, int r0, int add) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nb) return;
    int64_t k = i / nb;
    int r = (int)(i % nb);
    double *dst = X + (int64_t)(r0 + r) * ldx + perm[k];
    *dst = add ? *dst + (double)z[i] : (double)z[i];
}

// Stages the chunk's diagonal block L_cc and its reciprocal pivots, then scales
// it for division-free substitution: scale_cols: l[j][k] = L_jk / L_kk (j > k,
// forward); otherwise l[k][j] = L_kj / L_kk (j < k, backward).
template <typename T>
__device__ void load_diag(T (*l)[kMaxChunk + 1], T *rinv, const T *lnz, const ChunkDev &ch, bool scale_cols) {
    stage_block(l, lnz + ch.off + (int64_t)ch.c0 * ch.ld + ch.c0, ch.ld, ch.w, ch.w);
    __syncthreads();
    if (threadIdx.x < ch.w) rinv[threadIdx.x] = T(1) / l[threadIdx.x][threadIdx.x];
    __syncthreads();
    for (int idx = threadIdx.x; idx < ch.w * ch.w; idx += blockDim.x) {
        const int r = idx / ch.w, c = idx % ch.w;
        if (r > c) l[r][c] *= scale_cols ? rinv[c] : rinv[r];
    }
    __syncthreads();
}

// v[0..w) of one right-hand side held by a warp (lane i: entries i and i+32).
// Forward substitution on the numerators u_k = x_k - sum_{q<k} L_kq v_q with
// the column-scaled block M_jk = L_jk / L_kk: u_j -= M_jk u_k; then v = u / L_kk.
// Each step's critical path is one shuffle and one FMA.
template <typename T>
__device__ void warp_lower_solve(const T (*m)[kMaxChunk + 1], const T *rinv, int w, T &x0, T &x1) {
    const int lane = threadIdx.x % 32;
    for (int k = 0; k < w; k++) {
        const T uk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31);
        if (lane > k) x0 -= m[lane][k] * uk;
        if (lane + 32 > k && lane + 32 < w) x1 -= m[lane + 32][k] * uk;
    }
    if (lane < w) x0 *= rinv[lane];
    if (lane + 32 < w) x1 *= rinv[lane + 32];
}

// Backward substitution with L_cc^T on numerators, row-scaled block
// M_kj = L_kj / L_kk: for k = w-1..0: t_j -= M_kj t_k (j < k); then z = t / L_kk.
template <typename T>
__device__ void warp_upper_solve(const T (*m)[kMaxChunk + 1], const T *rinv, int w, T &x0, T &x1) {
    const int lane = threadIdx.x % 32;
    for (int k = w - 1; k >= 0; k--) {
        const T tk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31);
        if (lane < k) x0 -= m[k][lane] * tk;
        if (lane + 32 < k) x1 -= m[k][lane + 32] * tk;
    }
    if (lane < w) x0 *= rinv[lane];
    if (lane + 32 < w) x1 *= rinv[lane + 32];
}

// Thread mapping of the sweeps' block products (256 threads over a 64-row
// block and up to 64 right-hand sides): NR rows per thread, from i, R
// right-hand sides per row from r0. FP32 blocks of more than 16 right-hand
// sides take two rows (i and i + 32) of 8 or 4 right-hand sides: the rows share
// the thread's loads of b, 4 shared-memory wavefronts per 16 multiply-adds
// instead of 5; otherwise one row i of RPT right-hand sides.
template <typename T, int RPT>
struct RhsMap {
    static constexpr int NR = (sizeof(T) == 4 && RPT >= 8) ? 2 : 1;
    static constexpr int R = RPT / NR;
    static constexpr int kStep = kMaxChunk / NR;
    int i, r0;
    __device__ __forceinline__ RhsMap() : i((int)threadIdx.x % kStep), r0(((int)threadIdx.x / kStep) * R) {}
    __device__ __forceinline__ int row(int h) const { return i + h * kStep; }
};

// Block product of the sweeps, register-blocked over rows and right-hand
// sides: o[h][j] = sum_{k < K} a(row(h), k) b[k][r0 + j], with a(r, k) = a[r][k]
// (or a[k][r] when kTrans) and b of row stride ldb. A warp reads a at
// consecutive banks and b as broadcast 16-byte words (FP32, R a multiple of 4)
// or 16-byte pairs (FP64, R even). Rows past the caller's range are formed from
// whatever the buffer holds and not used. rhs_product_acc adds into o;
// rhs_product overwrites it.
template <typename T, int RPT, bool kTrans>
__device__ __forceinline__ void rhs_product_acc(const T (*a)[kMaxChunk + 1], const T *__restrict__ b, int ldb,
                                                const RhsMap<T, RPT> &m, int K,
                                                T (&o)[RhsMap<T, RPT>::NR][RhsMap<T, RPT>::R]) {
    constexpr int NR = RhsMap<T, RPT>::NR, R = RhsMap<T, RPT>::R;
#pragma unroll 4
    for (int k = 0; k < K; k++) {
        T av[NR];
#pragma unroll
        for (int h = 0; h < NR; h++) av[h] = kTrans ? a[k][m.row(h)] : a[m.row(h)][k];
        const T *bk = b + k * ldb + m.r0;
        if constexpr (sizeof(T) == 4 && R % 4 == 0) {
#pragma unroll
            for (int j = 0; j < R; j += 4) {
                const float4 bv = *reinterpret_cast<const float4 *>(bk + j);
#pragma unroll
                for (int h = 0; h < NR; h++) {
                    o[h][j] += av[h] * bv.x;
                    o[h][j + 1] += av[h] * bv.y;
                    o[h][j + 2] += av[h] * bv.z;
                    o[h][j + 3] += av[h] * bv.w;
                }
            }
        } else if constexpr (sizeof(T) == 8 && R % 2 == 0) {
#pragma unroll
            for (int j = 0; j < R; j += 2) {
                const double2 bv = *reinterpret_cast<const double2 *>(bk + j);
#pragma unroll
                for (int h = 0; h < NR; h++) {
                    o[h][j] += av[h] * bv.x;
                    o[h][j + 1] += av[h] * bv.y;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < R; j++) {
                const T bj = bk[j];
#pragma unroll
                for (int h = 0; h < NR; h++) o[h][j] += av[h] * bj;
            }
        }
    }
}

template <typename T, int RPT, bool kTrans>
__device__ __forceinline__ void rhs_product(const T (*a)[kMaxChunk + 1], const T *__restrict__ b, int ldb,
                                            const RhsMap<T, RPT> &m, int K,
                                            T (&o)[RhsMap<T, RPT>::NR][RhsMap<T, RPT>::R]) {
#pragma unroll
    for (int h = 0; h < RhsMap<T, RPT>::NR; h++)
#pragma unroll
        for (int j = 0; j < RhsMap<T, RPT>::R; j++) o[h][j] = T(0);
    rhs_product_acc<T, RPT, kTrans>(a, b, ldb, m, K, o);
}

// Reductions into global memory that return nothing (red): the issuing thread
// does not wait for them; the fence before a release orders them.
__device__ __forceinline__ void red_add(float *p, float a) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(a) : "memory");
}
__device__ __forceinline__ void red_add(double *p, double a) {
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(a) : "memory");
}
__device__ __forceinline__ void red_add4(float *p, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// dst[0..RPT) += sign * o over the valid right-hand sides r0 + j < nb, by
// reductions (16-byte vector reductions where the four values are valid and aligned)
template <typename T, int RPT>
__device__ __forceinline__ void add_rhs(T *dst, const T (&o)[RPT], T sign, int r0, int nb) {
    if constexpr (sizeof(T) == 4 && RPT % 4 == 0) {
        if ((nb & 3) == 0) {
#pragma unroll
            for (int j = 0; j < RPT; j += 4)
                if (r0 + j < nb) red_add4(dst + j, sign * o[j], sign * o[j + 1], sign * o[j + 2], sign * o[j + 3]);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < RPT; j++)
        if (r0 + j < nb) red_add(dst + j, sign * o[j]);
}

// Bounded wait until *flag >= target (acquire at GPU scope). Gives up, setting
// *err to `code`, after spin_limit polls, or at once when another CTA has
// already given up.
__device__ bool wait_flag(const int32_t *flag, int32_t target, int32_t *err, long long spin_limit, int code) {
    for (long long i = 0; i < spin_limit; i++) {
        int32_t v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v >= target) return true;
        if (*(volatile int32_t *)err) return false;
        if (i > 64) __nanosleep(32);
    }
    atomicCAS(err, 0, code);
    return false;
}

// next tile index of a sweep for this CTA (broadcast through shared memory);
// `total` once the sweep is done or a wait has given up
__device__ __forceinline__ int grab_tile(int32_t *work, int total, int32_t *err, int *slot) {
    if (threadIdx.x == 0) *slot = *(volatile int32_t *)err ? total : atomicAdd(work, 1);
    __syncthreads();
    return *slot;
}

// ---- tiles of narrow chunks (w <= kSmallW): one warp per tile, eight per CTA
// (a SolveUnit with cnt > 0). v / z of the diagonal step are kept in a
// per-warp shared-memory slice of kSmallW rows of ldv values.
constexpr int kSmallW = 16;

// Forward step of one narrow tile by one warp: wait for the chunk's arrivals,
// v = L_cc^{-1} x_c (stored FP32 inverse, or substitution per right-hand side
// in FP64), subtract L_{rows,c} v from x, count the arrivals. false when a wait
// gave up.
template <typename T>
__device__ bool fwd_tile_warp(const T *__restrict__ lnz, const ChunkDev &ch, const TrsmTile &tl, int t,
                              const int32_t *__restrict__ dep_ptr, const int32_t *__restrict__ dep,
                              const int32_t *__restrict__ need, const int32_t *__restrict__ glbind, T *__restrict__ x,
                              T *__restrict__ y, int nb, const float *__restrict__ inv, int32_t *__restrict__ arrive,
                              int32_t *__restrict__ err, long long spin_limit, T *vw, int ldv) {
    const int lane = threadIdx.x % 32, w = ch.w;
    const bool first = tl.r0 == ch.c0 + w;
    const int rows = max(0, min(kSolveRows, ch.m - tl.r0));
    int ok = 1;
    if (lane == 0) ok = wait_flag(arrive + (int64_t)tl.chunk * kSyncStride, need[tl.chunk], err, spin_limit, 5);
    if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
    const T *dg = lnz + ch.off + (int64_t)ch.c0 * ch.ld + ch.c0;
    if constexpr (sizeof(T) == 4) {
        const float *iv = inv + ch.inv;
        for (int e = lane; e < w * nb; e += 32) {
            const int k = e / nb, r = e % nb;
            T acc = T(0);
            for (int q = 0; q <= k; q++) acc += iv[k * w + q] * __ldcg(x + (int64_t)(ch.col0 + q) * nb + r);
            vw[k * ldv + r] = acc;
            if (first) y[(int64_t)(ch.col0 + k) * nb + r] = acc;
        }
    } else {
        for (int r = lane; r < nb; r += 32) {
            for (int k = 0; k < w; k++) {
                T sum = __ldcg(x + (int64_t)(ch.col0 + k) * nb + r);
                for (int q = 0; q < k; q++) sum -= dg[(int64_t)k * ch.ld + q] * vw[q * ldv + r];
                vw[k * ldv + r] = sum / dg[(int64_t)k * ch.ld + k];
                if (first) y[(int64_t)(ch.col0 + k) * nb + r] = vw[k * ldv + r];
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < rows * nb; e += 32) {
        const int i = e / nb, r = e % nb;
        const T *lr = lnz + ch.off + (int64_t)(tl.r0 + i) * ch.ld + ch.c0;
        T acc = T(0);
        for (int k = 0; k < w; k++) acc += lr[k] * vw[k * ldv + r];
        red_add(x + (int64_t)glbind[ch.gl + tl.r0 + i] * nb + r, -acc);
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        for (int p = dep_ptr[t]; p < dep_ptr[t + 1]; p++) atomicAdd(arrive + (int64_t)dep[p] * kSyncStride, 1);
    }
    __syncwarp();
    return true;
}

// Backward step of one narrow tile by one warp: wait until z is final in the
// chunks its rows fall in, add L_{rows,c}^T z_rows into acc_c, and when it is
// the chunk's last tile, z_c = L_cc^{-T} (y_c - acc_c) and mark the chunk done.
template <typename T>
__device__ bool bwd_tile_warp(const T *__restrict__ lnz, const ChunkDev &ch, const TrsmTile &tl, int t,
                              const int32_t *__restrict__ dep_ptr, const int32_t *__restrict__ dep,
                              const int32_t *__restrict__ ntiles, const int32_t *__restrict__ glbind,
                              const T *__restrict__ y, T *__restrict__ z, T *__restrict__ acc, int nb,
                              const float *__restrict__ inv, int32_t *__restrict__ cnt, int32_t *__restrict__ done,
                              int32_t *__restrict__ err, long long spin_limit, T *vw, int ldv) {
    const int lane = threadIdx.x % 32, w = ch.w;
    const int rows = max(0, min(kSolveRows, ch.m - tl.r0));
    if (rows > 0) {
        int ok = 1;
        if (lane == 0)
            for (int p = dep_ptr[t]; p < dep_ptr[t + 1] && ok; p++)
                ok = wait_flag(done + (int64_t)dep[p] * kSyncStride, 1, err, spin_limit, 6);
        if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
        for (int e = lane; e < w * nb; e += 32) {
            const int k = e / nb, r = e % nb;
            T sum = T(0);
            for (int i = 0; i < rows; i++)
                sum += lnz[ch.off + (int64_t)(tl.r0 + i) * ch.ld + ch.c0 + k] *
                       __ldcg(z + (int64_t)glbind[ch.gl + tl.r0 + i] * nb + r);
            red_add(acc + (int64_t)(ch.col0 + k) * nb + r, sum);
        }
    }
    __syncwarp();
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(cnt + (int64_t)tl.chunk * kSyncStride, 1) == ntiles[tl.chunk] - 1;
        if (last) __threadfence();
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return true;
    const T *dg = lnz + ch.off + (int64_t)ch.c0 * ch.ld + ch.c0;
    for (int e = lane; e < w * nb; e += 32) {
        const int k = e / nb, r = e % nb;
        const int64_t g = (int64_t)(ch.col0 + k) * nb + r;
        vw[k * ldv + r] = y[g] - __ldcg(acc + g);
    }
    __syncwarp();
    if constexpr (sizeof(T) == 4) {
        const float *iv = inv + ch.inv;
        for (int e = lane; e < w * nb; e += 32) {
            const int k = e / nb, r = e % nb;
            T sum = T(0);
            for (int q = k; q < w; q++) sum += iv[q * w + k] * vw[q * ldv + r];
            z[(int64_t)(ch.col0 + k) * nb + r] = sum;
        }
    } else {
        for (int r = lane; r < nb; r += 32) {
            for (int k = w - 1; k >= 0; k--) {
                T sum = vw[k * ldv + r];
                for (int q = k + 1; q < w; q++) sum -= dg[(int64_t)q * ch.ld + k] * vw[q * ldv + r];
                vw[k * ldv + r] = sum / dg[(int64_t)k * ch.ld + k];
                z[(int64_t)(ch.col0 + k) * nb + r] = vw[k * ldv + r];
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        atomicExch(done + (int64_t)tl.chunk * kSyncStride, 1);
    }
    __syncwarp();
    return true;
}

// Pointers of one sweep CTA's dynamic shared memory.
template <typename T>
struct SweepSmem {
    T (*l)[kMaxChunk + 1];   // diagonal block L_cc (or its FP32 inverse)
    T (*lr)[kMaxChunk + 1];  // the tile's rows of L
    T *v;                    // 64 x ldv: y_c (forward), z of the tile's rows (backward)
    T *xin;                  // 64 x ldv: x_c (forward), y_c - acc_c (backward)
    __device__ SweepSmem(unsigned char *raw, int ldv) {
        l = reinterpret_cast<T (*)[kMaxChunk + 1]>(raw);
        lr = l + kMaxChunk;
        v = reinterpret_cast<T *>(lr + kMaxChunk);
        xin = v + kMaxChunk * ldv;
    }
};

// Forward sweep: one persistent launch over all tiles in level order, every
// unit all right-hand sides of one block (up to kRhsBlk). A wide chunk's first
// tile waits until every tile that updates the chunk's rows of x has arrived,
// solves y_c = L_cc^{-1} x_c once (the stored FP32 inverse as a product, or
// FP64 substitution), writes y_c and publishes it (ready flag); the chunk's
// other tiles wait for that flag and read y_c. Every tile stages its rows of L
// before waiting, subtracts L_{rows,c} y_c from x (atomic adds: tiles of
// several chunks update the same rows) and counts one arrival at every chunk
// its rows fall in. A tile only waits for tiles taken earlier (lower levels,
// or its own chunk's first tile), so the sweep needs no co-residency.
template <typename T, int RPT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fwd(const T *__restrict__ lnz, const ChunkDev *__restrict__ chunks,
                                             const TrsmTile *__restrict__ tiles, const SolveUnit *__restrict__ units,
                                             int total, const int32_t *__restrict__ dep_ptr,
                                             const int32_t *__restrict__ dep, const int32_t *__restrict__ need,
                                             const int32_t *__restrict__ glbind, T *__restrict__ x0,
                                             T *__restrict__ y0, int nrhs, int64_t vstride,
                                             const float *__restrict__ inv, int32_t *__restrict__ arrive0,
                                             int32_t *__restrict__ ready0, int64_t sstride, int32_t *__restrict__ work,
                                             int32_t *__restrict__ err, long long spin_limit) {
    using Map = RhsMap<T, RPT>;
    extern __shared__ __align__(16) unsigned char smem_fwd[];
    const int ldv = rhs_ld(min(nrhs, kRhsBlk));
    SweepSmem<T> sm(smem_fwd, ldv);
    __shared__ T rinv[kMaxChunk];
    __shared__ int s_t, s_ok;
    const int nblk = (nrhs + kRhsBlk - 1) / kRhsBlk;
    for (;;) {
        const int ug = grab_tile(work, total, err, &s_t);
        if (ug >= total) break;
        // unit-major over the right-hand-side blocks: each block keeps its own order
        const int bk = ug % nblk;
        const SolveUnit su = units[ug / nblk];
        const int nb = min(kRhsBlk, nrhs - bk * kRhsBlk);
        T *x = x0 + bk * vstride, *y = y0 + bk * vstride;
        int32_t *arrive = arrive0 + bk * sstride, *ready = ready0 + bk * sstride;
        if (su.cnt > 0) {  // narrow tiles, one per warp
            const int wp = threadIdx.x / 32;
            if (wp < su.cnt) {
                const int t = su.t0 + wp;
                const TrsmTile tl = tiles[t];
                const ChunkDev ch = chunks[tl.chunk];
                fwd_tile_warp(lnz, ch, tl, t, dep_ptr, dep, need, glbind, x, y, nb, inv, arrive, err, spin_limit,
                              sm.v + wp * kSmallW * ldv, ldv);
            }
            __syncthreads();
            continue;
        }
        if (su.cnt < 0) {  // further tiles of one wide chunk: y_c staged once, tiles one after another
            const int g = -su.cnt;
            const ChunkDev ch = chunks[tiles[su.t0].chunk];
            const int w = ch.w;
            const int c = tiles[su.t0].chunk;
            {
                const TrsmTile tl = tiles[su.t0];
                stage_block(sm.lr, lnz + ch.off + (int64_t)tl.r0 * ch.ld + ch.c0, ch.ld,
                            max(0, min(kSolveRows, ch.m - tl.r0)), w);
            }
            if (threadIdx.x == 0) s_ok = wait_flag(ready + (int64_t)c * kSyncStride, 1, err, spin_limit, 7);
            __syncthreads();
            if (!s_ok) break;
            stage_rhs(sm.v, ldv, (const T *)y, nb, w, [&](int r) { return ch.col0 + r; });
            __syncthreads();
            const Map m;
            for (int q = 0; q < g; q++) {
                const int tq = su.t0 + q;
                const TrsmTile tl = tiles[tq];
                const int rows = max(0, min(kSolveRows, ch.m - tl.r0));
                if (q > 0) {
                    stage_block(sm.lr, lnz + ch.off + (int64_t)tl.r0 * ch.ld + ch.c0, ch.ld, rows, w);
                    __syncthreads();
                }
                if (m.row(0) < rows && m.r0 < nb) {
                    T o[Map::NR][Map::R];
                    rhs_product<T, RPT, false>(sm.lr, sm.v, ldv, m, w, o);
#pragma unroll
                    for (int h = 0; h < Map::NR; h++)
                        if (m.row(h) < rows)
                            add_rhs<T, Map::R>(x + (int64_t)glbind[ch.gl + tl.r0 + m.row(h)] * nb + m.r0, o[h], T(-1),
                                               m.r0, nb);
                }
                // each tile's arrivals go out as soon as its rows are updated: a later
                // chunk's step must not wait for the rest of the unit
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    for (int p = dep_ptr[tq]; p < dep_ptr[tq + 1]; p++) atomicAdd(arrive + (int64_t)dep[p] * kSyncStride, 1);
                }
            }
            continue;
        }
        const int t = su.t0;
        const TrsmTile tl = tiles[t];
        const ChunkDev ch = chunks[tl.chunk];
        const int w = ch.w;
        const bool first = tl.r0 == ch.c0 + w;  // the chunk's first tile solves and publishes y_c
        const int rows = max(0, min(kSolveRows, ch.m - tl.r0));
        // loads that need no other tile: the tile's rows of L (and the diagonal block)
        stage_block(sm.lr, lnz + ch.off + (int64_t)tl.r0 * ch.ld + ch.c0, ch.ld, rows, w);
        if (first) {
            if constexpr (sizeof(T) == 4) stage_block(sm.l, (const T *)(inv + ch.inv), w, w, w);
            else load_diag(sm.l, rinv, lnz, ch, true);
            if (threadIdx.x == 0)
                s_ok = wait_flag(arrive + (int64_t)tl.chunk * kSyncStride, need[tl.chunk], err, spin_limit, 5);
            __syncthreads();
            if (!s_ok) break;
            stage_rhs(sm.xin, ldv, x, nb, w, [&](int r) { return ch.col0 + r; });
            __syncthreads();
            if constexpr (sizeof(T) == 4) {
                // y_c = inv(L_cc) x_c: the block's stored inverse (zero above its diagonal)
                const Map m;
                if (m.row(0) < w && m.r0 < nb) {
                    T o[Map::NR][Map::R];
                    rhs_product<T, RPT, false>(sm.l, sm.xin, ldv, m, w, o);
#pragma unroll
                    for (int h = 0; h < Map::NR; h++) {
                        const int k = m.row(h);
#pragma unroll
                        for (int j = 0; j < Map::R; j++)
                            if (k < w && m.r0 + j < nb) {
                                sm.v[k * ldv + m.r0 + j] = o[h][j];
                                y[(int64_t)(ch.col0 + k) * nb + m.r0 + j] = o[h][j];
                            }
                    }
                }
            } else {
                const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
                for (int r = warp; r < nb; r += blockDim.x / 32) {
                    T u0 = lane < w ? sm.xin[lane * ldv + r] : T(0);
                    T u1 = lane + 32 < w ? sm.xin[(lane + 32) * ldv + r] : T(0);
                    warp_lower_solve(sm.l, rinv, w, u0, u1);
                    if (lane < w) {
                        sm.v[lane * ldv + r] = u0;
                        y[(int64_t)(ch.col0 + lane) * nb + r] = u0;
                    }
                    if (lane + 32 < w) {
                        sm.v[(lane + 32) * ldv + r] = u1;
                        y[(int64_t)(ch.col0 + lane + 32) * nb + r] = u1;
                    }
                }
            }
            __syncthreads();
            // y_c is published as soon as it is written: the chunk's other tiles start
            // while this one updates its own rows (the next chunk's, on the chain)
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(ready + (int64_t)tl.chunk * kSyncStride, 1);
            }
        } else {
            if (threadIdx.x == 0) s_ok = wait_flag(ready + (int64_t)tl.chunk * kSyncStride, 1, err, spin_limit, 7);
            __syncthreads();
            if (!s_ok) break;
            stage_rhs(sm.v, ldv, (const T *)y, nb, w, [&](int r) { return ch.col0 + r; });
            __syncthreads();
        }
        // x_rows -= L_{rows,c} y_c
        {
            const Map m;
            if (m.row(0) < rows && m.r0 < nb) {
                T o[Map::NR][Map::R];
                rhs_product<T, RPT, false>(sm.lr, sm.v, ldv, m, w, o);
#pragma unroll
                for (int h = 0; h < Map::NR; h++)
                    if (m.row(h) < rows)
                        add_rhs<T, Map::R>(x + (int64_t)glbind[ch.gl + tl.r0 + m.row(h)] * nb + m.r0, o[h], T(-1),
                                           m.r0, nb);
            }
        }
        // release: the barrier orders every thread's updates before thread 0's fence
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            for (int p = dep_ptr[t]; p < dep_ptr[t + 1]; p++) atomicAdd(arrive + (int64_t)dep[p] * kSyncStride, 1);
        }
    }
}

// Backward sweep: one persistent launch over all tiles in reverse level order,
// every unit all right-hand sides of one block. A tile stages its rows of L,
// waits until z is final in every chunk its rows fall in, and forms
// L_{rows,c}^T z_rows. For a wide chunk, every tile but the first adds it into
// acc_c and counts itself; the first tile (taken last: reverse order) keeps its
// own part, waits for the count, solves z_c = L_cc^{-T} (y_c - acc_c - own)
// and marks the chunk done. Narrow chunks' warp tiles add and count, and the
// last to finish solves.
template <typename T, int RPT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_bwd(const T *__restrict__ lnz, const ChunkDev *__restrict__ chunks,
                                             const TrsmTile *__restrict__ tiles, const SolveUnit *__restrict__ units,
                                             int total, const int32_t *__restrict__ dep_ptr,
                                             const int32_t *__restrict__ dep, const int32_t *__restrict__ ntiles,
                                             const int32_t *__restrict__ glbind, const T *__restrict__ y0,
                                             T *__restrict__ z0, T *__restrict__ acc0, int nrhs, int64_t vstride,
                                             const float *__restrict__ inv, int32_t *__restrict__ cnt0,
                                             int32_t *__restrict__ done0, int64_t sstride, int32_t *__restrict__ work,
                                             int32_t *__restrict__ err, long long spin_limit) {
    using Map = RhsMap<T, RPT>;
    extern __shared__ __align__(16) unsigned char smem_bwd[];
    const int ldv = rhs_ld(min(nrhs, kRhsBlk));
    SweepSmem<T> sm(smem_bwd, ldv);
    __shared__ T rinv[kMaxChunk];
    __shared__ int32_t grow[kSolveRows];
    __shared__ int s_t, s_ok;
    const int nblk = (nrhs + kRhsBlk - 1) / kRhsBlk;
    for (;;) {
        const int tr = grab_tile(work, total, err, &s_t);
        if (tr >= total) break;
        const int ug = total - 1 - tr;
        const int bk = ug % nblk;
        const SolveUnit su = units[ug / nblk];
        const int nb = min(kRhsBlk, nrhs - bk * kRhsBlk);
        const T *y = y0 + bk * vstride;
        T *z = z0 + bk * vstride, *acc = acc0 + bk * vstride;
        int32_t *cnt = cnt0 + bk * sstride, *done = done0 + bk * sstride;
        if (su.cnt > 0) {  // narrow tiles, one per warp
            const int wp = threadIdx.x / 32;
            if (wp < su.cnt) {
                const int t = su.t0 + wp;
                const TrsmTile tl = tiles[t];
                const ChunkDev ch = chunks[tl.chunk];
                bwd_tile_warp(lnz, ch, tl, t, dep_ptr, dep, ntiles, glbind, y, z, acc, nb, inv, cnt, done, err,
                              spin_limit, sm.v + wp * kSmallW * ldv, ldv);
            }
            __syncthreads();
            continue;
        }
        if (su.cnt < 0) {  // further tiles of one wide chunk: their parts summed in registers
            const int g = -su.cnt;
            const int c = tiles[su.t0].chunk;
            const ChunkDev ch = chunks[c];
            const int w = ch.w;
            if (threadIdx.x == 0) {
                bool ok = true;
                for (int p = dep_ptr[su.t0]; p < dep_ptr[su.t0 + g] && ok; p++)
                    ok = wait_flag(done + (int64_t)dep[p] * kSyncStride, 1, err, spin_limit, 6);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) break;
            const Map m;
            T o[Map::NR][Map::R];
#pragma unroll
            for (int h = 0; h < Map::NR; h++)
#pragma unroll
                for (int j = 0; j < Map::R; j++) o[h][j] = T(0);
            for (int q = 0; q < g; q++) {
                const TrsmTile tl = tiles[su.t0 + q];
                const int rows = max(0, min(kSolveRows, ch.m - tl.r0));
                if (q > 0) __syncthreads();  // the previous tile's L rows and z rows are no longer read
                if (threadIdx.x < rows) grow[threadIdx.x] = glbind[ch.gl + tl.r0 + threadIdx.x];
                stage_block(sm.lr, lnz + ch.off + (int64_t)tl.r0 * ch.ld + ch.c0, ch.ld, rows, w);
                __syncthreads();
                stage_rhs(sm.v, ldv, (const T *)z, nb, rows, [&](int r) { return grow[r]; });
                __syncthreads();
                if (m.row(0) < w && m.r0 < nb) rhs_product_acc<T, RPT, true>(sm.lr, sm.v, ldv, m, rows, o);
            }
            if (m.r0 < nb) {
#pragma unroll
                for (int h = 0; h < Map::NR; h++)
                    if (m.row(h) < w)
                        add_rhs<T, Map::R>(acc + (int64_t)(ch.col0 + m.row(h)) * nb + m.r0, o[h], T(1), m.r0, nb);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();  // release this unit's contributions
                atomicAdd(cnt + (int64_t)c * kSyncStride, g);
            }
            continue;
        }
        const int t = su.t0;
        const TrsmTile tl = tiles[t];
        const ChunkDev ch = chunks[tl.chunk];
        const int w = ch.w;
        // the chunk's first tile (rows just below the chunk) is taken after its other
        // tiles (reverse order) and solves for z_c; it stages the diagonal block
        // before it waits and keeps its own contribution in registers
        const bool first = tl.r0 == ch.c0 + w;
        const int rows = max(0, min(kSolveRows, ch.m - tl.r0));
        const Map m;
        T o[Map::NR][Map::R];
#pragma unroll
        for (int h = 0; h < Map::NR; h++)
#pragma unroll
            for (int j = 0; j < Map::R; j++) o[h][j] = T(0);
        if (first) {
            if constexpr (sizeof(T) == 4) stage_block(sm.l, (const T *)(inv + ch.inv), w, w, w);
            else load_diag(sm.l, rinv, lnz, ch, false);
        }
        if (rows > 0) {
            if (threadIdx.x < rows) grow[threadIdx.x] = glbind[ch.gl + tl.r0 + threadIdx.x];
            stage_block(sm.lr, lnz + ch.off + (int64_t)tl.r0 * ch.ld + ch.c0, ch.ld, rows, w);
            if (threadIdx.x == 0) {
                bool ok = true;
                for (int p = dep_ptr[t]; p < dep_ptr[t + 1] && ok; p++)
                    ok = wait_flag(done + (int64_t)dep[p] * kSyncStride, 1, err, spin_limit, 6);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) break;
            stage_rhs(sm.v, ldv, (const T *)z, nb, rows, [&](int r) { return grow[r]; });
            __syncthreads();
            // this tile's part of L_{S,c}^T z_S
            if (m.row(0) < w && m.r0 < nb) {
                rhs_product<T, RPT, true>(sm.lr, sm.v, ldv, m, rows, o);
                if (!first) {
#pragma unroll
                    for (int h = 0; h < Map::NR; h++)
                        if (m.row(h) < w)
                            add_rhs<T, Map::R>(acc + (int64_t)(ch.col0 + m.row(h)) * nb + m.r0, o[h], T(1), m.r0,
                                               nb);
                }
            }
        }
        if (!first) {
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();  // release this tile's contributions
                atomicAdd(cnt + (int64_t)tl.chunk * kSyncStride, 1);
            }
            continue;
        }
        // the chunk's other tiles have added theirs into acc_c
        if (threadIdx.x == 0)
            s_ok = ntiles[tl.chunk] <= 1 ||
                   wait_flag(cnt + (int64_t)tl.chunk * kSyncStride, ntiles[tl.chunk] - 1, err, spin_limit, 8);
        __syncthreads();
        if (!s_ok) break;
        // xin = y_c - acc_c - (own contribution)
        stage_rhs(sm.xin, ldv, y, nb, w, [&](int r) { return ch.col0 + r; });
        stage_rhs(sm.v, ldv, (const T *)acc, nb, w, [&](int r) { return ch.col0 + r; });
        __syncthreads();
        if (m.r0 < nb) {
#pragma unroll
            for (int h = 0; h < Map::NR; h++) {
                const int k = m.row(h);
#pragma unroll
                for (int j = 0; j < Map::R; j++)
                    if (k < w && m.r0 + j < nb) sm.xin[k * ldv + m.r0 + j] -= sm.v[k * ldv + m.r0 + j] + o[h][j];
            }
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            // z_c = inv(L_cc)^T (y_c - acc_c) with the block's stored inverse
            if (m.row(0) < w && m.r0 < nb) {
                T zo[Map::NR][Map::R];
                rhs_product<T, RPT, true>(sm.l, sm.xin, ldv, m, w, zo);
#pragma unroll
                for (int h = 0; h < Map::NR; h++) {
                    const int k = m.row(h);
#pragma unroll
                    for (int j = 0; j < Map::R; j++)
                        if (k < w && m.r0 + j < nb) z[(int64_t)(ch.col0 + k) * nb + m.r0 + j] = zo[h][j];
                }
            }
        } else {
            const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
            for (int r = warp; r < nb; r += blockDim.x / 32) {
                T u0 = lane < w ? sm.xin[lane * ldv + r] : T(0);
                T u1 = lane + 32 < w ? sm.xin[(lane + 32) * ldv + r] : T(0);
                warp_upper_solve(sm.l, rinv, w, u0, u1);
                if (lane < w) z[(int64_t)(ch.col0 + lane) * nb + r] = u0;
                if (lane + 32 < w) z[(int64_t)(ch.col0 + lane + 32) * nb + r] = u1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(done + (int64_t)tl.chunk * kSyncStride, 1);
        }
    }
}

__global__ void k_gather_vals(double *__restrict__ out, const double *__restrict__ values,
                              const int64_t *__restrict__ map, int64_t nnz) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nnz) out[i] = values[map[i]];
}

// atomic maximum of non-negative doubles by their bit patterns, which order
// like the values; a NaN with the sign bit clear orders above +inf, so it wins
__device__ inline void atomic_max_nonneg(double *addr, double v) {
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// max of two non-negative values or NaNs (a NaN wins: fmax would drop it)
__device__ inline double nan_max(double a, double b) { return (a != a || a > b) ? a : b; }

// Reductions of the vector kernels below: every kernel is grid-stride over the
// rows of one column (blockIdx.y), reduces its values over the block (warp
// shuffles, then the eight warp results through shared memory) and thread 0
// adds or maxes the block's value into the column's word, so a column's words
// take one atomic per block (a few dozen) instead of one per warp.
__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// block (256 threads) reduction of NV values; the result is valid in thread 0
template <int NV, bool kMax>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
    __shared__ double part[8][NV];
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
    for (int q = 0; q < NV; q++) v[q] = kMax ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; q++) part[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double r = part[0][q];
            for (int w = 1; w < 8; w++) r = kMax ? nan_max(r, part[w][q]) : r + part[w][q];
            v[q] = r;
        }
}

// ||A||_inf of the full symmetric matrix from its CSR
__global__ void __launch_bounds__(256) k_anorm(const int64_t *__restrict__ ptr, const double *__restrict__ val,
                                               int64_t n, double *out) {
    double m[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = ptr[i]; p < ptr[i + 1]; p++) s += fabs(val[p]);
        m[0] = nan_max(m[0], s);
    }
    block_reduce<1, true>(m);
    if (threadIdx.x == 0) atomic_max_nonneg(out, m[0]);
}

// r = b - A x (FP64), and per column: red[3c] = max|r|, red[3c+1] = max|x|, red[3c+2] = max|b|
__global__ void __launch_bounds__(256) k_residual(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                                  const double *__restrict__ val, const double *__restrict__ X,
                                                  const double *__restrict__ B, double *__restrict__ R, int64_t n,
                                                  int nrhs, double *__restrict__ red) {
    const int c = blockIdx.y;
    const double *x = X + (int64_t)c * n;
    double m[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double b = B[(int64_t)c * n + i];
        double s = b;
        for (int64_t p = ptr[i]; p < ptr[i + 1]; p++) s -= val[p] * x[col[p]];
        R[(int64_t)c * n + i] = s;
        m[0] = nan_max(m[0], fabs(s));
        m[1] = nan_max(m[1], fabs(x[i]));
        m[2] = nan_max(m[2], fabs(b));
    }
    block_reduce<3, true>(m);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(red + 3 * c, m[0]);
        atomic_max_nonneg(red + 3 * c + 1, m[1]);
        atomic_max_nonneg(red + 3 * c + 2, m[2]);
    }
}

// ---- conjugate gradients preconditioned by the factor (M = L L^T in the
// factor's precision, FP64 vectors), all right-hand sides at once; per-column
// scalars live on the device.

// Q = A P and pq[c] += P(:,c) . Q(:,c)
__global__ void __launch_bounds__(256) k_spmv_dot(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                                  const double *__restrict__ val, const double *__restrict__ P,
                                                  double *__restrict__ Q, int64_t n, double *__restrict__ pq) {
    const int c = blockIdx.y;
    const double *p = P + (int64_t)c * n;
    double d[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; e++) s += val[e] * p[col[e]];
        Q[(int64_t)c * n + i] = s;
        d[0] += p[i] * s;
    }
    block_reduce<1, false>(d);
    if (threadIdx.x == 0) atomicAdd(pq + c, d[0]);
}

// out[c] += X(:,c) . Y(:,c)
__global__ void __launch_bounds__(256) k_dot(const double *__restrict__ X, const double *__restrict__ Y, int64_t n,
                                             double *__restrict__ out) {
    const int c = blockIdx.y;
    double d[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[0] += X[(int64_t)c * n + i] * Y[(int64_t)c * n + i];
    block_reduce<1, false>(d);
    if (threadIdx.x == 0) atomicAdd(out + c, d[0]);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; maxima of |r|, |x|, |b| for eta
__global__ void __launch_bounds__(256) k_cg_step(double *__restrict__ X, double *__restrict__ R,
                                                 const double *__restrict__ P, const double *__restrict__ Q,
                                                 const double *__restrict__ B, const double *__restrict__ rz,
                                                 const double *__restrict__ pq, int64_t n, double *__restrict__ red) {
    const int c = blockIdx.y;
    const double a = pq[c] != 0.0 ? rz[c] / pq[c] : 0.0;
    double m[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = (int64_t)c * n + i;
        const double x = X[g] + a * P[g], r = R[g] - a * Q[g];
        X[g] = x;
        R[g] = r;
        m[0] = nan_max(m[0], fabs(r));
        m[1] = nan_max(m[1], fabs(x));
        m[2] = nan_max(m[2], fabs(B[g]));
    }
    block_reduce<3, true>(m);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(red + 3 * c, m[0]);
        atomic_max_nonneg(red + 3 * c + 1, m[1]);
        atomic_max_nonneg(red + 3 * c + 2, m[2]);
    }
}

// p = z + (rz_new / rz_old) p  (p = z when rz_old is 0)
__global__ void __launch_bounds__(256) k_cg_dir(double *__restrict__ P, const double *__restrict__ Z,
                                                const double *__restrict__ rz_new, const double *__restrict__ rz_old,
                                                int64_t n) {
    const int c = blockIdx.y;
    const double b = rz_old[c] != 0.0 ? rz_new[c] / rz_old[c] : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = (int64_t)c * n + i;
        P[g] = Z[g] + b * P[g];
    }
}

// grid of the column-wise vector kernels: about eight CTAs of 256 threads per
// SM over all columns, at most one CTA per 256 rows of a column
dim3 vec_grid(const sc_numeric *h, int64_t n, int64_t ncols) {
    const int64_t per_col = std::max<int64_t>(1, (int64_t)h->num_sms * 8 / std::max<int64_t>(1, ncols));
    return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, per_col)), (unsigned)ncols);
}

template <typename T>
int set_sweep_attrs();

int ensure_solve(sc_numeric *h, int64_t nrhs) {
    const sc_symbolic *s = h->sym;
    int64_t n = s->n;
    if (!h->solve_ready) {
        auto up = [&](auto *&dst, const auto &src) -> int {
            using U = typename std::remove_reference<decltype(src)>::type::value_type;
            size_t b = std::max<size_t>(1, src.size()) * sizeof(U);
            if (cudaMalloc((void **)&dst, b) != cudaSuccess) return SC_ERR_OOM;
            h->device_bytes += (int64_t)b;
            if (!src.empty() && cudaMemcpy(dst, src.data(), src.size() * sizeof(U), cudaMemcpyHostToDevice) != cudaSuccess)
                return SC_ERR_CUDA;
            return SC_OK;
        };
        int rc;
        if ((rc = up(h->d_glbind, s->glbind))) return rc;
        if ((rc = up(h->d_perm, s->perm))) return rc;
        if ((rc = up(h->d_csr_ptr, s->csr_ptr))) return rc;
        if ((rc = up(h->d_csr_col, s->csr_col))) return rc;
        if ((rc = up(h->d_csr_map, s->csr_map))) return rc;
        if (cudaMalloc((void **)&h->d_csr_val, std::max<size_t>(1, s->csr_col.size()) * 8) != cudaSuccess)
            return SC_ERR_OOM;
        // solve tiles in level order: per chunk, row tiles below the diagonal block
        std::vector<TrsmTile> tiles;
        std::vector<int32_t> ntiles(s->chunks.size(), 0);
        for (size_t lv = 0; lv < s->levels.size(); lv++) {
            for (int32_t c : s->levels[lv].chunks) {
                const Chunk &ch = s->chunks[c];
                int32_t m = (int32_t)(s->gl_ptr[ch.sn + 1] - s->gl_ptr[ch.sn]);
                int32_t r0 = ch.c0 + ch.w;
                if (r0 >= m) {
                    tiles.push_back(TrsmTile{c, r0});
                    ntiles[c] = 1;
                }
                for (; r0 < m; r0 += kSolveRows) {
                    tiles.push_back(TrsmTile{c, r0});
                    ntiles[c]++;
                }
            }
        }
        // per tile the distinct chunks its rows fall in (glbind is ascending and
        // chunk_of_col monotone, so a change of chunk along the rows starts a new
        // one); per chunk the number of tiles whose rows fall in it
        std::vector<int32_t> dep_ptr(tiles.size() + 1, 0), dep, need(s->chunks.size(), 0);
        for (size_t t = 0; t < tiles.size(); t++) {
            const Chunk &ch = s->chunks[tiles[t].chunk];
            const int64_t gl = s->gl_ptr[ch.sn];
            const int32_t m = (int32_t)(s->gl_ptr[ch.sn + 1] - gl);
            int32_t prev = -1;
            for (int32_t r = tiles[t].r0; r < std::min(m, tiles[t].r0 + kSolveRows); r++) {
                int32_t c = s->chunk_of_col[s->glbind[gl + r]];
                if (c != prev) {
                    dep.push_back(c);
                    need[c]++;
                    prev = c;
                }
            }
            dep_ptr[t + 1] = (int32_t)dep.size();
        }
        // grab units in level order: the first tile of a chunk wider than kSmallW
        // alone (one CTA; the chunk's step on the chain), its other tiles in runs of
        // up to solve_group (one CTA, one after another), else up to eight
        // consecutive narrow tiles of one level (a warp each)
        std::vector<SolveUnit> units;
        {
            // runs of 2 tiles for FP64 factors (two sweep CTAs per SM), 4 for FP32
            const int kg = knobs_of(s->tune).solve_group;
            const size_t group = (size_t)(kg > 0 ? kg : h->elt == 8 ? 2 : 4);
            size_t t = 0;
            for (size_t lv = 0; lv < s->levels.size(); lv++) {
                size_t tend = t;
                for (int32_t c : s->levels[lv].chunks) tend += ntiles[c];
                while (t < tend) {
                    const Chunk &cw = s->chunks[tiles[t].chunk];
                    if (cw.w > kSmallW) {
                        if (tiles[t].r0 == cw.c0 + cw.w) {
                            units.push_back(SolveUnit{(int32_t)t, 0});
                            t++;
                            continue;
                        }
                        size_t e = t;
                        while (e < tend && e - t < group && tiles[e].chunk == tiles[t].chunk &&
                               tiles[e].r0 != cw.c0 + cw.w)
                            e++;
                        units.push_back(SolveUnit{(int32_t)t, -(int32_t)(e - t)});
                        t = e;
                        continue;
                    }
                    size_t e = t;
                    while (e < tend && e - t < 8 && s->chunks[tiles[e].chunk].w <= kSmallW) e++;
                    units.push_back(SolveUnit{(int32_t)t, (int32_t)(e - t)});
                    t = e;
                }
            }
        }
        // per level its first tiles, then its other units: the forward sweep
        // starts every chunk's diagonal step of a level at once and its runs,
        // taken after them, find y_c published sooner; the backward sweep (the
        // reverse order) takes a level's runs of every chunk before its first
        // tiles, which wait for them
        std::vector<SolveUnit> funits;
        funits.reserve(units.size());
        {
            size_t u = 0;
            for (size_t lv = 0; lv < s->levels.size(); lv++) {
                size_t tend = 0;
                for (int32_t c : s->levels[lv].chunks) tend += ntiles[c];
                const size_t u0 = u;
                size_t seen = 0;
                while (u < units.size() && seen < tend) {
                    const SolveUnit su = units[u++];
                    seen += su.cnt > 0 ? su.cnt : su.cnt < 0 ? -su.cnt : 1;
                }
                for (size_t q = u0; q < u; q++)
                    if (units[q].cnt == 0) funits.push_back(units[q]);
                for (size_t q = u0; q < u; q++)
                    if (units[q].cnt != 0) funits.push_back(units[q]);
            }
        }
        if (funits.size() != units.size()) return SC_ERR_INTERNAL;
        h->solve_tiles = (int32_t)units.size();
        if ((rc = up(h->d_solve_tiles, tiles))) return rc;
        if ((rc = up(h->d_solve_units, funits))) return rc;
        if ((rc = up(h->d_dep_ptr, dep_ptr))) return rc;
        if ((rc = up(h->d_dep, dep))) return rc;
        // constants: tile counts [nchunks], then expected forward arrivals [nchunks]
        std::vector<int32_t> cnt2(2 * s->chunks.size(), 0);
        std::copy(ntiles.begin(), ntiles.end(), cnt2.begin());
        std::copy(need.begin(), need.end(), cnt2.begin() + s->chunks.size());
        if ((rc = up(h->d_counters, cnt2))) return rc;
        // per-sweep synchronisation words (allocated with the work vectors, zeroed
        // before every solve): per block of right-hand sides, arrivals, backward
        // counters and done flags (nchunks words each, kSyncStride apart); then
        // the two work counters
        if (cudaMalloc((void **)&h->d_serr, sizeof(int32_t)) != cudaSuccess) return SC_ERR_OOM;
        if (cudaMalloc((void **)&h->d_red, 4096 * sizeof(double)) != cudaSuccess) return SC_ERR_OOM;
        if (set_sweep_attrs<double>() || set_sweep_attrs<float>()) return SC_ERR_CUDA;
        h->solve_ready = true;
    }
    if (nrhs > h->solve_cap) {
        for (auto &g : h->sg)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        h->sg_nrhs = -1;
        double **d64[] = {&h->d_x, &h->d_r, &h->d_b, &h->d_xbest};
        for (double **p : d64) {
            if (*p) cudaFree(*p);
            if (cudaMalloc((void **)p, (size_t)n * nrhs * sizeof(double)) != cudaSuccess) return SC_ERR_OOM;
        }
        const int64_t nblk = (nrhs + kRhsBlk - 1) / kRhsBlk;
        void **dw[] = {&h->d_y, &h->d_z, &h->d_acc, &h->d_xw};
        for (void **p : dw) {
            if (*p) cudaFree(*p);
            if (cudaMalloc(p, (size_t)n * std::min<int64_t>(nrhs, kRhsBlk) * nblk * h->elt) != cudaSuccess)
                return SC_ERR_OOM;
        }
        if (h->d_sync) cudaFree(h->d_sync);
        if (cudaMalloc((void **)&h->d_sync,
                       (kSyncWords * s->chunks.size() * kSyncStride * nblk + 2) * sizeof(int32_t)) != cudaSuccess)
            return SC_ERR_OOM;
        h->solve_cap = nrhs;
    }
    return SC_OK;
}

// One triangular solve with the factor: X = A^{-1} B (or X += A^{-1} B), B and X
// column-major n x nrhs FP64 device arrays.
template <typename T, int RPT>
void launch_sweeps(sc_numeric *h, int nrhs, int64_t vs, int64_t ss, T *xw, T *y, T *z, T *acc, int32_t *sync,
                   int nblk, cudaStream_t st) {
    const sc_symbolic *s = h->sym;
    const T *lnz = (const T *)h->d_lnz;
    const size_t nch = s->chunks.size();
    const int nbmax = std::min(nrhs, kRhsBlk);
    const size_t smem = solve_smem<T>(nbmax);
    int per_sm = 1, a = 1, b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_fwd<T, RPT>, 256, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bwd<T, RPT>, 256, smem);
    per_sm = std::max(1, std::min(a, b));
    const long long spin = (long long)s->opt.spin_limit;
    const int total = h->solve_tiles * nblk;
    // persistent sweeps: as many CTAs as fit on the device at once (fewer if there is less work)
    const int grid = std::max(1, std::min(total, per_sm * h->num_sms));
    int32_t *arrive = sync, *ready = sync + nch * kSyncStride, *cnt = sync + 2 * nch * kSyncStride,
            *done = sync + 3 * nch * kSyncStride, *work = sync + nblk * ss;
    k_fwd<T, RPT><<<grid, 256, smem, st>>>(lnz, h->d_chunks, h->d_solve_tiles, h->d_solve_units, total, h->d_dep_ptr,
                                           h->d_dep, h->d_counters + nch, h->d_glbind, xw, y, nrhs, vs,
                                           (const float *)h->d_inv, arrive, ready, ss, work, h->d_serr, spin);
    k_bwd<T, RPT><<<grid, 256, smem, st>>>(lnz, h->d_chunks, h->d_solve_tiles, h->d_solve_units, total, h->d_dep_ptr,
                                           h->d_dep, h->d_counters, h->d_glbind, y, z, acc, nrhs, vs,
                                           (const float *)h->d_inv, cnt, done, ss, work + 1, h->d_serr, spin);
}

template <typename T>
int set_sweep_attrs() {
    const int smem = (int)solve_smem<T>(kRhsBlk);
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *k) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    set((const void *)k_fwd<T, 1>), set((const void *)k_bwd<T, 1>);
    set((const void *)k_fwd<T, 2>), set((const void *)k_bwd<T, 2>);
    set((const void *)k_fwd<T, 4>), set((const void *)k_bwd<T, 4>);
    set((const void *)k_fwd<T, 8>), set((const void *)k_bwd<T, 8>);
    set((const void *)k_fwd<T, 16>), set((const void *)k_bwd<T, 16>);
    return e == cudaSuccess ? 0 : 1;
}

template <typename T>
int tri_solve(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int add,
              cudaStream_t st, int &launches) {
    const sc_symbolic *s = h->sym;
    const int64_t n = s->n;
    T *xw = (T *)h->d_xw, *y = (T *)h->d_y, *z = (T *)h->d_z, *acc = (T *)h->d_acc;
    const size_t nch = s->chunks.size();
    // every block of kRhsBlk right-hand sides has its own work vectors and
    // synchronisation words; one persistent launch per sweep serves them all
    const int nblk = (int)((nrhs + kRhsBlk - 1) / kRhsBlk);
    const int64_t vs = n * std::min<int64_t>(nrhs, kRhsBlk), ss = kSyncWords * (int64_t)nch * kSyncStride;
    for (int bk = 0; bk < nblk; bk++) {
        const int nb = (int)std::min<int64_t>(kRhsBlk, nrhs - bk * kRhsBlk);
        const unsigned g = (unsigned)((n * nb + 255) / 256);
        k_perm_in<T><<<g, 256, 0, st>>>(xw + bk * vs, B, ldb, h->d_perm, n, nb, bk * kRhsBlk);
        launches++;
    }
    SC_CUDA(cudaMemsetAsync(h->d_sync, 0, (nblk * ss + 2) * sizeof(int32_t), st));
    SC_CUDA(cudaMemsetAsync(acc, 0, (size_t)nblk * vs * sizeof(T), st));
    switch (rhs_per_thread((int)std::min<int64_t>(nrhs, kRhsBlk))) {
        case 1: launch_sweeps<T, 1>(h, (int)nrhs, vs, ss, xw, y, z, acc, h->d_sync, nblk, st); break;
        case 2: launch_sweeps<T, 2>(h, (int)nrhs, vs, ss, xw, y, z, acc, h->d_sync, nblk, st); break;
        case 4: launch_sweeps<T, 4>(h, (int)nrhs, vs, ss, xw, y, z, acc, h->d_sync, nblk, st); break;
        case 8: launch_sweeps<T, 8>(h, (int)nrhs, vs, ss, xw, y, z, acc, h->d_sync, nblk, st); break;
        default: launch_sweeps<T, 16>(h, (int)nrhs, vs, ss, xw, y, z, acc, h->d_sync, nblk, st); break;
    }
    launches += 2;
    for (int bk = 0; bk < nblk; bk++) {
        const int nb = (int)std::min<int64_t>(kRhsBlk, nrhs - bk * kRhsBlk);
        const unsigned g = (unsigned)((n * nb + 255) / 256);
        k_perm_out<T><<<g, 256, 0, st>>>(X, ldx, z + bk * vs, h->d_perm, n, nb, bk * kRhsBlk, add);
        launches++;
    }
    SC_CUDA(cudaGetLastError());
    return SC_OK;
}

int tri_solve_any(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int add,
                  cudaStream_t st, int &launches) {
    return h->elt == 8 ? tri_solve<double>(h, nrhs, B, ldb, X, ldx, add, st, launches)
                       : tri_solve<float>(h, nrhs, B, ldb, X, ldx, add, st, launches);
}

// eta per column for the current iterate in h->d_x; returns host values
// enqueues the residual r = b - A x and the per-column maxima for eta
int enqueue_residual(sc_numeric *h, int64_t nrhs, cudaStream_t st, int &launches) {
    const int64_t n = h->sym->n;
    SC_CUDA(cudaMemsetAsync(h->d_red, 0, 3 * nrhs * sizeof(double), st));
    k_residual<<<vec_grid(h, n, nrhs), 256, 0, st>>>(h->d_csr_ptr, h->d_csr_col, h->d_csr_val, h->d_x, h->d_b, h->d_r, n, (int)nrhs,
                                  h->d_red);
    launches++;
    return SC_OK;
}

// one refinement step on the device: step 0: x = solve(b); step 1: x += solve(r); then the residual
int enqueue_step(sc_numeric *h, int64_t nrhs, int step, cudaStream_t st, int &launches) {
    const int64_t n = h->sym->n;
    int rc = step == 0 ? tri_solve_any(h, nrhs, h->d_b, n, h->d_x, n, 0, st, launches)
                       : tri_solve_any(h, nrhs, h->d_r, n, h->d_x, n, 1, st, launches);
    if (rc) return rc;
    return enqueue_residual(h, nrhs, st, launches);
}

// runs a step, replaying a CUDA graph of it when the handle uses graphs
int run_step(sc_numeric *h, int64_t nrhs, int step, cudaStream_t st, int &launches) {
    if (!h->use_graph) return enqueue_step(h, nrhs, step, st, launches);
    if (h->sg_nrhs != nrhs) {
        for (auto &g : h->sg)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        h->sg_nrhs = nrhs;
    }
    if (!h->sg[step]) {
        if (!h->cap_stream) SC_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g;
        int cnt = 0;
        SC_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_step(h, nrhs, step, h->cap_stream, cnt);
        cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc) return rc;
        SC_CUDA(ce);
        SC_CUDA(cudaGraphInstantiate(&h->sg[step], g, 0));
        cudaGraphDestroy(g);
        h->sg_launches[step] = cnt;
    }
    SC_CUDA(cudaGraphLaunch(h->sg[step], st));
    launches += h->sg_launches[step];
    return SC_OK;
}

// eta per column from the maxima of the last residual
int read_eta(sc_numeric *h, int64_t nrhs, cudaStream_t st, std::vector<double> &eta) {
    std::vector<double> red(3 * nrhs);
    int32_t werr = 0;
    SC_CUDA(cudaMemcpyAsync(red.data(), h->d_red, red.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    SC_CUDA(cudaMemcpyAsync(&werr, h->d_serr, sizeof(werr), cudaMemcpyDeviceToHost, st));
    SC_CUDA(cudaStreamSynchronize(st));
    if (werr) return SC_ERR_TIMEOUT;
    eta.resize(nrhs);
    for (int64_t c = 0; c < nrhs; c++) {
        const double r = red[3 * c], den = h->anorm * red[3 * c + 1] + red[3 * c + 2];
        // a NaN or infinity in the residual, the iterate or the right-hand side
        // gives eta = NaN, never a value that passes the tolerance
        if (!std::isfinite(r) || !std::isfinite(den)) eta[c] = NAN;
        else eta[c] = den > 0 ? r / den : (r == 0.0 ? 0.0 : INFINITY);
    }
    return SC_OK;
}

// largest eta over the columns; +inf when some column's eta is NaN, so the
// refinement loops treat it as not converged
double max_eta(const std::vector<double> &eta) {
    double m = 0.0;
    for (double e : eta) {
        if (std::isnan(e)) return INFINITY;
        m = std::max(m, e);
    }
    return m;
}

}  // namespace

int numeric_solve(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int on_device,
                  cudaStream_t st, sc_solve_info *info);

namespace {
// Test hook: one solve in which the forward sweep expects one arrival more at
// chunk h->stall_chunk than it will receive, so that chunk's bounded waits give
// up and the solve returns SC_ERR_TIMEOUT. The expected count is restored and
// the hook cleared afterwards.
int solve_with_stall(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int on_device,
                     cudaStream_t st, sc_solve_info *info) {
    const int32_t c = h->stall_chunk;
    h->stall_chunk = -1;
    const size_t nch = h->sym->chunks.size();
    if (c >= (int32_t)nch) return -1;
    int rc0 = ensure_solve(h, nrhs);
    if (rc0) return rc0;
    int32_t *slot = h->d_counters + nch + c, need = 0;
    SC_CUDA(cudaMemcpy(&need, slot, sizeof(need), cudaMemcpyDeviceToHost));
    const int32_t raised = need + 1;
    SC_CUDA(cudaMemcpy(slot, &raised, sizeof(raised), cudaMemcpyHostToDevice));
    int rc = numeric_solve(h, nrhs, B, ldb, X, ldx, on_device, st, info);
    cudaStreamSynchronize(st);
    if (cudaMemcpy(slot, &need, sizeof(need), cudaMemcpyHostToDevice) != cudaSuccess) return SC_ERR_CUDA;
    return rc;
}
}  // namespace

namespace {
// Conjugate gradients on A x = b preconditioned by the factor, started from the
// iterate in h->d_x whose residual is in h->d_r (step 0 of the solve). Each
// iteration reads the per-column eta of the recursively updated residual; when
// it reaches tol, the true residual b - A x is formed and checked, and CG
// restarts from it if it is not yet below tol. h->d_xbest receives the best
// iterate by the true residual; best / best_eta its eta.
int pcg(sc_numeric *h, int64_t nrhs, cudaStream_t st, double tol, int maxit, double emax0, double &best,
        std::vector<double> &best_eta, int &it, int &launches) {
    const int64_t n = h->sym->n;
    if (h->cg_cap < nrhs) {
        double **arr[] = {&h->d_cgz, &h->d_cgp, &h->d_cgq};
        for (double **p : arr) {
            if (*p) cudaFree(*p);
            if (cudaMalloc((void **)p, (size_t)n * nrhs * sizeof(double)) != cudaSuccess) return SC_ERR_OOM;
        }
        if (h->d_cgs) cudaFree(h->d_cgs);
        if (cudaMalloc((void **)&h->d_cgs, 3 * nrhs * sizeof(double)) != cudaSuccess) return SC_ERR_OOM;
        h->cg_cap = nrhs;
    }
    const dim3 g = vec_grid(h, n, nrhs);
    double *rz = h->d_cgs, *rz2 = h->d_cgs + nrhs, *pq = h->d_cgs + 2 * nrhs;
    int rc;
    // z = M^-1 r, p = z, rz = r . z
    auto restart = [&]() -> int {
        int r2 = tri_solve_any(h, nrhs, h->d_r, n, h->d_cgz, n, 0, st, launches);
        if (r2) return r2;
        SC_CUDA(cudaMemcpyAsync(h->d_cgp, h->d_cgz, (size_t)n * nrhs * 8, cudaMemcpyDeviceToDevice, st));
        SC_CUDA(cudaMemsetAsync(rz, 0, nrhs * sizeof(double), st));
        k_dot<<<g, 256, 0, st>>>(h->d_r, h->d_cgz, n, rz);
        launches++;
        return SC_OK;
    };
    if ((rc = restart())) return rc;
    std::vector<double> eta;
    double emax = emax0;
    while (it < maxit) {
        SC_CUDA(cudaMemsetAsync(pq, 0, nrhs * sizeof(double), st));
        k_spmv_dot<<<g, 256, 0, st>>>(h->d_csr_ptr, h->d_csr_col, h->d_csr_val, h->d_cgp, h->d_cgq, n, pq);
        SC_CUDA(cudaMemsetAsync(h->d_red, 0, 3 * nrhs * sizeof(double), st));
        k_cg_step<<<g, 256, 0, st>>>(h->d_x, h->d_r, h->d_cgp, h->d_cgq, h->d_b, rz, pq, n, h->d_red);
        launches += 2;
        it++;
        if ((rc = read_eta(h, nrhs, st, eta))) return rc;
        emax = max_eta(eta);
        if (emax <= tol) {
            // the true residual decides
            if ((rc = enqueue_residual(h, nrhs, st, launches))) return rc;
            if ((rc = read_eta(h, nrhs, st, eta))) return rc;
            emax = max_eta(eta);
            if (emax < best) {
                best = emax;
                best_eta = eta;
                SC_CUDA(cudaMemcpyAsync(h->d_xbest, h->d_x, (size_t)n * nrhs * 8, cudaMemcpyDeviceToDevice, st));
            }
            if (emax <= tol) break;
            if ((rc = restart())) return rc;
            continue;
        }
        // z = M^-1 r; rz2 = r . z; p = z + (rz2 / rz) p
        if ((rc = tri_solve_any(h, nrhs, h->d_r, n, h->d_cgz, n, 0, st, launches))) return rc;
        SC_CUDA(cudaMemsetAsync(rz2, 0, nrhs * sizeof(double), st));
        k_dot<<<g, 256, 0, st>>>(h->d_r, h->d_cgz, n, rz2);
        k_cg_dir<<<g, 256, 0, st>>>(h->d_cgp, h->d_cgz, rz2, rz, n);
        launches += 2;
        std::swap(rz, rz2);
    }
    if (emax > tol) {
        // cap reached: keep the better of the last iterate and the best so far, by the true residual
        if ((rc = enqueue_residual(h, nrhs, st, launches))) return rc;
        if ((rc = read_eta(h, nrhs, st, eta))) return rc;
        emax = max_eta(eta);
        if (emax < best) {
            best = emax;
            best_eta = eta;
            SC_CUDA(cudaMemcpyAsync(h->d_xbest, h->d_x, (size_t)n * nrhs * 8, cudaMemcpyDeviceToDevice, st));
        }
    }
    return SC_OK;
}
}  // namespace

int numeric_solve(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int on_device,
                  cudaStream_t st, sc_solve_info *info) {
    const sc_symbolic *s = h->sym;
    const int64_t n = s->n;
    int rc = ensure_solve(h, nrhs);
    if (rc) return rc;
    h->last_stream = st;
    if (nrhs > 1365) return -2;  // the reduction buffer holds 3 values per column (+ ||A||)
    if (h->stall_chunk >= 0) return solve_with_stall(h, nrhs, B, ldb, X, ldx, on_device, st, info);
    struct Events {  // destroyed on every return path
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (cudaEvent_t &x : ev.e) SC_CUDA(cudaEventCreate(&x));
    // e0 .. e_in: B in; e_out .. e1: X out
    cudaEvent_t e0 = ev.e[0], e_in = ev.e[1], e_out = ev.e[2], e1 = ev.e[3];
    SC_CUDA(cudaEventRecord(e0, st));
    // b (column-major, ld = n) on the device: one copy when the columns are contiguous
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (ldb == n) {
        SC_CUDA(cudaMemcpyAsync(h->d_b, B, (size_t)n * nrhs * sizeof(double), kin, st));
    } else {
        for (int64_t c = 0; c < nrhs; c++)
            SC_CUDA(cudaMemcpyAsync(h->d_b + c * n, B + c * ldb, n * sizeof(double), kin, st));
    }
    SC_CUDA(cudaEventRecord(e_in, st));
    // matrix values in CSR order and ||A||_inf (values may change with every refactor)
    int64_t nnzc = (int64_t)s->csr_col.size();
    k_gather_vals<<<(unsigned)((nnzc + 255) / 256), 256, 0, st>>>(h->d_csr_val, h->d_values, h->d_csr_map, nnzc);
    SC_CUDA(cudaMemsetAsync(h->d_red + 4095, 0, sizeof(double), st));
    k_anorm<<<vec_grid(h, n, 1), 256, 0, st>>>(h->d_csr_ptr, h->d_csr_val, n, h->d_red + 4095);
    SC_CUDA(cudaMemcpyAsync(&h->anorm, h->d_red + 4095, sizeof(double), cudaMemcpyDeviceToHost, st));
    SC_CUDA(cudaMemsetAsync(h->d_serr, 0, sizeof(int32_t), st));
    int launches = 2;
    // x0 = solve(b), then its residual
    if ((rc = run_step(h, nrhs, 0, st, launches))) return rc;
    const bool refine = info && info->refine >= 0 ? info->refine != 0 : h->precision != SC_FP64;
    const double tol = s->opt.ir_tol;
    const int maxit = s->opt.ir_maxit;
    std::vector<double> eta, best_eta;
    std::vector<double> hist;
    if ((rc = read_eta(h, nrhs, st, eta))) return rc;
    double emax = max_eta(eta);
    double best = emax;
    best_eta = eta;
    SC_CUDA(cudaMemcpyAsync(h->d_xbest, h->d_x, (size_t)n * nrhs * 8, cudaMemcpyDeviceToDevice, st));
    hist.push_back(emax);
    int it = 0;
    const bool cg = info && info->method == 1;
    if (refine && cg && emax > tol) {
        if ((rc = pcg(h, nrhs, st, tol, info->max_iterations > 0 ? info->max_iterations : maxit, emax, best, best_eta,
                      it, launches)))
            return rc;
    } else if (refine) {
        while (emax > tol && it < maxit) {
            // d = solve(r); x += d; new residual
            if ((rc = run_step(h, nrhs, 1, st, launches))) return rc;
            it++;
            if ((rc = read_eta(h, nrhs, st, eta))) return rc;
            emax = max_eta(eta);
            hist.push_back(emax);
            if (emax < best) {
                best = emax;
                best_eta = eta;
                SC_CUDA(cudaMemcpyAsync(h->d_xbest, h->d_x, (size_t)n * nrhs * 8, cudaMemcpyDeviceToDevice, st));
            }
            // stagnation: no halving over the last 3 iterations
            if (hist.size() > 3 && emax > 0.5 * hist[hist.size() - 4]) break;
        }
    }
    SC_CUDA(cudaEventRecord(e_out, st));
    const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (ldx == n) {
        SC_CUDA(cudaMemcpyAsync(X, h->d_xbest, (size_t)n * nrhs * sizeof(double), kout, st));
    } else {
        for (int64_t c = 0; c < nrhs; c++)
            SC_CUDA(cudaMemcpyAsync(X + c * ldx, h->d_xbest + c * n, n * sizeof(double), kout, st));
    }
    SC_CUDA(cudaEventRecord(e1, st));
    SC_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f, ms_in = 0.f, ms_out = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventElapsedTime(&ms_in, e0, e_in);
    cudaEventElapsedTime(&ms_out, e_out, e1);
    bool conv = best <= tol;
    if (info) {
        info->copy_in_ms = ms_in;
        info->copy_out_ms = ms_out;
        info->iterations = it;
        info->converged = conv ? 1 : 0;
        info->eta_max = best;
        info->solve_ms = ms;
        info->kernel_launches = launches;
        if (info->eta) std::copy(best_eta.begin(), best_eta.end(), info->eta);
    }
    if (refine && !conv) return SC_ERR_NOT_CONVERGED;
    return SC_OK;
}

}  // namespace sc
