// Device kernels of the numeric factorization and the solve (SIMT part).
// Factor storage: supernode J is a row-major m_J x ld_J panel at element offset
// off_J of one buffer (row r = glbind(J)[r], column c = column f_J + c).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "device_types.h"

namespace sc {



// TF32 rounding (round to nearest, ties away from zero; the low 13 mantissa
// bits of the result are zero).
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// Split of a final factor entry for the three-product TF32 form: hi = tf32(x),
// lo = tf32(x - hi) (x - hi is exact in FP32), written at the same element
// offset of the hi and lo copies of the factor storage.
__device__ __forceinline__ void store_split(float *__restrict__ hi, float *__restrict__ lo, int64_t e, float x) {
    const float h = tf32_rna(x);
    hi[e] = h;
    lo[e] = tf32_rna(x - h);
}

// --------------------------------------------------------------------- K0
template <typename T>
__global__ void k_scatter_values(T *__restrict__ lnz, const int64_t *__restrict__ valmap,
                                 const double *__restrict__ values, int64_t nnz) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < nnz; i += stride) lnz[valmap[i]] = (T)values[i];
}

// --------------------------------------------------------------------- K1
// POTRF of each chunk's w x w diagonal block (lower) in shared memory,
// right-looking by panels of 8 columns. Per panel:
//   1. the panel's 8 x 8 diagonal block is factored in registers: FP32 by one
//      thread (no shuffles on the serial chain of pivots), FP64 by warp 0 (lane
//      i holds row i; pivots and column entries are broadcast by shuffles);
//   2. every row below it is solved against that block, one thread per row
//      (x <- x L_d^{-T}, reciprocal pivots);
//   3. all 256 threads apply the panel's rank-8 update to the trailing triangle.
//   T = double: one pass in FP64; a pivot d <= 0 sets info.
//   T = float : one pass in FP32. If some pivot d (before the square root)
//               is <= tau * |A_jj| (A_jj = the diagonal entry of the input
//               matrix), the block is refactored in FP64 from the same stored
//               values and low_pivots is incremented; a pivot <= 0 in that
//               pass sets info.
// info receives the minimum failing column (1-based, final ordering). thr[k] =
// tau * |A_jj| of the block's column k, staged in shared memory.
template <typename S>
__device__ bool potrf_pass(S (*a)[kMaxChunk + 1], int w, const double *thr, int col0, bool check_low,
                           int32_t *__restrict__ info, int *flag) {
    constexpr int PW = 8;  // panel width
    __shared__ S rpiv[PW];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads
    for (int p0 = 0; p0 < w; p0 += PW) {
        const int pw = min(PW, w - p0), p1 = p0 + pw;
        if (sizeof(S) == 8 && threadIdx.x < 32) {
            // FP64: warp 0, lane i holding row i, pivots and column entries broadcast
            // by shuffles (one thread's FP64 chain would be slower)
            const int lane = threadIdx.x;
            S r[PW];
#pragma unroll
            for (int j = 0; j < PW; j++) r[j] = (lane < pw && j <= lane) ? a[p0 + lane][p0 + j] : S(0);
#pragma unroll
            for (int k = 0; k < PW; k++) {
                if (k < pw) {
                    S d = __shfl_sync(0xffffffffu, r[k], k);  // the same value in every lane
                    if (!(d > S(0))) {
                        if (lane == 0) atomicMin(info, col0 + p0 + k + 1);
                        d = S(1);
                    }
                    const S rk = rsqrt(d), sq = d * rk;
                    if (lane == k) r[k] = sq;
                    else if (lane > k) r[k] *= rk;
                    if (lane == 0) rpiv[k] = rk;
#pragma unroll
                    for (int j = k + 1; j < PW; j++) {
                        const S ljk = __shfl_sync(0xffffffffu, r[k], j);
                        if (lane >= j) r[j] -= r[k] * ljk;
                    }
                }
            }
            if (lane < pw) {
#pragma unroll
                for (int j = 0; j < PW; j++)
                    if (j <= lane) a[p0 + lane][p0 + j] = r[j];
            }
        } else if (sizeof(S) == 4 && threadIdx.x == 0) {
            // FP32: the panel's diagonal block in one thread's registers, no shuffles
            // on the serial chain of pivots (rows past pw hold the identity)
            S r[PW][PW];
#pragma unroll
            for (int i = 0; i < PW; i++)
#pragma unroll
                for (int j = 0; j <= i; j++) r[i][j] = i < pw ? a[p0 + i][p0 + j] : S(i == j ? 1 : 0);
            bool low = false;
#pragma unroll
            for (int k = 0; k < PW; k++) {
                if (k < pw) {
                    S d = r[k][k];
                    if (check_low) {
                        // the pivot threshold tau |A_jj| in the block's precision
                        if (!(d > (S)thr[p0 + k])) low = true;
                    } else if (!(d > S(0))) {
                        atomicMin(info, col0 + p0 + k + 1);
                    }
                    if (!(d > S(0))) d = S(1);
                    const S rk = rsqrt(d);
                    r[k][k] = d * rk;
                    rpiv[k] = rk;
#pragma unroll
                    for (int i = k + 1; i < PW; i++) r[i][k] *= rk;
#pragma unroll
                    for (int i = k + 1; i < PW; i++)
#pragma unroll
                        for (int j = k + 1; j <= i; j++) r[i][j] -= r[i][k] * r[j][k];
                }
            }
#pragma unroll
            for (int i = 0; i < PW; i++)
#pragma unroll
                for (int j = 0; j <= i; j++)
                    if (i < pw) a[p0 + i][p0 + j] = r[i][j];
            if (low) *flag = 1;
        }
        __syncthreads();
        if (check_low && *flag) return false;
        // rows below the diagonal block: x <- x L_d^{-T}
        for (int i = p1 + threadIdx.x; i < w; i += blockDim.x) {
            S x[PW];
#pragma unroll
            for (int j = 0; j < PW; j++) x[j] = j < pw ? a[i][p0 + j] : S(0);
#pragma unroll
            for (int k = 0; k < PW; k++) {
                x[k] *= rpiv[k];
#pragma unroll
                for (int j = k + 1; j < PW; j++) x[j] -= x[k] * a[p0 + j][p0 + k];
            }
#pragma unroll
            for (int j = 0; j < PW; j++)
                if (j < pw) a[i][p0 + j] = x[j];
        }
        __syncthreads();
        // rank-(p1-p0) update of the trailing lower triangle
        for (int i = p1 + ty; i < w; i += 16) {
            S ai[PW];
#pragma unroll
            for (int t = 0; t < PW; t++) ai[t] = p0 + t < p1 ? a[i][p0 + t] : S(0);
            for (int j = p1 + tx; j <= i; j += 16) {
                S acc = S(0);
#pragma unroll
                for (int t = 0; t < PW; t++) acc += ai[t] * (p0 + t < p1 ? a[j][p0 + t] : S(0));
                a[i][j] -= acc;
            }
        }
        __syncthreads();
    }
    return true;
}

// Loads the lower triangle of a w x w block (row stride ld) into shared memory
// (upper part zero) with a fixed trip count per thread (256 threads), so each
// thread keeps all of its loads in flight.
template <typename S, typename T>
__device__ __forceinline__ void load_block(S (*a)[kMaxChunk + 1], const T *__restrict__ src, int64_t ld, int w) {
    constexpr int kIters = kMaxChunk * kMaxChunk / 256;
    T tmp[kIters];
#pragma unroll
    for (int it = 0; it < kIters; it++) {
        const int idx = threadIdx.x + it * 256, r = idx / kMaxChunk, c = idx % kMaxChunk;
        tmp[it] = (r < w && c <= r) ? src[(int64_t)r * ld + c] : T(0);
    }
#pragma unroll
    for (int it = 0; it < kIters; it++) {
        const int idx = threadIdx.x + it * 256;
        a[idx / kMaxChunk][idx % kMaxChunk] = (S)tmp[it];
    }
}

// dynamic shared memory of k_potrf (the block, FP64 or FP32) and of k_inverse
// (the FP32 block, then the FP32 inverse)
constexpr int kPotrfSmem = kMaxChunk * (kMaxChunk + 1) * 8;

// Inverse of the factored w x w lower-triangular block held in shared memory,
// stored row-major (ld = w) in FP32 for the solve sweeps of FP32 / TF32
// factors. Thread j builds column j by forward substitution in FP32, keeping
// the column in the shared buffer iv (each thread reads only its own column).
template <typename S>
__device__ void tri_inverse(const S (*a)[kMaxChunk + 1], int w, float (*iv)[kMaxChunk + 1],
                            float *__restrict__ out) {
    const int j = threadIdx.x;
    if (j < w) {
        for (int i = 0; i < j; i++) iv[i][j] = 0.f;
        for (int i = j; i < w; i++) {
            float acc = i == j ? 1.f : 0.f;
            for (int t = j; t < i; t++) acc -= (float)a[i][t] * iv[t][j];
            iv[i][j] = acc / (float)a[i][i];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) out[idx] = iv[idx / w][idx % w];
}

// POTRF of chunk c by one CTA of 256 threads (the body of k_potrf and of the
// per-level kernel's POTRF units); kPotrfSmem bytes of dynamic shared memory.
template <typename T>
__device__ void potrf_chunk(T *__restrict__ lnz, const ChunkDev *__restrict__ chunks, int32_t c,
                            const double *__restrict__ adiag, int32_t *__restrict__ info,
                            int32_t *__restrict__ low_pivots, double tau, float *__restrict__ hi,
                            float *__restrict__ lo) {
    extern __shared__ double smem_potrf[];
    __shared__ int flag;
    __shared__ double thr[kMaxChunk];
    const ChunkDev ch = chunks[c];
    const int w = ch.w;
    T *base = lnz + ch.off + (int64_t)ch.c0 * ch.ld + ch.c0;
    if (threadIdx.x == 0) flag = 0;
    if (threadIdx.x < w) thr[threadIdx.x] = tau * fabs(adiag[ch.col0 + threadIdx.x]);
    if (sizeof(T) == 4) {
        auto a = reinterpret_cast<float (*)[kMaxChunk + 1]>(smem_potrf);
        load_block(a, base, ch.ld, w);
        __syncthreads();
        if (potrf_pass<float>(a, w, thr, ch.col0, true, info, &flag)) {
            for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
                int r = idx / w, c = idx % w;
                if (r >= c) {
                    base[(int64_t)r * ch.ld + c] = (T)a[r][c];
                    if (hi) store_split(hi, lo, (base - lnz) + (int64_t)r * ch.ld + c, a[r][c]);
                }
            }
            return;
        }
        if (threadIdx.x == 0) atomicAdd(low_pivots, 1);
        __syncthreads();
    }
    // FP64 factorization (the FP64 path, or the fallback of a low pivot)
    auto a = reinterpret_cast<double (*)[kMaxChunk + 1]>(smem_potrf);
    load_block(a, base, ch.ld, w);
    __syncthreads();
    potrf_pass<double>(a, w, thr, ch.col0, false, info, &flag);
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        int r = idx / w, c = idx % w;
        if (r >= c) {
            base[(int64_t)r * ch.ld + c] = (T)a[r][c];
            if (sizeof(T) == 4 && hi) store_split(hi, lo, (base - lnz) + (int64_t)r * ch.ld + c, (float)a[r][c]);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_potrf(T *__restrict__ lnz, const ChunkDev *__restrict__ chunks,
                                               const int32_t *__restrict__ list, const double *__restrict__ adiag,
                                               int32_t *__restrict__ info, int32_t *__restrict__ low_pivots,
                                               double tau, float *__restrict__ hi, float *__restrict__ lo) {
    potrf_chunk<T>(lnz, chunks, list[blockIdx.x], adiag, info, low_pivots, tau, hi, lo);
}

// --------------------------------------------------------------------- K2
// TRSM of the rows below each chunk's diagonal block: row x <- x L_cc^{-T} by
// forward substitution. Four threads share a row (thread q of the row holds
// columns q, q+4, ... in registers; the chunk is zero-padded to 64 columns so
// the substitution unrolls fully); each pivot value is broadcast from its
// owner with a width-4 shuffle; pivots are applied as reciprocals; L_cc is
// read from shared memory. Storage precision.
// Rows per TRSM tile: 32 in FP32; 16 in FP64, so a wide chunk's rows spread
// over twice as many SMs (the FP64 pipe of one SM is narrow).
template <typename T>
__host__ __device__ constexpr int trsm_rows() {
    return sizeof(T) == 8 ? 16 : 32;
}

// Substitution of one row for a chunk of width <= W (W in {8, 16, 32, 64}): the
// loops unroll to W, so narrow chunks do not spend FMA-pipe cycles on padding.
template <typename T, int W>
__device__ __forceinline__ void trsm_row(const T (*l)[kMaxChunk + 1], const T *rinv, T *xr, bool live, int w, int q,
                                         T *lnz, float *hi, float *lo) {
    constexpr int NJ = W / 4;
    T x[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; jj++) {
        const int j = q + 4 * jj;
        x[jj] = (live && j < w) ? xr[j] : T(0);
    }
#pragma unroll
    for (int k = 0; k < W; k++) {
        T v = (q == (k & 3)) ? x[k >> 2] * rinv[k] : T(0);
        v = __shfl_sync(0xffffffffu, v, k & 3, 4);
        if (q == (k & 3)) x[k >> 2] = v;
#pragma unroll
        for (int jj = 0; jj < NJ; jj++) {
            if (4 * jj + 3 > k) {  // resolved at compile time: some lane of the quad has j > k
                const int j = q + 4 * jj;
                if (j > k) x[jj] -= v * l[j][k];
            }
        }
    }
    if (live) {
#pragma unroll
        for (int jj = 0; jj < NJ; jj++) {
            const int j = q + 4 * jj;
            if (j < w) {
                xr[j] = x[jj];
                if (sizeof(T) == 4 && hi) store_split(hi, lo, (xr - lnz) + j, (float)x[jj]);
            }
        }
    }
}

// TRSM of one tile (trsm_rows<T>() rows, four threads each) by the first
// trsm_rows<T>() * 4 threads of the CTA; every thread of the CTA takes part in
// the barriers (the body of k_trsm and of the per-level kernel's TRSM units).
template <typename T>
__device__ void trsm_tile(T *__restrict__ lnz, const ChunkDev *__restrict__ chunks, const TrsmTile &tl,
                          float *__restrict__ hi, float *__restrict__ lo) {
    __shared__ T l[kMaxChunk][kMaxChunk + 1];
    __shared__ T rinv[kMaxChunk];
    constexpr int kThreads = trsm_rows<T>() * 4;
    const ChunkDev ch = chunks[tl.chunk];
    const int w = ch.w;
    const T *diag = lnz + ch.off + (int64_t)ch.c0 * ch.ld + ch.c0;
    if (threadIdx.x < kThreads) {
        // fixed-trip staging through registers, 16 loads in flight per thread
        constexpr int kIters = kMaxChunk * kMaxChunk / kThreads;
        for (int it0 = 0; it0 < kIters; it0 += 16) {
            T tmp[16];
#pragma unroll
            for (int it = 0; it < 16; it++) {
                const int idx = threadIdx.x + (it0 + it) * kThreads, r = idx / kMaxChunk, c = idx % kMaxChunk;
                tmp[it] = (r < w && c <= r) ? diag[(int64_t)r * ch.ld + c] : T(0);
            }
#pragma unroll
            for (int it = 0; it < 16; it++) {
                const int idx = threadIdx.x + (it0 + it) * kThreads;
                l[idx / kMaxChunk][idx % kMaxChunk] = tmp[it];
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kMaxChunk; k += blockDim.x) rinv[k] = k < w ? T(1) / l[k][k] : T(0);
    __syncthreads();
    if (threadIdx.x >= kThreads) return;  // whole warps: the shuffles below stay within a warp
    const int q = threadIdx.x % 4;
    const int row = tl.r0 + threadIdx.x / 4;
    const bool live = row < ch.m;
    T *xr = lnz + ch.off + (int64_t)(live ? row : tl.r0) * ch.ld + ch.c0;
    if (w <= 8) trsm_row<T, 8>(l, rinv, xr, live, w, q, lnz, hi, lo);
    else if (w <= 16) trsm_row<T, 16>(l, rinv, xr, live, w, q, lnz, hi, lo);
    else if (w <= 32) trsm_row<T, 32>(l, rinv, xr, live, w, q, lnz, hi, lo);
    else trsm_row<T, 64>(l, rinv, xr, live, w, q, lnz, hi, lo);
}

template <typename T>
__global__ void __launch_bounds__(trsm_rows<T>() * 4) k_trsm(T *__restrict__ lnz, const ChunkDev *__restrict__ chunks,
                                                       const TrsmTile *__restrict__ tiles, float *__restrict__ hi,
                                                       float *__restrict__ lo) {
    trsm_tile<T>(lnz, chunks, tiles[blockIdx.x], hi, lo);
}

// --------------------------------------------------------------------- K3
// The multiply-adds of one staged K slice for a warp whose micro-tiles reach
// NI row groups and NJ column groups inside the task.
template <typename T, int NI, int NJ, int BK>
__device__ __forceinline__ void tile_fma(const T (*As)[64 + 1], const T (*Bs)[64 + 1], int r0, int c0, int kn,
                                         T (&acc)[4][4]) {
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
        if (kk < kn) {
            T a[NI], b[NJ];
#pragma unroll
            for (int i = 0; i < NI; i++) a[i] = As[kk][r0 + 4 * i];
#pragma unroll
            for (int j = 0; j < NJ; j++) b[j] = Bs[kk][c0 + 8 * j];
#pragma unroll
            for (int i = 0; i < NI; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) acc[i][j] += a[i] * b[j];
        }
    }
}

// Tiled product C -= A B^T (or C = -A B^T into an RL update matrix) on SIMT
// FMA units. 256 threads, 64 x 64 tile; warp w owns the 16 x 32 sub-tile
// (rows 16 (w / 2), columns 32 (w % 2)) and each lane a 4 x 4 strided micro-tile
// of it. A warp whose sub-tile lies outside m x n, or wholly above the diagonal
// of a lower task, skips its multiply-adds (it still helps stage the operands);
// a warp at the ragged edge runs only the row groups (4 rows apart) and column
// groups (8 columns apart) that reach inside the task, and the last K slice
// runs only its valid columns, so ragged tiles spend few FMA-pipe cycles on
// padding. The scatter into Lnz(P) is an atomic add
// unless the task is the only writer of its target: supernodes of one level
// may update the same ancestor entries.
// One tile by one CTA of 256 threads (the body of k_gemm_tiles and of the
// per-level kernel's product units). atomic_only: every target entry is added
// atomically, also for an exclusive target (other units of the same launch may
// update it concurrently).
template <typename T, int BM, int BN, int BK>
__device__ void gemm_tile(T *__restrict__ lnz, T *__restrict__ pool, const Task *__restrict__ tasks,
                          const GemmTile &tl, bool atomic_only) {
    static_assert(BM == 64 && BN == 64, "8 warps of 16 x 32 sub-tiles");
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const Task tk = tasks[tl.task];
    const int row0 = tl.tm * BM, col0 = tl.tn * BN;
    const T *A = lnz + tk.a_off;
    const T *B = lnz + tk.b_off;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r0 = (warp / 2) * 16 + lane / 8;  // rows r0 + 4 i
    const int c0 = (warp % 2) * 32 + lane % 8;  // columns c0 + 8 j
    const bool lower = tk.flags & kTaskLower;
    // warp-uniform: does the sub-tile hold any entry that is written?
    const int sr = row0 + (warp / 2) * 16, sc = col0 + (warp % 2) * 32;
    const bool active = sr < tk.m && sc < tk.n && !(lower && min(sr + 15, tk.m - 1) < sc);
    // row groups (4 rows apart) and column groups (8 columns apart) of the
    // warp's micro-tiles that reach inside the task: the others skip their FMAs
    const int shape = min(4, (tk.m - sr + 3) / 4) * 5 + min(4, (tk.n - sc + 7) / 8);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    const bool split = tl.ks >= 0;
    const int ksz = (tk.flags & kTaskCrit) ? kSplitKCrit : kSplitK;
    const int kb = split ? tl.ks * ksz : 0, ke = split ? min(tk.k, kb + ksz) : tk.k;
    // operands of the next K slice are fetched into registers while the
    // current one is multiplied
    constexpr int kLd = BM * BK / 256;
    T pa[kLd], pb[kLd];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int it = 0; it < kLd; it++) {
            const int idx = threadIdx.x + it * 256, r = idx / BK, gk = k0 + idx % BK;
            pa[it] = (row0 + r < tk.m && gk < ke) ? A[(int64_t)(row0 + r) * tk.lds + gk] : T(0);
            pb[it] = (col0 + r < tk.n && gk < ke) ? B[(int64_t)(col0 + r) * tk.lds + gk] : T(0);
        }
    };
    fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int it = 0; it < kLd; it++) {
            const int idx = threadIdx.x + it * 256;
            As[idx % BK][idx / BK] = pa[it];
            Bs[idx % BK][idx / BK] = pb[it];
        }
        __syncthreads();
        if (k0 + BK < ke) fetch(k0 + BK);
        if (active) {
            const int kn = min(BK, ke - k0);
            switch (shape) {  // warp-uniform: only the row / column groups inside the task
#define SC_TILE_CASE(NI, NJ)                                                                      \
    case NI * 5 + NJ: tile_fma<T, NI, NJ, BK>(As, Bs, r0, c0, kn, acc); break;
                SC_TILE_CASE(1, 1) SC_TILE_CASE(1, 2) SC_TILE_CASE(1, 3) SC_TILE_CASE(1, 4)
                SC_TILE_CASE(2, 1) SC_TILE_CASE(2, 2) SC_TILE_CASE(2, 3) SC_TILE_CASE(2, 4)
                SC_TILE_CASE(3, 1) SC_TILE_CASE(3, 2) SC_TILE_CASE(3, 3) SC_TILE_CASE(3, 4)
                SC_TILE_CASE(4, 1) SC_TILE_CASE(4, 2) SC_TILE_CASE(4, 3)
                default: tile_fma<T, 4, 4, BK>(As, Bs, r0, c0, kn, acc); break;
#undef SC_TILE_CASE
            }
        }
        __syncthreads();
    }
    if (!active) return;
    const bool store = tk.flags & kTaskStoreU;
    const bool excl = (tk.flags & kTaskExclusive) && !split && !atomic_only;
    T *C = (store ? pool : lnz) + tk.c_off;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int gi = row0 + r0 + 4 * i;
        if (gi >= tk.m) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int gj = col0 + c0 + 8 * j;
            if (gj >= tk.n || (lower && gj > gi)) continue;
            T *c = C + (int64_t)gi * tk.ldc + gj;
            if (store) *c = -acc[i][j];
            else if (excl) *c -= acc[i][j];
            else atomicAdd(c, -acc[i][j]);
        }
    }
}

template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_gemm_tiles(T *__restrict__ lnz, T *__restrict__ pool,
                                                    const Task *__restrict__ tasks,
                                                    const GemmTile *__restrict__ tiles) {
    gemm_tile<T, BM, BN, BK>(lnz, pool, tasks, tiles[blockIdx.x], false);
}

// Tiny product tasks: one warp per task, one output entry per lane step.
// Tasks unit * 8 .. unit * 8 + 7 of the list, one per warp of a 256-thread CTA.
template <typename T>
__device__ void small_tasks(T *__restrict__ lnz, T *__restrict__ pool, const Task *__restrict__ tasks,
                            const int32_t *__restrict__ list, int32_t count, int unit) {
    int warp = unit * 8 + threadIdx.x / 32;
    int lane = threadIdx.x % 32;
    if (warp >= count) return;
    const Task tk = tasks[list[warp]];
    const bool lower = tk.flags & kTaskLower;
    const bool store = tk.flags & kTaskStoreU;
    T *C = (store ? pool : lnz) + tk.c_off;
    const int total = tk.m * tk.n;
    for (int e = lane; e < total; e += 32) {
        int i = e / tk.n, j = e % tk.n;
        if (lower && j > i) continue;
        const T *a = lnz + tk.a_off + (int64_t)i * tk.lds;
        const T *b = lnz + tk.b_off + (int64_t)j * tk.lds;
        T acc = T(0);
        for (int k = 0; k < tk.k; k++) acc += a[k] * b[k];
        if (store) C[(int64_t)i * tk.ldc + j] = -acc;
        else atomicAdd(C + (int64_t)i * tk.ldc + j, -acc);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_small_tasks(T *__restrict__ lnz, T *__restrict__ pool,
                                                     const Task *__restrict__ tasks,
                                                     const int32_t *__restrict__ list, int32_t count) {
    small_tasks<T>(lnz, pool, tasks, list, count, blockIdx.x);
}

// --------------------------------------------------------------------- K3 (device loops)
// One warp forms a block of up to NI x NJ = 32 outputs C[i][j] = sum_k A_i[k]
// B_j[k] of two row slabs of a panel (row stride ld, K columns): the lanes walk
// K (coalesced loads of NI A rows and NJ B rows per step, 32 FMAs per lane),
// then a transpose-reduction (31 shuffles) leaves output (l / NJ, l % NJ) in
// lane l, which subtracts it from C (row stride ldc) atomically where it is
// inside the block (ni x nj) and, for a lower block, on or below the diagonal
// (row i0 + i >= column j0 + j).
template <typename T, int NI>
__device__ __forceinline__ void warp_block(const T *__restrict__ A, const T *__restrict__ Bm, int64_t ld, int K,
                                           int ni, int nj, T *__restrict__ C, int64_t ldc, bool lower, int i0,
                                           int j0) {
    constexpr int NJ = 32 / NI;
    const int lane = threadIdx.x % 32;
    T v[32];
#pragma unroll
    for (int q = 0; q < 32; q++) v[q] = T(0);
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
    for (int k = lane; k < K; k += 32) {
        T a[NI], b[NJ];
#pragma unroll
        for (int i = 0; i < NI; i++) a[i] = i < ni ? A[(int64_t)i * ld + k] : T(0);
#pragma unroll
        for (int j = 0; j < NJ; j++) b[j] = j < nj ? Bm[(int64_t)j * ld + k] : T(0);
#pragma unroll
        for (int i = 0; i < NI; i++)
#pragma unroll
            for (int j = 0; j < NJ; j++) v[i * NJ + j] += a[i] * b[j];
    }
    // recursive halving: at offset o a lane keeps the half of its values whose
    // index bit o matches its own lane bit, and adds the partner's copy of it
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int q = 0; q < o; q++) {
            const T send = up ? v[q] : v[q + o];
            const T keep = up ? v[q + o] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    const int i = lane / NJ, j = lane % NJ;
    if (i < ni && j < nj && (!lower || i0 + i >= j0 + j)) atomicAdd(C + (int64_t)i * ldc + j, -v[0]);
}

// Rows x nb product C -= A B^T cut into NI x NJ warp blocks, dealt round-robin
// to the CTA's warps; `task` counts blocks across the CTA's products.
template <typename T, int NI>
__device__ __forceinline__ void warp_blocks(const T *A, const T *Bm, int64_t ld, int K, int rows, int nb, T *C,
                                            int64_t ldc, bool lower, int &task) {
    constexpr int NJ = 32 / NI;
    const int warp = threadIdx.x / 32, nwarps = blockDim.x / 32;
    for (int i0 = 0; i0 < rows; i0 += NI)
        for (int j0 = 0; j0 < nb && (!lower || j0 <= i0 + NI - 1); j0 += NJ) {
            if ((task++ % nwarps) != warp) continue;
            warp_block<T, NI>(A + (int64_t)i0 * ld, Bm + (int64_t)j0 * ld, ld, K, min(NI, rows - i0),
                              min(NJ, nb - j0), C + (int64_t)i0 * ldc + j0, ldc, lower, i0, j0);
        }
}

// Short inner dimension (K < 32, where most lanes of a warp block would idle):
// one output per thread, K-loop in registers, outputs dealt over the CTA.
template <typename T>
__device__ __forceinline__ void thread_outputs(const T *A, const T *Bm, int64_t ld, int K, int rows, int nb, T *C,
                                               int64_t ldc, bool lower) {
    const int total = rows * nb;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        if (lower && j > i) continue;
        const T *a = A + (int64_t)i * ld, *b = Bm + (int64_t)j * ld;
        T acc = T(0);
        for (int k = 0; k < K; k++) acc += a[k] * b[k];
        atomicAdd(C + (int64_t)i * ldc + j, -acc);
    }
}

template <typename T>
__device__ __forceinline__ void product_blocks(const T *A, const T *Bm, int64_t ld, int K, int rows, int nb, T *C,
                                               int64_t ldc, bool lower, int &task) {
    if (K < 32) {
        thread_outputs(A, Bm, ld, K, rows, nb, C, ldc, lower);
        return;
    }
    switch (block_rows(rows, nb, sizeof(T) == 8 ? 2 : 1, lower)) {
        case 1:
            if constexpr (sizeof(T) == 4) warp_blocks<T, 1>(A, Bm, ld, K, rows, nb, C, ldc, lower, task);
            break;
        case 2: warp_blocks<T, 2>(A, Bm, ld, K, rows, nb, C, ldc, lower, task); break;
        case 4: warp_blocks<T, 4>(A, Bm, ld, K, rows, nb, C, ldc, lower, task); break;
        default: warp_blocks<T, 8>(A, Bm, ld, K, rows, nb, C, ldc, lower, task); break;
    }
}

// Product tasks with one dimension <= kThinDim (a block B or a run B' of a few
// rows against a long panel): each CTA takes kThinWarps consecutive warp
// blocks of one task (ThinUnit), one per warp, so a long thin product spreads
// over many SMs.
constexpr int kThinDim = 8;
// Warp `wu` (0..kThinWarps-1) of thin unit u: one warp block of u's task.
template <typename T>
__device__ void thin_warp(T *__restrict__ lnz, const Task *__restrict__ tasks, const ThinUnit &u, int wu) {
    const Task tk = tasks[u.task];
    const bool lower = (tk.flags & kTaskLower) != 0;
    const int ni_min = sizeof(T) == 8 ? 2 : 1;
    const int NI = block_rows(tk.m, tk.n, ni_min, lower), NJ = 32 / NI;
    const int nbj = (tk.n + NJ - 1) / NJ, nblk = ((tk.m + NI - 1) / NI) * nbj;
    const int b = u.blk0 + wu;
    if (b >= nblk) return;
    const int i0 = (b / nbj) * NI, j0 = (b % nbj) * NJ;
    if (lower && j0 > i0 + NI - 1) return;  // wholly above the diagonal
    const T *A = lnz + tk.a_off + (int64_t)i0 * tk.lds, *Bm = lnz + tk.b_off + (int64_t)j0 * tk.lds;
    T *C = lnz + tk.c_off + (int64_t)i0 * tk.ldc + j0;
    const int ni = min(NI, tk.m - i0), nj = min(NJ, tk.n - j0);
    switch (NI) {
        case 1:
            if constexpr (sizeof(T) == 4) warp_block<T, 1>(A, Bm, tk.lds, tk.k, ni, nj, C, tk.ldc, lower, i0, j0);
            break;
        case 2: warp_block<T, 2>(A, Bm, tk.lds, tk.k, ni, nj, C, tk.ldc, lower, i0, j0); break;
        case 4: warp_block<T, 4>(A, Bm, tk.lds, tk.k, ni, nj, C, tk.ldc, lower, i0, j0); break;
        default: warp_block<T, 8>(A, Bm, tk.lds, tk.k, ni, nj, C, tk.ldc, lower, i0, j0); break;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThinWarps * 32) k_thin_tasks(T *__restrict__ lnz, const Task *__restrict__ tasks,
                                                                const ThinUnit *__restrict__ units) {
    thin_warp<T>(lnz, tasks, units[blockIdx.x], threadIdx.x / 32);
}

// Alg. 5's inner loops for a range of J's blocks, in one CTA: for each block B
// (inside ancestor P): SYRK L_{B,B} -= L_{B,J} L_{B,J}^T, then for each maximal
// run B' of blocks below B: GEMM L_{B',B} -= L_{B',J} L_{B,J}^T, both straight
// into Lnz(P) at the rows given by relindB(J,P). Products that tile_task()
// routes to the tiled kernels are skipped here. The products are cut into
// 32-output warp blocks (warp_block) dealt round-robin to the CTA's warps.
// Entries are added atomically (other supernodes of the level may update the
// same ancestor entries).
// Calls f(A, B, ld, K, rows, nb, C, ldc, lower) for every product of one loop
// item: the SYRK on B when the item starts at B, then the GEMM of each
// maximal run B' below B in the item's range.
template <typename T, typename F>
__device__ __forceinline__ void item_products(T *lnz, const LoopItem &it, const SnDev *sn, const BlkDev *blk,
                                              const int32_t *rb_val, F &&f) {
    const SnDev J = sn[it.sn];
    const int K = J.n;
    const T *src = lnz + J.off;
    const BlkDev B = blk[it.b];
    const SnDev P = sn[B.owner];
    const int colB = B.first - P.f;
    const int nb = B.size;
    const T *rowsB = src + (int64_t)B.pos * J.ld;
    if (it.r_lo == it.b)  // SYRK on B: lower triangle of L_{B,B}
        f(rowsB, rowsB, (int64_t)J.ld, K, nb, nb, lnz + P.off + (int64_t)colB * P.ld + colB, (int64_t)P.ld, true);
    int r = it.r_lo == it.b ? it.b + 1 : it.r_lo;
    while (r < it.r_hi) {
        int e = r;
        int rows = blk[r].size;
        while (e + 1 < J.b1 && blk[e + 1].first == blk[e].first + blk[e].size) {
            e++;
            rows += blk[e].size;
        }
        const int rowP = P.m - 1 - rb_val[B.rb + (r - B.bs)];
        f(src + (int64_t)blk[r].pos * J.ld, rowsB, (int64_t)J.ld, K, rows, nb,
          lnz + P.off + (int64_t)rowP * P.ld + colB, (int64_t)P.ld, false);
        r = e + 1;
    }
}

// One device-loop item by one CTA (the body of k_rlb_loop and of the per-level
// kernel's loop units).
template <typename T>
__device__ void loop_item(T *__restrict__ lnz, const LoopItem &it, const SnDev *__restrict__ sn,
                          const BlkDev *__restrict__ blk, const int32_t *__restrict__ rb_val) {
    int task = 0;
    item_products(lnz, it, sn, blk, rb_val,
                  [&](const T *A, const T *Bm, int64_t ld, int K, int rows, int nb, T *C, int64_t ldc, bool lower) {
                      product_blocks(A, Bm, ld, K, rows, nb, C, ldc, lower, task);
                  });
}

template <typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 2 : 1)) k_rlb_loop(T *__restrict__ lnz,
                                                                         const LoopItem *__restrict__ items,
                                                                         const SnDev *__restrict__ sn,
                                                                         const BlkDev *__restrict__ blk,
                                                                         const int32_t *__restrict__ rb_val) {
    loop_item<T>(lnz, items[blockIdx.x], sn, blk, rb_val);
}

// Loop items of a supernode narrower than 32 columns: one warp per item (eight
// per CTA), one output per lane with the K-loop in registers.
// Items unit * 8 .. unit * 8 + 7 of a list of narrow supernodes' items, one per warp.
template <typename T>
__device__ void loop_items_warp(T *__restrict__ lnz, const LoopItem *__restrict__ items, int count, int unit,
                                const SnDev *__restrict__ sn, const BlkDev *__restrict__ blk,
                                const int32_t *__restrict__ rb_val) {
    const int idx = unit * 8 + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (idx >= count) return;
    item_products(lnz, items[idx], sn, blk, rb_val,
                  [&](const T *A, const T *Bm, int64_t ld, int K, int rows, int nb, T *C, int64_t ldc, bool lower) {
                      for (int e = lane; e < rows * nb; e += 32) {
                          const int i = e / nb, j = e % nb;
                          if (lower && j > i) continue;
                          const T *a = A + (int64_t)i * ld, *b = Bm + (int64_t)j * ld;
                          T acc = T(0);
                          for (int k = 0; k < K; k++) acc += a[k] * b[k];
                          atomicAdd(C + (int64_t)i * ldc + j, -acc);
                      }
                  });
}

template <typename T>
__global__ void __launch_bounds__(256) k_rlb_loop_warp(T *__restrict__ lnz, const LoopItem *__restrict__ items,
                                                       int count, const SnDev *__restrict__ sn,
                                                       const BlkDev *__restrict__ blk,
                                                       const int32_t *__restrict__ rb_val) {
    loop_items_warp<T>(lnz, items, count, blockIdx.x, sn, blk, rb_val);
}

// --------------------------------------------------------------------- K4b
// RL assembly (Alg. 4, the scatter-add step): for every column c of U_J inside P and every
// row r >= c, Lnz(P)[m_P-1-relind[r]][m_P-1-relind[c]] += U_J[r][c].
template <typename T>
__global__ void k_rl_assemble(T *__restrict__ lnz, const T *__restrict__ pool, const RLPair *__restrict__ pairs,
                              const int32_t *__restrict__ relind) {
    const RLPair pr = pairs[blockIdx.y];
    const int32_t *ri = relind + pr.ri_off;  // entries for rows c_begin..s-1
    const int ncols = pr.c_end - pr.c_begin;
    const int nrows = pr.s - pr.c_begin;
    const int64_t total = (int64_t)ncols * nrows;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int cc = (int)(e / nrows), rr = (int)(e % nrows);
        if (rr < cc) continue;
        int c = pr.c_begin + cc, r = pr.c_begin + rr;
        int64_t prow = pr.mP - 1 - ri[rr];
        int64_t pcol = pr.mP - 1 - ri[cc];
        atomicAdd(lnz + pr.p_off + prow * pr.ldp + pcol, pool[pr.u_off + (int64_t)r * pr.s + c]);
    }
}

// Target-owned RL assembly (deterministic plans): the CTA owns rows [row0, row1)
// of Lnz(P) and adds into them the update matrices of P's pairs one pair after
// another, in the order of their source supernodes, with plain read-modify-
// writes; a barrier between two pairs orders the adds to an entry. The target
// row m_P-1-relind[rr] grows with rr, so the rows of a pair that land in the
// slab are one range [ra, rb), found by binary search.
template <typename T>
__global__ void __launch_bounds__(256) k_rl_assemble_ordered(T *__restrict__ lnz, const T *__restrict__ pool,
                                                             const RLPair *__restrict__ pairs,
                                                             const RLSlab *__restrict__ slabs,
                                                             const int32_t *__restrict__ relind) {
    const RLSlab sl = slabs[blockIdx.x];
    for (int32_t q = 0; q < sl.npairs; q++) {
        const RLPair pr = pairs[sl.pair0 + q];
        const int32_t *ri = relind + pr.ri_off;  // entries for rows c_begin..s-1
        const int ncols = pr.c_end - pr.c_begin;
        const int nrows = pr.s - pr.c_begin;
        // first rr whose target row is >= v: target row >= v <=> relind <= m_P-1-v
        auto first_at = [&](int32_t v) {
            int lo = 0, hi = nrows;
            while (lo < hi) {
                const int mid = (lo + hi) / 2;
                if (pr.mP - 1 - ri[mid] >= v) hi = mid;
                else lo = mid + 1;
            }
            return lo;
        };
        const int ra = first_at(sl.row0), rb = first_at(sl.row1);
        if (ra >= rb) continue;  // uniform over the CTA: no barrier needed
        const int64_t total = (int64_t)(rb - ra) * ncols;
        for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
            const int rr = ra + (int)(e / ncols), cc = (int)(e % ncols);
            if (cc > rr) continue;
            const int64_t prow = pr.mP - 1 - ri[rr];
            const int64_t pcol = pr.mP - 1 - ri[cc];
            lnz[pr.p_off + prow * pr.ldp + pcol] +=
                pool[pr.u_off + (int64_t)(pr.c_begin + rr) * pr.s + pr.c_begin + cc];
        }
        __syncthreads();
    }
}

}  // namespace sc
