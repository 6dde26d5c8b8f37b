// Tensor-core product tiles for SC_TF32 (sm_103a): C[128 x BN tile] -= A B^T
// with A, B row slabs of one FP32 supernode panel, TF32 inputs, FP32 accumulate.
//
// Persistent, warp-specialised kernel (one or two CTAs per SM, looping over the
// level's tiles):
//   warp 0  producer: TMA loads (cp.async.bulk.tensor, 128-byte swizzle, tensor
//           maps per source panel held in global memory) into a 4-stage ring;
//   warp 1  MMA issuer: tcgen05.mma.cta_group::1.kind::tf32 (M = 128, N = BN,
//           K = 8) into one of two TMEM accumulators; tcgen05.commit frees ring
//           stages and hands finished accumulators to the epilogue;
//   warps 2-9 epilogue: tcgen05.ld of 32 lanes x half the columns each, subtract into the target
//           block of Lnz(P) (plain read-modify-write for an exclusive target,
//           a no-return reduction otherwise; 16-byte vectors when aligned), then release
//           the accumulator -- so one tile's epilogue overlaps the next tile's
//           loads and MMAs.
// Operands are K-major: a panel row is contiguous along the supernode's
// columns, the inner (K) dimension of every update product.
// Every wait is bounded by spin_limit polls; on expiry the kernel sets *err and
// the roles stop; TMEM is freed before the CTA exits.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include <vector>

#include "kernels.cuh"

namespace sc {
namespace tc {

constexpr int BM = 128, BK = 32;  // BK fp32 = 128 bytes = one swizzle row
constexpr int A_BYTES = BM * BK * 4;

constexpr int kEpiWarps = 8;                 // two per TMEM lane quarter, each half of the columns
constexpr int kThreads = 32 * (2 + kEpiWarps);  // producer warp, MMA warp, epilogue warps

// X3: the three-product split form (SC_TF32X3): a stage holds hi and lo tiles
// of A and B (A_hi, A_lo, B_hi, B_lo), and each K step issues hi*hi, hi*lo,
// lo*hi into the same accumulator.
// BN = 256: half the shared-memory operand reads per flop of A (each A row
// meets 256 B rows per MMA); a stage is 48 KB (96 KB for X3), so X3 keeps two
// stages, and the two accumulators fill the SM's 512 TMEM columns.
template <int BN, bool X3>
struct Cfg {
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int NSPLIT = X3 ? 2 : 1;
    static constexpr int STAGES = X3 ? (BN == 256 ? 2 : 3) : 4;
    static constexpr int STAGE_BYTES = NSPLIT * (A_BYTES + B_BYTES);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*alignment*/ + 256 /*barriers*/;
    static constexpr int TMEM_COLS = 2 * BN;  // two accumulators
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
    // 512 columns: no other tensor-core CTA fits beside this one's shared memory, so the
    // allocation never waits for another CTA's columns
    static_assert(TMEM_COLS <= 512, "TMEM columns per SM");
    static constexpr int CTAS_PER_SM = (BN == 64 && !X3) ? 2 : 1;
    // instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = BN
    static constexpr uint32_t IDESC =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and *err set) when spin_limit polls pass without completion
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long spin_limit, int32_t *err,
                                          int code) {
    for (long long i = 0; i < spin_limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, code);
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// the same load delivered to the same shared-memory offset, and its bytes counted
// on the barrier at the same offset, in every CTA of the cluster in `mask`
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster (release / acquire)
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // swizzle mode: 128 B
    return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// one arrival, when this CTA's MMAs issued so far complete, on the barrier at
// offset `bar` of every CTA of the cluster in `mask`
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::
                     "r"(bar),
                 "h"(mask)
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// no-return reductions into the target (the epilogue never needs the old value)
__device__ __forceinline__ void red_sub4(float *p, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(-a), "f"(-b), "f"(-c),
                 "f"(-d)
                 : "memory");
}
__device__ __forceinline__ void red_sub(float *p, float a) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(-a) : "memory");
}

// C row segment -= v[0..32) for columns gj0..gj0+31 of row gi (masked at n, and
// to j <= gi for a lower task). For an exclusive target with an aligned full
// segment, the caller has already loaded the old values into c (prefetch).
__device__ __forceinline__ bool seg_vec(int gi, int gj0, int n, bool lower, bool vec) {
    return vec && gj0 + 32 <= n && (!lower || gj0 + 31 <= gi);
}
__device__ __forceinline__ void epilogue_row(float *__restrict__ crow, const float (&v)[32], const float4 (&c)[8],
                                             int gi, int gj0, int n, bool lower, bool excl, bool vec) {
    if (seg_vec(gi, gj0, n, lower, vec)) {
        float4 *c4 = reinterpret_cast<float4 *>(crow + gj0);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (excl) {
                c4[q] = make_float4(c[q].x - v[4 * q], c[q].y - v[4 * q + 1], c[q].z - v[4 * q + 2],
                                    c[q].w - v[4 * q + 3]);
            } else {
                red_sub4(reinterpret_cast<float *>(c4 + q), v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 32; j++) {
        const int gj = gj0 + j;
        if (gj < n && (!lower || gj <= gi)) {
            if (excl) crow[gj] -= v[j];
            else red_sub(crow + gj, v[j]);
        }
    }
}

// Shared memory of stage s: A tiles (hi, then lo for X3) of all stages first,
// then B tiles; every tile starts on a 1024-byte boundary (the swizzle atom).
template <int BN, bool X3>
__device__ __forceinline__ uint32_t a_tile(const unsigned char *smem, int s, int part) {
    return smem_u32(smem + (s * Cfg<BN, X3>::NSPLIT + part) * A_BYTES);
}
template <int BN, bool X3>
__device__ __forceinline__ uint32_t b_tile(const unsigned char *smem, int s, int part) {
    using C = Cfg<BN, X3>;
    return smem_u32(smem + C::STAGES * C::NSPLIT * A_BYTES + (s * C::NSPLIT + part) * C::B_BYTES);
}

// CL = 2 (BN = 256 only): clusters of two CTAs take the two tiles of a pair
// (vertically adjacent tiles of one product and column block; the plan lists
// them in pairs, the second possibly one that writes nothing). Each CTA loads
// its own A tiles and one 128-row half of the B tiles, multicast to both CTAs,
// so a stage costs each SM 64 KB of loads instead of 96 KB (X3). A stage is
// refilled only when the MMAs of both CTAs are done with it (its empty barrier
// counts both CTAs' commits); the CTAs start after a cluster barrier that
// follows the barrier set-up, and leave after every commit of the partner has
// reached them and a second cluster barrier.
template <int BN, bool X3, int CL = 1>
__global__ void __launch_bounds__(kThreads, (Cfg<BN, X3>::CTAS_PER_SM))
    k_tc_gemm(float *__restrict__ lnz, const Task *__restrict__ tasks, const GemmTile *__restrict__ tiles, int ntiles,
              const CUtensorMap *__restrict__ tmaps, int lo_maps, const int32_t *__restrict__ tmap_of_sn,
              int32_t *__restrict__ err, long long spin_limit) {
    using C = Cfg<BN, X3>;
    constexpr int STAGES = C::STAGES;
    static_assert(CL == 1 || (CL == 2 && BN == 256), "clusters of two take 256-column tiles");
    const int rank = CL == 2 ? (int)cluster_rank() : 0;
    // this CTA's first tile and its stride: pairs go to clusters, tile 2p + rank to rank
    const int t_first = CL == 2 ? 2 * ((int)blockIdx.x / 2) + rank : (int)blockIdx.x;
    const int t_step = (int)gridDim.x;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE_BYTES);
    uint64_t *full = bars, *empty = bars + STAGES, *accf = bars + 2 * STAGES, *acce = bars + 2 * STAGES + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 4);
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; s++) mbar_init(smem_u32(full + s), 1);
        for (int s = 0; s < STAGES; s++) mbar_init(smem_u32(empty + s), CL);  // one commit per CTA of the cluster
        for (int a = 0; a < 2; a++) {
            mbar_init(smem_u32(accf + a), 1);  // one tcgen05.commit per tile
            mbar_init(smem_u32(acce + a), kEpiWarps);  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();  // thread 0 rejoins warp 0 before the warp-collective allocation
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    if constexpr (CL == 2) cluster_sync();  // the partner's barriers exist before any multicast
    fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            uint32_t g = 0;
            for (int t = t_first; t < ntiles && !abort_flag; t += t_step) {
                const GemmTile tl = tiles[t];
                const Task tk = tasks[tl.task];
                const int mi = tmap_of_sn[tk.src];
                const CUtensorMap *amap = tmaps + 2 * mi;
                const CUtensorMap *bmap = tmaps + 2 * mi + (BN == 64 ? 1 : 0);  // 128-row boxes (two for BN = 256)
                const int nk = (tk.k + BK - 1) / BK;
                const int ay = tk.a_row + tl.tm * BM, by = tk.b_row + tl.tn * BN;
                for (int kb = 0; kb < nk; kb++, g++) {
                    const int s = g % STAGES;
                    const uint32_t ph = (g / STAGES) & 1u;
                    if (g >= STAGES && !mbar_wait(smem_u32(empty + s), ph ^ 1u, spin_limit, err, 1)) {
                        abort_flag = 1;
                        break;
                    }
                    const uint32_t fb = smem_u32(full + s);
                    mbar_expect_tx(fb, C::STAGE_BYTES);
                    const int x = tk.kx0 + kb * BK;
                    // a 256-row B tile is two 128-row boxes: with the 128-byte swizzle, rows
                    // sit in 1024-byte groups of 8, so the second box continues the first's layout
                    for (int part = 0; part < C::NSPLIT; part++) {
                        const CUtensorMap *ap = amap + 2 * lo_maps * part, *bp = bmap + 2 * lo_maps * part;
                        tma_load_2d(a_tile<BN, X3>(smem, s, part), ap, x, ay, fb);
                        if constexpr (CL == 2) {
                            // this CTA's half of B, into both CTAs
                            tma_load_2d_mc(b_tile<BN, X3>(smem, s, part) + rank * 128 * BK * 4, bp, x, by + 128 * rank,
                                           fb, (uint16_t)0x3);
                        } else {
                            tma_load_2d(b_tile<BN, X3>(smem, s, part), bp, x, by, fb);
                            if constexpr (BN == 256)
                                tma_load_2d(b_tile<BN, X3>(smem, s, part) + 128 * BK * 4, bp, x, by + 128, fb);
                        }
                    }
                }
            }
            if constexpr (CL == 2) {
                // the last use of every stage released by both CTAs: the partner's
                // commits have all reached this CTA's barriers, and its MMAs have read
                // every multicast piece
                for (uint32_t u = g > (uint32_t)STAGES ? g - STAGES : 0; u < g; u++)
                    if (!mbar_wait(smem_u32(empty + u % STAGES), (u / STAGES) & 1u, spin_limit, err, 5)) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            uint32_t g = 0;
            int i = 0;
            for (int t = t_first; t < ntiles && !abort_flag; t += t_step, i++) {
                const Task tk = tasks[tiles[t].task];
                const int nk = (tk.k + BK - 1) / BK;
                const int a = i & 1, u = i >> 1;
                if (u > 0 && !mbar_wait(smem_u32(acce + a), (uint32_t)(u - 1) & 1u, spin_limit, err, 2)) {
                    abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t td = tmem + (uint32_t)(a * BN);
                for (int kb = 0; kb < nk; kb++, g++) {
                    const int s = g % STAGES;
                    const uint32_t ph = (g / STAGES) & 1u;
                    if (!mbar_wait(smem_u32(full + s), ph, spin_limit, err, 3)) {
                        abort_flag = 1;
                        break;
                    }
                    fence_after();
                    const uint32_t a0 = a_tile<BN, X3>(smem, s, 0), b0 = b_tile<BN, X3>(smem, s, 0);
                    // the box holds BK columns; only the 8-column steps inside K are
                    // multiplied (the columns after K in the box belong to other work)
                    const int ksteps = min(BK / kTcKStep, (tk.k - kb * BK + kTcKStep - 1) / kTcKStep);
#pragma unroll
                    for (int kk = 0; kk < BK / 8; kk++) {  // 8 tf32 = 32 bytes along K inside the swizzle row
                        if (kk >= ksteps) break;
                        if constexpr (X3) {
                            // small terms first: lo*hi, hi*lo, then hi*hi
                            const uint32_t a1 = a_tile<BN, X3>(smem, s, 1), b1 = b_tile<BN, X3>(smem, s, 1);
                            mma_tf32(td, umma_desc_sw128(a1 + kk * 32), umma_desc_sw128(b0 + kk * 32), C::IDESC,
                                     (kb > 0 || kk > 0) ? 1u : 0u);
                            mma_tf32(td, umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b1 + kk * 32), C::IDESC, 1u);
                            mma_tf32(td, umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b0 + kk * 32), C::IDESC, 1u);
                        } else {
                            mma_tf32(td, umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b0 + kk * 32), C::IDESC,
                                     (kb > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    // frees ring stage s (in both CTAs of a cluster) when these MMAs finish
                    if constexpr (CL == 2) mma_commit_mc(smem_u32(empty + s), (uint16_t)0x3);
                    else mma_commit(smem_u32(empty + s));
                }
                mma_commit(smem_u32(accf + a));  // accumulator a complete
            }
        }
    } else {
        // epilogue warps 2..9: TMEM lanes 32*(warp % 4) .. +31, column half (warp - 2) / 4
        const int quarter = warp % 4, half = (warp - 2) / 4;
        int i = 0;
        for (int t = t_first; t < ntiles; t += t_step, i++) {
            const GemmTile tl = tiles[t];
            const Task tk = tasks[tl.task];
            const int gi = tl.tm * BM + quarter * 32 + lane;
            const bool lower = tk.flags & kTaskLower;
            const bool excl = tk.flags & kTaskExclusive;
            const bool vec = (tk.ldc % 4 == 0) && (tk.c_off % 4 == 0);
            float *crow = lnz + tk.c_off + (int64_t)gi * tk.ldc;
            const int a = i & 1, u = i >> 1;
            const bool ok = mbar_wait(smem_u32(accf + a), (uint32_t)u & 1u, spin_limit, err, 4);
            if (!__all_sync(0xffffffffu, ok && !abort_flag)) break;
            fence_after();
#pragma unroll 1
            for (int cc = half * (BN / 64); cc < (half + 1) * (BN / 64); cc++) {
                const int gj0 = tl.tn * BN + cc * 32;
                // issue the target's loads before the accumulator read so their latencies overlap
                float4 c[8];
                const bool pre = excl && gi < tk.m && seg_vec(gi, gj0, tk.n, lower, vec);
                if (pre) {
                    const float4 *c4 = reinterpret_cast<const float4 *>(crow + gj0);
#pragma unroll
                    for (int q = 0; q < 8; q++) c[q] = c4[q];
                }
                float v[32];
                tmem_ld32(tmem + (uint32_t)(a * BN) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cc * 32), v);
                if (gi < tk.m) epilogue_row(crow, v, c, gi, gj0, tk.n, lower, excl, vec);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acce + a));
        }
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    if constexpr (CL == 2) cluster_sync();  // no multicast or commit is still on its way to this CTA
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

}  // namespace tc

// ---------------------------------------------------------------- host side
inline bool tc_gemm_init() {
    using namespace tc;
    return cudaFuncSetAttribute(k_tc_gemm<256, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<256, false>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<256, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<256, true>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<256, false>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<256, true>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<128, false>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<64, false>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<128, true>::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(k_tc_gemm<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<64, true>::SMEM) == cudaSuccess;
}

// Tile width for a product on the tensor cores (tc_route_width): a source panel
// without a tensor map stays on the SIMT units.
inline int tc_width(const Task &t, const std::vector<int32_t> &tmap_of_sn, int src_width, int min_k, int wide_n,
                    bool ignore_tail) {
    if (tmap_of_sn[t.src] < 0) return 0;
    return tc_route_width(t, src_width, min_k, wide_n, ignore_tail);
}

// 256-column tiles for clusters of two: per column block, the row tiles in
// pairs (2p, 2p + 1); a pair whose second (or first) tile does not exist gets
// it anyway -- past the product's rows, or above the diagonal of a lower
// product -- and that tile's epilogue writes nothing.
inline void tc_tile_pairs_of(const Task &t, int32_t id, std::vector<GemmTile> &out) {
    const int tm = (t.m + tc::BM - 1) / tc::BM, tn = (t.n + 255) / 256;
    auto live = [&](int i, int j) { return i < tm && !((t.flags & kTaskLower) && (i * tc::BM + tc::BM - 1) < j * 256); };
    for (int j = 0; j < tn; j++)
        for (int i = 0; i < tm; i += 2)
            if (live(i, j) || live(i + 1, j)) {
                out.push_back(GemmTile{id, i, j, -1});
                out.push_back(GemmTile{id, i + 1, j, -1});
            }
}

inline void tc_tiles_of(const Task &t, int32_t id, int bn, std::vector<GemmTile> &out) {
    int tm = (t.m + tc::BM - 1) / tc::BM, tn = (t.n + bn - 1) / bn;
    for (int i = 0; i < tm; i++)
        for (int j = 0; j < tn; j++) {
            if ((t.flags & kTaskLower) && (i * tc::BM + tc::BM - 1) < j * bn) continue;
            out.push_back(GemmTile{id, i, j, -1});
        }
}

// Encodes two 2D tensor maps per panel of width >= 16 (dims {ld_J, m_J}, boxes
// {32, 128} and {32, 64}, 128-byte swizzle, zero fill outside the panel):
// maps[2 * tmap_of_sn[J]] and maps[2 * tmap_of_sn[J] + 1].
inline int tc_encode_maps(const sc_symbolic *s, float *d_lnz, std::vector<CUtensorMap> &maps,
                          std::vector<int32_t> &tmap_of_sn) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return SC_ERR_CUDA;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    tmap_of_sn.assign(s->nsuper, -1);
    maps.clear();
    for (int64_t J = 0; J < s->nsuper; J++) {
        int32_t w = s->sup_ptr[J + 1] - s->sup_ptr[J];
        if (w < 16) continue;
        int64_t m = s->gl_ptr[J + 1] - s->gl_ptr[J];
        tmap_of_sn[J] = (int32_t)(maps.size() / 2);
        for (int rows : {tc::BM, 64}) {
            CUtensorMap map;
            cuuint64_t dims[2] = {(cuuint64_t)s->lnz_ld[J], (cuuint64_t)m};
            cuuint64_t strides[1] = {(cuuint64_t)s->lnz_ld[J] * 4};
            cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)rows};
            cuuint32_t estr[2] = {1, 1};
            CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(d_lnz + s->lnz_off[J]), dims,
                                strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return SC_ERR_CUDA;
            maps.push_back(map);
        }
    }
    return SC_OK;
}

// Launches the persistent kernel over `count` tiles of width bn; x3 selects
// the three-product split form (maps[2 * nmaps ...] are then the lo maps).
template <int BN, bool X3>
inline void launch_tc(float *lnz, const Task *tasks, const GemmTile *tiles, int32_t count, const CUtensorMap *maps,
                      int nmaps, const int32_t *tmap_of_sn, int32_t *err, long long spin_limit, int num_sms,
                      cudaStream_t st) {
    using C = tc::Cfg<BN, X3>;
    const int grid = std::min<int>(count, num_sms * C::CTAS_PER_SM);
    tc::k_tc_gemm<BN, X3><<<grid, tc::kThreads, C::SMEM, st>>>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err,
                                                               spin_limit);
}
// Clusters of two over `count` paired tiles (count even): as many clusters as
// fit on the device at once (fewer if there are fewer pairs).
template <bool X3>
inline void launch_tc_pairs(float *lnz, const Task *tasks, const GemmTile *tiles, int32_t count,
                            const CUtensorMap *maps, int nmaps, const int32_t *tmap_of_sn, int32_t *err,
                            long long spin_limit, int num_sms, cudaStream_t st) {
    using C = tc::Cfg<256, X3>;
    static int max_clusters_of[64] = {};  // per device ordinal
    int dev = 0;
    cudaGetDevice(&dev);
    int &max_clusters = max_clusters_of[dev & 63];
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2, at[0].val.clusterDim.y = 1, at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(tc::kThreads);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (!max_clusters) {
        cfg.gridDim = dim3((unsigned)(num_sms / 2 * 2));
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc::k_tc_gemm<256, X3, 2>, &cfg) != cudaSuccess || n < 1) n = num_sms / 2;
        max_clusters = n;
    }
    cfg.gridDim = dim3((unsigned)(2 * std::min<int>(count / 2, max_clusters)));
    cudaLaunchKernelEx(&cfg, tc::k_tc_gemm<256, X3, 2>, lnz, tasks, tiles, (int)count, maps, nmaps, tmap_of_sn, err,
                       spin_limit);
}
inline void launch_tc_gemm(int bn, bool x3, float *lnz, const Task *tasks, const GemmTile *tiles, int32_t count,
                           const CUtensorMap *maps, int nmaps, const int32_t *tmap_of_sn, int32_t *err,
                           long long spin_limit, int num_sms, cudaStream_t st, bool pairs = false) {
    if (bn == 256 && pairs) {
        if (x3) launch_tc_pairs<true>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
        else launch_tc_pairs<false>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
    } else if (bn == 256) {
        if (x3) launch_tc<256, true>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
        else launch_tc<256, false>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
    } else if (bn == 128) {
        if (x3) launch_tc<128, true>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
        else launch_tc<128, false>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
    } else {
        if (x3) launch_tc<64, true>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
        else launch_tc<64, false>(lnz, tasks, tiles, count, maps, nmaps, tmap_of_sn, err, spin_limit, num_sms, st);
    }
}

}  // namespace sc
