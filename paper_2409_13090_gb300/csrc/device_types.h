// Plain data types shared by the host launch plan and the device kernels.
#pragma once
#include <cstdint>

#include "sc_internal.h"

namespace sc {

// Per-chunk data needed on the device.
struct ChunkDev {
    int64_t off;   // offset of the supernode's panel
    int64_t gl;    // offset of glbind(J)
    int64_t inv;   // offset of the chunk's w x w diagonal-block inverse (FP32 / TF32 factors)
    int32_t ld;    // panel leading dimension
    int32_t m;     // rows of the panel (m_J)
    int32_t c0;    // first local column of the chunk
    int32_t w;     // chunk width
    int32_t col0;  // global column of the chunk's first column
    int32_t pad;
};

// One tile of the row-wise TRSM: rows [r0, min(r0+rows, m)) of chunk c.
struct TrsmTile {
    int32_t chunk, r0;
};

// What a CTA of a persistent solve sweep takes at once: tile t0 alone (cnt 0:
// the first tile of a wide chunk), narrow tiles t0 .. t0 + cnt - 1, one per
// warp (cnt 1..8), or -cnt further tiles t0 .. t0 - cnt - 1 of one wide chunk,
// one after another (cnt -1..-solve_group, a launch-plan setting).
struct SolveUnit {
    int32_t t0, cnt;
};

// One output tile of a product task. ks < 0: the whole inner dimension;
// ks >= 0: only its slice [ks * S, (ks + 1) * S), added atomically, with
// S = kSplitKCrit for a critical task and kSplitK otherwise (SIMT tiles of
// critical tasks, and of tasks with few tiles and a long inner dimension).
struct GemmTile {
    int32_t task, tm, tn, ks;
};
constexpr int kSplitK = 256;
constexpr int kSplitKCrit = 32;  // slice width of split critical tasks (kTaskCrit)

// Work of one CTA of the thin-product kernel: warp blocks blk0 .. blk0 + 3 of
// a task (blocks numbered row-major over the task's NI x NJ block grid).
struct ThinUnit {
    int32_t task, blk0;
};
constexpr int kThinWarps = 4;

// Warp-block shape for a rows x nb product: the NI in {ni_min, ..., 8}
// (powers of two; NJ = 32 / NI) with the fewest blocks, ties to the smaller
// NI + NJ (fewer loads per step). Lower (triangular) products use 4 x 8.
SC_HD inline int block_rows(int rows, int nb, int ni_min, bool lower) {
    if (lower) return 4;
    int best = ni_min, bestn = 1 << 30;
    for (int ni = ni_min; ni <= 8; ni *= 2) {
        const int nj = 32 / ni;
        const int cnt = ((rows + ni - 1) / ni) * ((nb + nj - 1) / nj);
        if (cnt < bestn || (cnt == bestn && ni + nj < best + 32 / best)) {
            best = ni;
            bestn = cnt;
        }
    }
    return best;
}

constexpr int kMaxChunk = 64;

// Supernode descriptor for the device-side RLB loops.
struct SnDev {
    int64_t off;  // offset of Lnz(J)
    int32_t ld;   // leading dimension of Lnz(J)
    int32_t m;    // m_J = |glbind(J)|
    int32_t f;    // first column
    int32_t n;    // |J|
    int32_t b1;   // one past J's last block
    int32_t pad;
};

// Block descriptor (Sec. 1 / Alg. 5): rows pos..pos+size-1 of Lnz(J) hold the
// global rows first..first+size-1, which are columns of supernode owner.
// relindB(J, owner) starts at rb_val[rb] and covers J's blocks bs.. onward.
struct BlkDev {
    int32_t pos, size, first, owner;
    int64_t rb;
    int32_t bs, pad;
};

constexpr int kLoopSmemBytes = 48 * 1024;

// Target-owned RL assembly (deterministic plans): rows [row0, row1) of Lnz(P)
// receive the update matrices of pairs pair0 .. pair0 + npairs - 1 (all with
// target P, in the order of their source supernodes) from one CTA.
struct RLSlab {
    int32_t pair0, npairs, row0, row1;
};
constexpr int kRLSlabRows = 64;

// One unit of the per-level persistent kernel (k_level): a POTRF of a chunk, a
// TRSM tile, a product tile, one or two thin units, up to eight small tasks, a
// device-loop item or up to eight narrow loop items. idx indexes the list of
// its kind (for small tasks and narrow loop items: the first of cnt entries).
struct FlowUnit {
    int32_t kind, idx, cnt, pad;
};
enum : int32_t { kFlowPotrf = 0, kFlowTrsm, kFlowGemm, kFlowThin, kFlowSmall, kFlowLoop, kFlowLoopW };
// one counter word per 128-byte line in the per-chunk arrays of k_level
constexpr int kFlowStride = 32;

}  // namespace sc
