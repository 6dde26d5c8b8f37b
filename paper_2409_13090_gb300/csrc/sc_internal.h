// Internal data structures of libsc shared by the host analysis and the CUDA
// numeric path. Not part of the C ABI (include/sc.h is).
#pragma once
#include <atomic>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sc.h"
#include <nvtx3/nvToolsExt.h>

namespace sc {

// Update task C[m x n] -= A[m x k] * B[n x k]^T on row-major panels.
// A and B are row slabs of one source panel (leading dimension lds);
// C is a dense block of the target panel (leading dimension ldc).
// Offsets are element indices into the factor storage Lnz (or the RL pool
// for C when kTaskStoreU is set).
struct Task {
    int64_t a_off, b_off, c_off;
    int32_t lds, ldc, m, n, k, flags;
    int32_t src;    // source supernode J
    int32_t a_row;  // first row of A in Lnz(J)
    int32_t b_row;  // first row of B in Lnz(J)
    int32_t kx0;    // first column of A and B in Lnz(J)
    int32_t tcol;   // global column of C's first column (its chunk decides kTaskCrit)
};
enum : int32_t {
    kTaskLower = 1,      // only entries with local row >= local column are written
    kTaskStoreU = 2,     // C is an RL update matrix: C = -A B^T (plain store, no accumulate)
    kTaskExclusive = 4,  // no other task of the level writes C: plain read-modify-write
    kTaskCrit = 8,       // C lies in a chunk of the next level: must finish before that level
};

#ifdef __CUDACC__
#define SC_HD __host__ __device__
#else
#define SC_HD
#endif

// Which RLB products run as tiled GEMMs (the rest run inside the device loop
// over J's blocks). entries = outputs of the product, k = inner dimension.
SC_HD inline bool tile_task(long long entries, int k, int min_entries, int min_k) {
    return (entries >= min_entries && k >= min_k) || entries >= 8LL * min_entries;
}

// Launch-plan settings of sc_tune_table with the defaults filled in.
struct Knobs {
    int tile_min_entries = 1024, tile_min_k = 16, loop_budget = 1 << 15;
    bool lookahead = true;
    int tc_min_k = 32, tc_wide_n = 96, thin_dim = 8;
    int defer_width = 512;
    bool fused = false;
    int tc_wide256 = 256;
    int solve_group = 0;  // 0: by the factor's precision (2 FP64, 4 FP32)
    bool tc_multicast = true;
};
inline Knobs knobs_of(const sc_tune_table &t) {
    Knobs k;
    if (t.tile_min_entries) k.tile_min_entries = t.tile_min_entries;
    if (t.tile_min_k) k.tile_min_k = t.tile_min_k;
    if (t.loop_budget) k.loop_budget = t.loop_budget;
    if (t.lookahead) k.lookahead = t.lookahead > 0;
    if (t.tc_min_k) k.tc_min_k = t.tc_min_k;
    if (t.tc_wide_n) k.tc_wide_n = t.tc_wide_n;
    if (t.thin_dim) k.thin_dim = t.thin_dim < 0 ? 0 : t.thin_dim;
    if (t.defer_width) k.defer_width = t.defer_width;
    if (t.fused) k.fused = t.fused > 0;
    if (t.tc_wide256) k.tc_wide256 = t.tc_wide256;
    if (t.solve_group) k.solve_group = t.solve_group;
    if (t.tc_multicast) k.tc_multicast = t.tc_multicast > 0;
    return k;
}
// Inner-dimension granularity of one tcgen05.mma of kind::tf32 (K = 8): the
// tensor-core tile consumes the columns [kx0, kx0 + round_up(k, kTcKStep)) of
// its source panel.
constexpr int kTcKStep = 8;

// Tile width of a product on the tensor cores: 128 or 64 columns (the launch
// plan widens a 128 to 256 for n >= the tc_wide256 setting), or 0 when the
// product stays on the SIMT units. Needs a tensor map of the source panel
// (src_width = |J| >= 16: 16-byte row stride), K >= 32 and m >= 64; min_k
// (>= 32) and wide_n (>= 16) are the plan's thresholds. The tile consumes K in
// steps of kTcKStep columns, so a K that is not a multiple of it is allowed
// only where the product's columns end at the panel's last real column (the
// columns after it are zero padding or outside the tensor map, read as zero):
// elsewhere the step would multiply the next columns of the panel in.
// ignore_tail (a test hook only) drops that condition. The tile's TMA loads
// start at column kx0, which must be 16-byte aligned (kx0 % 4 == 0); the
// schedule gives every K >= 32 product a kx0 that is a multiple of its K or 0,
// so this holds for every routed product, and the rule keeps it so.
inline int tc_route_width(const Task &t, int src_width, int min_k, int wide_n, bool ignore_tail = false) {
    if (src_width < 16 || t.k < 32 || t.k < min_k || t.m < 64 || (t.flags & kTaskStoreU)) return 0;
    if (t.kx0 % 4 != 0) return 0;
    if (!ignore_tail && t.k % kTcKStep != 0 && t.kx0 + t.k < src_width) return 0;
    if (t.n >= wide_n && t.n >= 16) return 128;
    if (t.n >= 16) return 64;
    return 0;
}

// Field ranges of sc_tune_table (0 = default everywhere).
inline bool tune_valid(const sc_tune_table &t) {
    auto in = [](int32_t v, int32_t lo, int32_t hi) { return v == 0 || (v >= lo && v <= hi); };
    return in(t.tile_min_entries, 1, 1 << 24) && in(t.tile_min_k, 1, 1 << 16) && in(t.loop_budget, 256, 1 << 28) &&
           (t.lookahead >= -1 && t.lookahead <= 1) && in(t.tc_min_k, 32, 1 << 16) && in(t.tc_wide_n, 16, 1 << 16) &&
           (t.thin_dim == -1 || in(t.thin_dim, 1, 8)) && in(t.defer_width, 256, 1 << 20) &&
           (t.fused >= -1 && t.fused <= 1) && in(t.tc_wide256, 16, 1 << 20) &&
           in(t.solve_group, 1, 1024) && (t.tc_multicast >= -1 && t.tc_multicast <= 1);
}

// Part of Alg. 5's inner loops for one block B of supernode J, run on the
// device by one CTA: the SYRK on B when r_lo == b, then the GEMMs of the
// maximal runs B' below B that start at block indices in [max(r_lo, b+1), r_hi).
struct LoopItem {
    int32_t sn;    // J
    int32_t b;     // block B (global block index)
    int32_t r_lo;  // b: include the SYRK on B; otherwise the first run start
    int32_t r_hi;  // runs starting at block indices below r_hi
};

// One panel of at most `chunk` columns of a supernode; the unit of the dense
// work (POTRF, TRSM) and of the level schedule.
struct Chunk {
    int32_t sn;   // supernode
    int32_t c0;   // first local column
    int32_t w;    // columns
    int32_t last; // 1 if this is the supernode's last chunk
};

// RL assembly of U_J's columns lying in ancestor P (Alg. 4, the scatter-add step).
struct RLPair {
    int64_t u_off;      // offset of U_J in the pool (row-major, ld = s)
    int64_t p_off;      // offset of Lnz(P)
    int64_t ri_off;     // offset into rl_relind of relind(J,P) for rows c_begin..s-1
    int32_t s;          // |S_J|
    int32_t c_begin;    // first row/column of U_J inside P
    int32_t c_end;      // one past the last column of U_J inside P
    int32_t ldp, mP, fP;
    int32_t pad;
};

struct Level {
    std::vector<int32_t> chunks;       // chunks factored at this level
    std::vector<int32_t> last_chunks;  // of which: the last chunk of their supernode
    std::vector<Task> tasks;           // tiled products: large RLB updates + intra-supernode trailing updates
    std::vector<LoopItem> loops;       // device-side RLB loops (the remaining products)
    std::vector<Task> rl_tasks;        // RL: U_J products (variant RL only)
    std::vector<RLPair> rl_pairs;      // RL: assembly work (variant RL only)
    int64_t rl_pool = 0;               // RL: pool elements needed by this level
    double loop_flops = 0;             // algorithmic flops of the device loops
};

}  // namespace sc

struct sc_symbolic {
    int64_t n = 0;
    sc_options opt{};      // opt.tune is not kept (NULL); the table is copied into `tune`
    sc_tune_table tune{};  // launch-plan settings (zero fields = defaults)
    // input pattern (lower, CSC) as given
    std::vector<int64_t> colptr;
    std::vector<int32_t> rowind;
    // final ordering
    std::vector<int32_t> perm, iperm, cparent;
    // supernodal structure
    int64_t nsuper = 0;
    std::vector<int32_t> sup_ptr, sup_parent, level;
    std::vector<int64_t> gl_ptr;
    std::vector<int32_t> glbind;
    std::vector<int64_t> ri_ptr;
    std::vector<int32_t> relind;
    std::vector<int64_t> blk_ptr;
    std::vector<int32_t> blk_first, blk_size, blk_owner;
    std::vector<int64_t> rb_pair_ptr;
    std::vector<int32_t> rb_pair_P;
    std::vector<int64_t> rb_val_ptr;
    std::vector<int32_t> rb_val;
    int64_t nnzL = 0;
    double flops = 0.0;
    // factor storage layout: supernode J occupies m_J rows x ld_J at element offset lnz_off[J]
    std::vector<int64_t> lnz_off;
    std::vector<int32_t> lnz_ld;
    int64_t lnz_size = 0;
    std::vector<int64_t> valmap;  // A entry p -> element offset in Lnz
    std::vector<int32_t> sup_of;  // column -> supernode
    // device schedule (precision independent)
    std::vector<sc::Chunk> chunks;
    std::vector<sc::Level> levels;
    std::vector<int32_t> chunk_of_col;  // column -> chunk
    std::vector<int32_t> rl_relind;     // RL: composed relind(J,P) lists
    int64_t rl_pool_max = 0;
    // full symmetric CSR of A in the caller's ordering (for the FP64 residual)
    std::vector<int64_t> csr_ptr;
    std::vector<int32_t> csr_col;
    std::vector<int64_t> csr_map;  // CSR entry -> index into values
    double anorm_inf_pattern = 0;  // unused placeholder
    std::atomic<int> refs{0};
    bool poisoned = false;  // a test hook altered the schedule: never factored
    bool test_tc_ignore_tail = false;  // test hook: tensor-core routing without the K-tail rule
    bool test_det_short_slab = false;  // test hook: a deterministic plan's first level of slabs misses a row
};

namespace sc {
// NVTX range over one library call: the phases show up in a profiler's
// timeline; without a tool attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
int analyze_impl(int64_t n, const int64_t *colptr, const int32_t *rowind, const sc_options &o,
                 sc_symbolic **out);
int build_schedule(sc_symbolic *s);
// Violation kind of the launch plans of a deterministic schedule (0 if none;
// the level in *bad_level): a product tile split along the inner dimension, or
// a target row of an RL assembly pair not owned by exactly one slab of its
// target, or a slab whose pairs are not one target's in source order.
int det_plan_check(const sc_symbolic *s, int64_t *bad_level);
int compose_relind(const int32_t *rJC, int64_t lenJC, const int32_t *rCP, int64_t lenCP, int32_t *out);
}  // namespace sc
