// Numeric handle of libsc: device buffers and the launch plan of one
// factorization (factor.cu) and of the solve (solve.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "device_types.h"
#include "sc_internal.h"

namespace sc {

// The product launches of one level that share a dependency class.
struct ProdLists {
    int32_t gemm_off = 0, gemm_cnt = 0;     // GemmTile (SIMT)
    int32_t tc_off = 0, tc_cnt = 0;         // GemmTile (tensor cores, 128-column tiles)
    int32_t tc64_off = 0, tc64_cnt = 0;     // GemmTile (tensor cores, 64-column tiles)
    int32_t tc256_off = 0, tc256_cnt = 0;   // GemmTile (tensor cores, 256-column tiles)
    int32_t thin_off = 0, thin_cnt = 0;     // ThinUnits of tasks with min(m, n) <= 8 (warp-block kernel)
    bool any() const { return gemm_cnt || tc_cnt || tc64_cnt || tc256_cnt || thin_cnt; }
};

// Launch plan of one level: offsets/counts into the flat device work lists.
// With lookahead, `crit` holds the products into chunks of the next level and
// `rest` the others, which may run concurrently with the next level.
struct LevelPlan {
    int32_t potrf_off = 0, potrf_cnt = 0;   // chunk ids
    int32_t trsm_off = 0, trsm_cnt = 0;     // TrsmTile
    ProdLists crit, rest;
    int32_t small_off = 0, small_cnt = 0;   // task ids (warp kernel)
    int32_t rlg_off = 0, rlg_cnt = 0;       // GemmTile of RL update matrices
    int32_t rls_off = 0, rls_cnt = 0;       // task ids of small RL update matrices
    int32_t loop_off = 0, loop_cnt = 0;     // LoopItem (device-side RLB loops), one CTA per item
    int32_t loopw_off = 0, loopw_cnt = 0;   // LoopItem of supernodes narrower than 32 columns, one warp per item
    int32_t rlp_off = 0, rlp_cnt = 0;       // RLPair
    int64_t rlp_max = 0;                    // largest assembly work item (elements)
    int32_t rlo_off = 0, rlo_cnt = 0;       // RLSlab (deterministic plans: target-owned assembly)
    int32_t flow_off = 0, flow_cnt = 0;     // FlowUnit of this level's k_level launch (fused plans)
};

// kernel classes of the per-kernel profile
enum { kProfK0 = 0, kProfPotrf, kProfTrsm, kProfGemm, kProfTc, kProfSmall, kProfRlUpd, kProfRlAsm, kProfLoop, kProfClasses };

template <typename T>
struct DevArray {
    T *p = nullptr;
    int64_t n = 0;
};

}  // namespace sc

struct sc_numeric {
    sc_symbolic *sym = nullptr;
    int precision = SC_FP64;
    size_t elt = 8;
    cudaStream_t last_stream = nullptr;
    // device memory
    void *d_lnz = nullptr;
    void *d_pool = nullptr;
    int64_t *d_valmap = nullptr;
    double *d_values = nullptr;
    int64_t *d_diagpos = nullptr;
    double *d_adiag = nullptr;
    int32_t *d_info = nullptr;  // [0] = failing column (min), [1] = low-precision pivot count
    sc::ChunkDev *d_chunks = nullptr;
    int32_t *d_potrf = nullptr;
    sc::TrsmTile *d_trsm = nullptr;
    sc::GemmTile *d_gemm = nullptr;
    int32_t *d_small = nullptr;
    sc::ThinUnit *d_thin = nullptr;
    sc::Task *d_tasks = nullptr;
    sc::RLPair *d_rlpairs = nullptr;
    sc::RLSlab *d_rlslabs = nullptr;
    sc::SnDev *d_sn = nullptr;
    sc::BlkDev *d_blk = nullptr;
    int32_t *d_rbval = nullptr;
    sc::LoopItem *d_loops = nullptr;
    CUtensorMap *d_tmaps = nullptr;   // one per panel of width >= 16 (SC_TF32)
    int32_t *d_tmap_of_sn = nullptr;
    int32_t *d_err = nullptr;         // nonzero after a bounded device wait gave up
    void *d_inv = nullptr;            // FP32 inverses of the chunks' diagonal blocks (FP32 / TF32 factors)
    float *d_hi = nullptr;            // SC_TF32X3: tf32(x) of every final factor entry (same layout as Lnz)
    float *d_lo = nullptr;            // SC_TF32X3: tf32(x - hi)
    int32_t nmaps = 0;                // panels with tensor maps (lo maps follow hi maps for SC_TF32X3)
    int32_t *d_rlrelind = nullptr;
    // solve
    int32_t *d_glbind = nullptr;
    int32_t *d_perm = nullptr;
    int64_t *d_csr_ptr = nullptr;
    int32_t *d_csr_col = nullptr;
    double *d_csr_val = nullptr;
    int64_t *d_csr_map = nullptr;
    int32_t *d_counters = nullptr;  // [nchunks] solve tiles per chunk, then [nchunks] expected forward arrivals
    int32_t *d_dep_ptr = nullptr;   // per solve tile: range in d_dep
    int32_t *d_dep = nullptr;       // distinct chunks the tile's rows fall in
    int32_t *d_sync = nullptr;      // per sweep: arrivals, backward counters, done flags, work counters
    int32_t *d_serr = nullptr;      // nonzero after a bounded wait of a solve sweep gave up
    int32_t solve_tiles = 0;        // grab units of one sweep
    int32_t stall_chunk = -1;       // test hook: chunk whose expected arrivals are raised by one
    int32_t stall_factor_chunk = -1;  // test hook: chunk whose k_level count target is raised by one
    void *d_xw = nullptr;           // permuted right-hand side / forward work vector
    sc::TrsmTile *d_solve_tiles = nullptr;
    sc::SolveUnit *d_solve_units = nullptr;  // per level its first tiles, then the rest (backward: reversed)
    int64_t solve_cap = 0;          // rhs capacity of the work vectors
    double *d_x = nullptr, *d_r = nullptr, *d_b = nullptr, *d_xbest = nullptr;
    void *d_y = nullptr, *d_z = nullptr, *d_acc = nullptr;  // permuted work vectors (storage precision)
    double *d_red = nullptr;        // reductions for eta
    double *d_cgz = nullptr, *d_cgp = nullptr, *d_cgq = nullptr;  // preconditioned CG vectors (FP64)
    double *d_cgs = nullptr;        // CG scalars: r.z (two), p.Ap, per column
    int64_t cg_cap = 0;             // rhs capacity of the CG vectors
    double anorm = 0.0;
    bool solve_ready = false;
    // solve graphs for sg_nrhs right-hand sides: [0] x = solve(b) + residual,
    // [1] x += solve(r) + residual
    int64_t sg_nrhs = -1;
    cudaGraphExec_t sg[2] = {nullptr, nullptr};
    int32_t sg_launches[2] = {0, 0};
    int64_t device_bytes = 0;
    // plan
    std::vector<sc::LevelPlan> plans;
    int32_t ntasks = 0;
    int32_t kernel_launches = 0;
    double class_flops[sc::kProfClasses] = {};
    // graph of the factorization (captured on first use on a stream)
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;  // side branch of the captured factor graph (device loops)
    cudaStream_t cap_stream3 = nullptr;  // lookahead branch (products not needed by the next level)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_trsm = nullptr, ev_rest[2] = {nullptr, nullptr};
    bool lookahead = false;              // plan split into crit / rest products
    bool fused = false;                  // one k_level launch per level (SIMT precisions, RLB)
    sc::FlowUnit *d_flow = nullptr;      // units of every level's launch, then the tail launch's
    int32_t flow_tail_off = 0, flow_tail_cnt = 0;  // the products that follow the last level
    int32_t *d_flow_ctr = nullptr;       // per chunk: POTRF + TRSM units done (kFlowStride apart); then work counters
    int32_t *d_flow_need = nullptr;      // per chunk: 1 + its TRSM tiles
    int32_t *d_task_chunk = nullptr;     // per task: the chunk whose columns it reads last (its source)
    int32_t *d_sn_chunk = nullptr;       // per supernode: its last chunk
    bool use_graph = true;
    int num_sms = 152;
};

namespace sc {
int numeric_create(sc_symbolic *s, int precision, sc_numeric **out);
int numeric_factor(sc_numeric *h, const double *values, int on_device, cudaStream_t st, sc_factor_info *info);
int numeric_solve(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int on_device,
                  cudaStream_t st, sc_solve_info *info);
int numeric_export_L(const sc_numeric *h, double *out);
int plan_stats(const sc_symbolic *s, int precision, int64_t *out, int nout);
int numeric_profile(sc_numeric *h, const double *values, int on_device, cudaStream_t st, double *ms, double *flops,
                    int32_t *launches);
void numeric_free(sc_numeric *h);
}  // namespace sc
