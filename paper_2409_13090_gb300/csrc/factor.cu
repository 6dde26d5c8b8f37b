// Numeric factorization of libsc on the GPU: builds the per-level launch plan
// from the host schedule, owns the device memory of a numeric handle, and
// runs the level sequence (Alg. 5 RLB or Alg. 4 RL, made level-parallel),
// replayed as one CUDA graph.
#include <algorithm>
#include <cstring>

#include "kernels.cuh"
#include "numeric.h"
#include "tc_gemm.cuh"

namespace sc {

#define SC_CUDA(x)                                  \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return SC_ERR_CUDA;  \
    } while (0)

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

// diagonal of the input matrix in the final ordering: adiag[k] = A(perm[k], perm[k])
__global__ void k_diag(double *__restrict__ adiag, const int64_t *__restrict__ diag_pos,
                       const double *__restrict__ values, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) adiag[i] = values[diag_pos[i]];
}


template <typename U>
int upload(U *&dst, const std::vector<U> &src, int64_t &bytes) {
    size_t b = std::max<size_t>(1, src.size()) * sizeof(U);
    if (cudaMalloc((void **)&dst, b) != cudaSuccess) return SC_ERR_OOM;
    bytes += (int64_t)b;
    if (!src.empty() && cudaMemcpy(dst, src.data(), src.size() * sizeof(U), cudaMemcpyHostToDevice) != cudaSuccess)
        return SC_ERR_CUDA;
    return SC_OK;
}

bool is_small(const Task &t) { return (int64_t)t.m * t.n <= 64; }

// algorithmic flops of a product task: 2 k per entry written
double task_flops(const Task &t) {
    double e = (t.flags & kTaskLower) ? (double)t.n * (t.n + 1) / 2 + (double)(t.m - t.n) * t.n : (double)t.m * t.n;
    return 2.0 * e * t.k;
}

void tiles_of(const Task &t, int32_t id, std::vector<GemmTile> &out, bool no_split) {
    int tm = (t.m + kBM - 1) / kBM, tn = (t.n + kBN - 1) / kBN;
    // a task of few tiles with a long inner dimension is split along it, so its
    // tiles do not serialise a level; a critical task (the next level waits for
    // it) is split into slices of kSplitKCrit so its latency is short (an RL
    // update matrix is stored, not added: never split; nor is anything in a
    // deterministic plan, where the slices' atomic adds would land in any order)
    int slices = 0;
    if (!(t.flags & kTaskStoreU) && !no_split) {
        if ((t.flags & kTaskCrit) && t.k >= 2 * kSplitKCrit) slices = (t.k + kSplitKCrit - 1) / kSplitKCrit;
        else if (tm * tn <= 8 && t.k > 2 * kSplitK) slices = (t.k + kSplitK - 1) / kSplitK;
    }
    for (int i = 0; i < tm; i++)
        for (int j = 0; j < tn; j++) {
            if ((t.flags & kTaskLower) && (i * kBM + kBM - 1) < j * kBN) continue;  // above the diagonal
            if (!slices) out.push_back(GemmTile{id, i, j, -1});
            for (int q = 0; q < slices; q++) out.push_back(GemmTile{id, i, j, q});
        }
}

// FP32 inverses of the factored diagonal blocks of all chunks, for the solve
// sweeps of FP32 / TF32 factors (one launch after the last level, off the
// factorization's critical path).
__global__ void __launch_bounds__(256) k_inverse(const float *__restrict__ lnz, const ChunkDev *__restrict__ chunks,
                                                 const int32_t *__restrict__ list, float *__restrict__ inv) {
    extern __shared__ double smem_potrf[];
    const ChunkDev ch = chunks[list[blockIdx.x]];
    auto a = reinterpret_cast<float (*)[kMaxChunk + 1]>(smem_potrf);
    auto iv = a + kMaxChunk;
    load_block(a, lnz + ch.off + (int64_t)ch.c0 * ch.ld + ch.c0, ch.ld, ch.w);
    __syncthreads();
    tri_inverse<float>(a, ch.w, iv, inv + ch.inv);
}


// ---- one persistent launch per level (SIMT precisions, RLB)
// Bounded wait until *flag >= target (acquire at GPU scope); gives up, setting
// *err, after spin_limit polls or once another CTA has given up.
__device__ bool flow_wait(const int32_t *flag, int32_t target, int32_t *err, long long spin_limit, int code) {
    for (long long i = 0; i < spin_limit; i++) {
        int32_t v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v >= target) return true;
        if (*(volatile int32_t *)err) return false;
        if (i > 64) __nanosleep(64);
    }
    atomicCAS(err, 0, code);
    return false;
}

template <typename T>
struct LevelArgs {
    T *lnz, *pool;
    const ChunkDev *chunks;
    const TrsmTile *trsm;
    const GemmTile *gemm;
    const Task *tasks;
    const ThinUnit *thin;
    const int32_t *small;
    const LoopItem *loops;
    const SnDev *sn;
    const BlkDev *blk;
    const int32_t *rbval;
    const double *adiag;
    int32_t *info, *low_pivots;
    double tau;
    const FlowUnit *units;
    int32_t nunits;
    int32_t *ctr;             // per chunk (kFlowStride apart): POTRF and TRSM units done
    const int32_t *need;      // per chunk: 1 + its TRSM tiles
    const int32_t *task_chunk;
    const int32_t *sn_chunk;
    int32_t *work;            // this launch's unit counter
    int32_t *err;
    long long spin_limit;
};

// All work of one level in one launch: CTAs take units in list order (POTRF of
// the level's chunks, their TRSM tiles, the previous level's lookahead
// products, this level's products, small tasks and device loops). A TRSM tile
// waits for its chunk's POTRF; a product, small task or loop item waits until
// the chunk it reads is factored (POTRF and every TRSM tile). Every wait is
// for a unit earlier in the list, taken by a running CTA, so the launch needs
// no co-residency; every wait is bounded (then *err is set and the CTAs stop).
// Product writes are atomic: units of one launch may update the same target.
template <typename T>
__global__ void __launch_bounds__(256, 2) k_level(LevelArgs<T> a) {
    __shared__ int s_u, s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_u = *(volatile int32_t *)a.err ? a.nunits : atomicAdd(a.work, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= a.nunits) break;
        const FlowUnit fu = a.units[u];
        // dependencies, checked by thread 0
        if (threadIdx.x == 0) {
            bool ok = true;
            auto src = [&](int32_t c) {
                if (ok) ok = flow_wait(a.ctr + (int64_t)c * kFlowStride, a.need[c], a.err, a.spin_limit, 9);
            };
            switch (fu.kind) {
                case kFlowTrsm:
                    ok = flow_wait(a.ctr + (int64_t)a.trsm[fu.idx].chunk * kFlowStride, 1, a.err, a.spin_limit, 9);
                    break;
                case kFlowGemm: src(a.task_chunk[a.gemm[fu.idx].task]); break;
                case kFlowThin:
                    for (int q = 0; q < fu.cnt; q++) src(a.task_chunk[a.thin[fu.idx + q].task]);
                    break;
                case kFlowSmall:
                    for (int q = 0; q < fu.cnt; q++) src(a.task_chunk[a.small[fu.idx + q]]);
                    break;
                case kFlowLoop: src(a.sn_chunk[a.loops[fu.idx].sn]); break;
                case kFlowLoopW:
                    for (int q = 0; q < fu.cnt; q++) src(a.sn_chunk[a.loops[fu.idx + q].sn]);
                    break;
                default: break;
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        switch (fu.kind) {
            case kFlowPotrf:
                potrf_chunk<T>(a.lnz, a.chunks, fu.idx, a.adiag, a.info, a.low_pivots, a.tau, nullptr, nullptr);
                break;
            case kFlowTrsm: trsm_tile<T>(a.lnz, a.chunks, a.trsm[fu.idx], nullptr, nullptr); break;
            case kFlowGemm: gemm_tile<T, 64, 64, 16>(a.lnz, a.pool, a.tasks, a.gemm[fu.idx], true); break;
            case kFlowThin: {
                const int wq = threadIdx.x / 32 / kThinWarps;
                if (wq < fu.cnt) thin_warp<T>(a.lnz, a.tasks, a.thin[fu.idx + wq], (threadIdx.x / 32) % kThinWarps);
                break;
            }
            case kFlowSmall: small_tasks<T>(a.lnz, a.pool, a.tasks, a.small + fu.idx, fu.cnt, 0); break;
            case kFlowLoop: loop_item<T>(a.lnz, a.loops[fu.idx], a.sn, a.blk, a.rbval); break;
            case kFlowLoopW: loop_items_warp<T>(a.lnz, a.loops + fu.idx, fu.cnt, 0, a.sn, a.blk, a.rbval); break;
            default: break;
        }
        if (fu.kind == kFlowPotrf || fu.kind == kFlowTrsm) {
            // release: the barrier orders the CTA's stores before thread 0's fence
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const int32_t c = fu.kind == kFlowPotrf ? fu.idx : a.trsm[fu.idx].chunk;
                atomicAdd(a.ctr + (int64_t)c * kFlowStride, 1);
            }
        }
        __syncthreads();
    }
}

// Optional per-kernel-class timing of one factorization (CUDA events around
// every launch; only used outside graph capture).
struct Prof {
    cudaStream_t st = nullptr;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    int cur = -1;
    void begin(int cls) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        ev.push_back({cls, {a, b}});
    }
    void end() { cudaEventRecord(ev.back().second.second, st); }
};

template <typename T>
// st2 (optional, graph capture only): a second stream on which each level's
// device RLB loops run concurrently with the level's tiled products.
int run_levels(sc_numeric *h, cudaStream_t st, Prof *prof = nullptr, cudaStream_t st2 = nullptr,
               cudaStream_t st3 = nullptr) {
    const sc_symbolic *s = h->sym;
    auto B = [&](int cls) {
        if (prof) prof->begin(cls);
    };
    auto E = [&]() {
        if (prof) prof->end();
    };
    T *lnz = (T *)h->d_lnz;
    T *pool = (T *)h->d_pool;
    int launches = 0;
    B(kProfK0);
    SC_CUDA(cudaMemsetAsync(h->d_lnz, 0, (size_t)s->lnz_size * sizeof(T), st));
    SC_CUDA(cudaMemsetAsync(h->d_info, 0x7f, sizeof(int32_t), st));
    SC_CUDA(cudaMemsetAsync(h->d_info + 1, 0, sizeof(int32_t), st));
    SC_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
    int64_t nnz = (int64_t)s->valmap.size();
    k_diag<<<(unsigned)((s->n + 255) / 256), 256, 0, st>>>(h->d_adiag, h->d_diagpos, h->d_values, s->n);
    k_scatter_values<T><<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 152 * 16), 256, 0, st>>>(
        lnz, h->d_valmap, h->d_values, nnz);
    E();
    launches += 2;
    const double tau = s->opt.pivot_tau;
    if (h->fused && !prof) {
        // one persistent launch per level, then the tail of lookahead products
        const size_t nch = s->chunks.size(), nlev = h->plans.size();
        SC_CUDA(cudaMemsetAsync(h->d_flow_ctr, 0, (nch * kFlowStride + nlev + 1) * sizeof(int32_t), st));
        LevelArgs<T> a{lnz, pool, h->d_chunks, h->d_trsm, h->d_gemm, h->d_tasks, h->d_thin, h->d_small, h->d_loops,
                       h->d_sn, h->d_blk, h->d_rbval, h->d_adiag, h->d_info, h->d_info + 1, tau, nullptr, 0,
                       h->d_flow_ctr, h->d_flow_need, h->d_task_chunk, h->d_sn_chunk, nullptr, h->d_err,
                       (long long)s->opt.spin_limit};
        int32_t *work = h->d_flow_ctr + nch * kFlowStride;
        for (size_t lv = 0; lv <= nlev; lv++) {
            const int32_t off = lv < nlev ? h->plans[lv].flow_off : h->flow_tail_off;
            const int32_t cnt = lv < nlev ? h->plans[lv].flow_cnt : h->flow_tail_cnt;
            if (!cnt) continue;
            a.units = h->d_flow + off;
            a.nunits = cnt;
            a.work = work + lv;
            const int grid = std::max(1, std::min(cnt, 2 * h->num_sms));
            k_level<T><<<grid, 256, kPotrfSmem, st>>>(a);
            launches++;
        }
        if constexpr (sizeof(T) == 4) {
            const int32_t nchk = (int32_t)s->chunks.size();
            if (nchk) {
                k_inverse<<<nchk, 256, kPotrfSmem, st>>>((const float *)lnz, h->d_chunks, h->d_potrf, (float *)h->d_inv);
                launches++;
            }
        }
        SC_CUDA(cudaGetLastError());
        h->kernel_launches = launches;
        return SC_OK;
    }
    // tiled products of one dependency class on stream ps
    auto products = [&](const ProdLists &pl, cudaStream_t ps) -> int {
        if (pl.gemm_cnt) {
            B(kProfGemm);
            k_gemm_tiles<T, kBM, kBN, kBK><<<pl.gemm_cnt, 256, 0, ps>>>(lnz, pool, h->d_tasks,
                                                                        h->d_gemm + pl.gemm_off);
            E();
            launches++;
        }
        if constexpr (sizeof(T) == 4) {
            if (pl.tc_cnt) {
                B(kProfTc);
                launch_tc_gemm(128, h->precision == SC_TF32X3, (float *)lnz, h->d_tasks, h->d_gemm + pl.tc_off,
                               pl.tc_cnt, h->d_tmaps, h->nmaps, h->d_tmap_of_sn, h->d_err,
                               (long long)s->opt.spin_limit, h->num_sms, ps);
                E();
                launches++;
            }
            if (pl.tc256_cnt) {
                B(kProfTc);
                launch_tc_gemm(256, h->precision == SC_TF32X3, (float *)lnz, h->d_tasks, h->d_gemm + pl.tc256_off,
                               pl.tc256_cnt, h->d_tmaps, h->nmaps, h->d_tmap_of_sn, h->d_err,
                               (long long)s->opt.spin_limit, h->num_sms, ps, knobs_of(s->tune).tc_multicast);
                E();
                launches++;
            }
            if (pl.tc64_cnt) {
                B(kProfTc);
                launch_tc_gemm(64, h->precision == SC_TF32X3, (float *)lnz, h->d_tasks, h->d_gemm + pl.tc64_off,
                               pl.tc64_cnt, h->d_tmaps, h->nmaps, h->d_tmap_of_sn, h->d_err,
                               (long long)s->opt.spin_limit, h->num_sms, ps);
                E();
                launches++;
            }
        }
        if (pl.thin_cnt) {
            B(kProfGemm);
            k_thin_tasks<T><<<pl.thin_cnt, kThinWarps * 32, 0, ps>>>(lnz, h->d_tasks, h->d_thin + pl.thin_off);
            E();
            launches++;
        }
        return SC_OK;
    };
    const size_t nlev = h->plans.size();
    for (size_t lv = 0; lv < nlev; lv++) {
        const LevelPlan &p = h->plans[lv];
        if (p.potrf_cnt) {
            B(kProfPotrf);
            k_potrf<T><<<p.potrf_cnt, 256, kPotrfSmem, st>>>(lnz, h->d_chunks, h->d_potrf + p.potrf_off, h->d_adiag,
                                                              h->d_info, h->d_info + 1, tau, h->d_hi, h->d_lo);
            E();
            launches++;
        }
        if (p.trsm_cnt) {
            B(kProfTrsm);
            k_trsm<T><<<p.trsm_cnt, trsm_rows<T>() * 4, 0, st>>>(lnz, h->d_chunks, h->d_trsm + p.trsm_off, h->d_hi,
                                                           h->d_lo);
            E();
            launches++;
        }
        // Lookahead: level lv's products into chunks two or more levels up run on
        // st3, overlapping level lv+1's POTRF, TRSM and device loops; level lv+1's
        // own products wait for them, so no target is written by two streams at
        // once (rest(lv) and crit(lv) have disjoint targets, and so have rest(lv)
        // and the device loops, which never target a supernode being factored).
        if (st3) {
            SC_CUDA(cudaEventRecord(h->ev_trsm, st));
            SC_CUDA(cudaStreamWaitEvent(st3, h->ev_trsm, 0));
            int rc = products(p.rest, st3);
            if (rc) return rc;
            SC_CUDA(cudaEventRecord(h->ev_rest[lv % 2], st3));
        }
        bool join = false;
        if (p.loop_cnt || p.loopw_cnt) {
            B(kProfLoop);
            cudaStream_t ls = st;
            if (st2 && (p.crit.any() || p.small_cnt)) {  // fork: loops and tiled products are independent
                SC_CUDA(cudaEventRecord(h->ev_fork, st));
                SC_CUDA(cudaStreamWaitEvent(st2, h->ev_fork, 0));
                ls = st2;
                join = true;
            }
            if (p.loop_cnt) {
                k_rlb_loop<T><<<p.loop_cnt, 256, 0, ls>>>(lnz, h->d_loops + p.loop_off, h->d_sn, h->d_blk,
                                                          h->d_rbval);
                launches++;
            }
            if (p.loopw_cnt) {
                k_rlb_loop_warp<T><<<(p.loopw_cnt + 7) / 8, 256, 0, ls>>>(lnz, h->d_loops + p.loopw_off, p.loopw_cnt,
                                                                          h->d_sn, h->d_blk, h->d_rbval);
                launches++;
            }
            if (join) SC_CUDA(cudaEventRecord(h->ev_join, st2));
            E();
        }
        {
            if (st3 && lv >= 1) SC_CUDA(cudaStreamWaitEvent(st, h->ev_rest[(lv - 1) % 2], 0));
            int rc = products(p.crit, st);
            if (rc) return rc;
            if (!st3 && (rc = products(p.rest, st))) return rc;
        }
        if (p.small_cnt) {
            B(kProfSmall);
            k_small_tasks<T><<<(p.small_cnt + 7) / 8, 256, 0, st>>>(lnz, pool, h->d_tasks, h->d_small + p.small_off,
                                                                    p.small_cnt);
            E();
            launches++;
        }
        if (p.rlg_cnt) {
            B(kProfRlUpd);
            k_gemm_tiles<T, kBM, kBN, kBK><<<p.rlg_cnt, 256, 0, st>>>(lnz, pool, h->d_tasks, h->d_gemm + p.rlg_off);
            E();
            launches++;
        }
        if (p.rls_cnt) {
            B(kProfRlUpd);
            k_small_tasks<T><<<(p.rls_cnt + 7) / 8, 256, 0, st>>>(lnz, pool, h->d_tasks, h->d_small + p.rls_off,
                                                                  p.rls_cnt);
            E();
            launches++;
        }
        if (join) SC_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
        if (p.rlo_cnt) {
            B(kProfRlAsm);
            k_rl_assemble_ordered<T><<<p.rlo_cnt, 256, 0, st>>>(lnz, pool, h->d_rlpairs, h->d_rlslabs + p.rlo_off,
                                                                h->d_rlrelind);
            E();
            launches++;
        }
        for (int32_t q0 = 0; q0 < p.rlp_cnt && !p.rlo_cnt; q0 += 65535) {  // grid.y holds at most 65535 pairs
            unsigned gx = (unsigned)std::min<int64_t>((p.rlp_max + 255) / 256, 64);
            unsigned gy = (unsigned)std::min<int32_t>(65535, p.rlp_cnt - q0);
            B(kProfRlAsm);
            k_rl_assemble<T><<<dim3(gx, gy), 256, 0, st>>>(lnz, pool, h->d_rlpairs + p.rlp_off + q0, h->d_rlrelind);
            E();
            launches++;
        }
    }
    if (st3 && nlev) SC_CUDA(cudaStreamWaitEvent(st, h->ev_rest[(nlev - 1) % 2], 0));  // join the lookahead branch
    if constexpr (sizeof(T) == 4) {
        // diagonal-block inverses for the solve, all chunks in one launch
        const int32_t nch = (int32_t)s->chunks.size();
        if (nch) {
            B(kProfPotrf);
            k_inverse<<<nch, 256, kPotrfSmem, st>>>((const float *)lnz, h->d_chunks, h->d_potrf, (float *)h->d_inv);
            E();
            launches++;
        }
    }
    SC_CUDA(cudaGetLastError());
    h->kernel_launches = launches;
    return SC_OK;
}

int set_smem_attrs() {
    static bool done = false;
    if (done) return SC_OK;
    SC_CUDA(cudaFuncSetAttribute(k_potrf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPotrfSmem));
    SC_CUDA(cudaFuncSetAttribute(k_potrf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPotrfSmem));
    SC_CUDA(cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, kPotrfSmem));
    SC_CUDA(cudaFuncSetAttribute(k_level<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPotrfSmem));
    SC_CUDA(cudaFuncSetAttribute(k_level<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPotrfSmem));
    if (!tc_gemm_init()) return SC_ERR_CUDA;
    done = true;
    return SC_OK;
}

// Host-only launch plan of one factorization for a precision: flat work lists
// with per-level offsets (no device memory touched).
struct Plan {
    std::vector<ChunkDev> cd;
    std::vector<int32_t> potrf, small;
    std::vector<ThinUnit> thin;
    std::vector<TrsmTile> trsm;
    std::vector<GemmTile> gemm;
    std::vector<Task> tasks;
    std::vector<RLPair> rlpairs;
    std::vector<RLSlab> rlslabs;
    std::vector<LoopItem> loops;
    std::vector<LevelPlan> levels;
    int64_t inv_size = 0;  // elements of the diagonal-block inverses
    double class_flops[kProfClasses] = {};
    // fused plans: the units of every level's k_level launch, then the tail launch's
    std::vector<FlowUnit> flow;
    int32_t flow_tail_off = 0, flow_tail_cnt = 0;
};

// Units of the per-level launches (fused plans): per level its POTRFs, TRSM
// tiles, the previous level's lookahead products (lookahead), its own products
// (with the rest as well when there is no lookahead), small tasks in eights,
// loop items, narrow loop items in eights; the last level's lookahead products
// form a tail launch.
void build_flow(Plan &P, bool lookahead) {
    P.flow.clear();
    auto products = [&](const ProdLists &pl) {
        for (int32_t i = 0; i < pl.gemm_cnt; i++) P.flow.push_back(FlowUnit{kFlowGemm, pl.gemm_off + i, 1, 0});
        for (int32_t i = 0; i < pl.thin_cnt; i += 2)
            P.flow.push_back(FlowUnit{kFlowThin, pl.thin_off + i, std::min<int32_t>(2, pl.thin_cnt - i), 0});
    };
    const size_t nlev = P.levels.size();
    for (size_t lv = 0; lv < nlev; lv++) {
        LevelPlan &p = P.levels[lv];
        p.flow_off = (int32_t)P.flow.size();
        for (int32_t i = 0; i < p.potrf_cnt; i++) P.flow.push_back(FlowUnit{kFlowPotrf, P.potrf[p.potrf_off + i], 1, 0});
        for (int32_t i = 0; i < p.trsm_cnt; i++) P.flow.push_back(FlowUnit{kFlowTrsm, p.trsm_off + i, 1, 0});
        if (lookahead && lv > 0) products(P.levels[lv - 1].rest);
        products(p.crit);
        if (!lookahead) products(p.rest);
        for (int32_t i = 0; i < p.small_cnt; i += 8)
            P.flow.push_back(FlowUnit{kFlowSmall, p.small_off + i, std::min<int32_t>(8, p.small_cnt - i), 0});
        for (int32_t i = 0; i < p.loop_cnt; i++) P.flow.push_back(FlowUnit{kFlowLoop, p.loop_off + i, 1, 0});
        for (int32_t i = 0; i < p.loopw_cnt; i += 8)
            P.flow.push_back(FlowUnit{kFlowLoopW, p.loopw_off + i, std::min<int32_t>(8, p.loopw_cnt - i), 0});
        p.flow_cnt = (int32_t)P.flow.size() - p.flow_off;
    }
    P.flow_tail_off = (int32_t)P.flow.size();
    if (lookahead && nlev) products(P.levels[nlev - 1].rest);
    P.flow_tail_cnt = (int32_t)P.flow.size() - P.flow_tail_off;
}

// lookahead: split each level's tiled products into those that target chunks
// of the next level (crit) and the rest (targets two or more levels up).
void build_plan(const sc_symbolic *s, int precision, Plan &P, bool lookahead) {
    const Knobs kn = knobs_of(s->tune);
    const bool det = s->opt.deterministic != 0;
    P.cd.resize(s->chunks.size());
    int64_t inv = 0;
    for (size_t c = 0; c < s->chunks.size(); c++) {
        const Chunk &ch = s->chunks[c];
        int32_t J = ch.sn;
        P.cd[c] = ChunkDev{s->lnz_off[J], s->gl_ptr[J], inv, s->lnz_ld[J], (int32_t)(s->gl_ptr[J + 1] - s->gl_ptr[J]),
                           ch.c0, ch.w, s->sup_ptr[J] + ch.c0, 0};
        inv += (int64_t)ch.w * ch.w;
    }
    P.inv_size = inv;
    const bool tc = precision == SC_TF32 || precision == SC_TF32X3;
    std::vector<int32_t> tmap_of_sn(s->nsuper, -1);
    {
        int32_t nm = 0;
        for (int64_t J = 0; J < s->nsuper; J++)
            if (s->sup_ptr[J + 1] - s->sup_ptr[J] >= 16) tmap_of_sn[J] = nm++;
    }
    P.levels.resize(s->levels.size());
    for (size_t lv = 0; lv < s->levels.size(); lv++) {
        const Level &L = s->levels[lv];
        LevelPlan &p = P.levels[lv];
        p.potrf_off = (int32_t)P.potrf.size();
        for (int32_t c : L.chunks) {
            P.potrf.push_back(c);
            double w = P.cd[c].w;
            P.class_flops[kProfPotrf] += w * w * w / 3.0;
            P.class_flops[kProfTrsm] += (double)(P.cd[c].m - P.cd[c].c0 - P.cd[c].w) * w * w;
        }
        p.potrf_cnt = (int32_t)P.potrf.size() - p.potrf_off;
        p.trsm_off = (int32_t)P.trsm.size();
        for (int32_t c : L.chunks) {
            const ChunkDev &ch = P.cd[c];
            const int32_t rows = precision == SC_FP64 ? trsm_rows<double>() : trsm_rows<float>();
            for (int32_t r0 = ch.c0 + ch.w; r0 < ch.m; r0 += rows) P.trsm.push_back(TrsmTile{c, r0});
        }
        p.trsm_cnt = (int32_t)P.trsm.size() - p.trsm_off;
        // product tasks: tensor-core tiles (TF32), SIMT tiles, warp tasks
        std::vector<int32_t> ids_small;
        std::vector<ThinUnit> units_thin[2];
        std::vector<GemmTile> g_simt[2], g_tc[2], g_tc64[2], g_tc256[2];
        const bool split = lookahead;
        for (Task t : L.tasks) {
            int32_t id = (int32_t)P.tasks.size();
            const int cls = split && !(t.flags & kTaskCrit) ? 1 : 0;  // 0 crit, 1 rest
            P.tasks.push_back(t);
            int bn = tc ? tc_width(t, tmap_of_sn, s->sup_ptr[t.src + 1] - s->sup_ptr[t.src], kn.tc_min_k,
                                    kn.tc_wide_n, s->test_tc_ignore_tail)
                        : 0;
            if (bn == 128 && t.n >= kn.tc_wide256) bn = 256;
            if (is_small(t)) {
                ids_small.push_back(id);
                P.class_flops[kProfSmall] += task_flops(t);
            } else if (bn) {
                if (bn == 256 && kn.tc_multicast) tc_tile_pairs_of(t, id, g_tc256[cls]);
                else tc_tiles_of(t, id, bn, bn == 256 ? g_tc256[cls] : bn == 128 ? g_tc[cls] : g_tc64[cls]);
                P.class_flops[kProfTc] += task_flops(t);
            } else if (std::min(t.m, t.n) <= std::min(kn.thin_dim, kThinDim) && !(t.flags & kTaskStoreU)) {
                // a 64 x 64 tile would be mostly padding: warp blocks, kThinWarps per CTA
                const int ni = block_rows(t.m, t.n, precision == SC_FP64 ? 2 : 1, (t.flags & kTaskLower) != 0);
                const int nblk = ((t.m + ni - 1) / ni) * ((t.n + 32 / ni - 1) / (32 / ni));
                for (int b0 = 0; b0 < nblk; b0 += kThinWarps) units_thin[cls].push_back(ThinUnit{id, b0});
                P.class_flops[kProfGemm] += task_flops(t);
            } else {
                tiles_of(t, id, g_simt[cls], det);
                P.class_flops[kProfGemm] += task_flops(t);
            }
        }
        for (int cls = 0; cls < 2; cls++) {
            ProdLists &pl = cls == 0 ? p.crit : p.rest;
            pl.gemm_off = (int32_t)P.gemm.size();
            P.gemm.insert(P.gemm.end(), g_simt[cls].begin(), g_simt[cls].end());
            pl.gemm_cnt = (int32_t)g_simt[cls].size();
            pl.tc_off = (int32_t)P.gemm.size();
            P.gemm.insert(P.gemm.end(), g_tc[cls].begin(), g_tc[cls].end());
            pl.tc_cnt = (int32_t)g_tc[cls].size();
            pl.tc64_off = (int32_t)P.gemm.size();
            P.gemm.insert(P.gemm.end(), g_tc64[cls].begin(), g_tc64[cls].end());
            pl.tc64_cnt = (int32_t)g_tc64[cls].size();
            pl.tc256_off = (int32_t)P.gemm.size();
            P.gemm.insert(P.gemm.end(), g_tc256[cls].begin(), g_tc256[cls].end());
            pl.tc256_cnt = (int32_t)g_tc256[cls].size();
            pl.thin_off = (int32_t)P.thin.size();
            P.thin.insert(P.thin.end(), units_thin[cls].begin(), units_thin[cls].end());
            pl.thin_cnt = (int32_t)units_thin[cls].size();
        }
        p.small_off = (int32_t)P.small.size();
        P.small.insert(P.small.end(), ids_small.begin(), ids_small.end());
        p.small_cnt = (int32_t)ids_small.size();
        // device-side RLB loops
        // (items of supernodes narrower than 32 columns: one warp each)
        p.loop_off = (int32_t)P.loops.size();
        for (const LoopItem &it : L.loops)
            if (s->sup_ptr[it.sn + 1] - s->sup_ptr[it.sn] >= 32) P.loops.push_back(it);
        p.loop_cnt = (int32_t)P.loops.size() - p.loop_off;
        p.loopw_off = (int32_t)P.loops.size();
        for (const LoopItem &it : L.loops)
            if (s->sup_ptr[it.sn + 1] - s->sup_ptr[it.sn] < 32) P.loops.push_back(it);
        p.loopw_cnt = (int32_t)P.loops.size() - p.loopw_off;
        P.class_flops[kProfLoop] += L.loop_flops;
        // RL update matrices and assembly
        std::vector<int32_t> rl_small;
        std::vector<GemmTile> rl_g;
        for (const Task &t : L.rl_tasks) {
            int32_t id = (int32_t)P.tasks.size();
            P.tasks.push_back(t);
            if (is_small(t)) rl_small.push_back(id);
            else tiles_of(t, id, rl_g, det);
            P.class_flops[kProfRlUpd] += task_flops(t);
        }
        p.rlg_off = (int32_t)P.gemm.size();
        P.gemm.insert(P.gemm.end(), rl_g.begin(), rl_g.end());
        p.rlg_cnt = (int32_t)rl_g.size();
        p.rls_off = (int32_t)P.small.size();
        P.small.insert(P.small.end(), rl_small.begin(), rl_small.end());
        p.rls_cnt = (int32_t)rl_small.size();
        p.rlp_off = (int32_t)P.rlpairs.size();
        for (const RLPair &pr : L.rl_pairs) {
            P.rlpairs.push_back(pr);
            p.rlp_max = std::max<int64_t>(p.rlp_max, (int64_t)(pr.c_end - pr.c_begin) * (pr.s - pr.c_begin));
            P.class_flops[kProfRlAsm] += (double)(pr.c_end - pr.c_begin) * (pr.s - pr.c_begin);
        }
        p.rlp_cnt = (int32_t)L.rl_pairs.size();
        if (det) {
            // target-owned assembly: the level's pairs grouped by target P, each
            // group in the order of its source supernodes (the order the level
            // lists them in), P's touched rows cut into slabs of kRLSlabRows
            auto first = P.rlpairs.begin() + p.rlp_off;
            std::stable_sort(first, P.rlpairs.end(),
                             [](const RLPair &a, const RLPair &b) { return a.p_off < b.p_off; });
            p.rlo_off = (int32_t)P.rlslabs.size();
            for (int32_t g0 = p.rlp_off, g1; g0 < (int32_t)P.rlpairs.size(); g0 = g1) {
                int32_t lo = INT32_MAX, hi = -1;
                for (g1 = g0; g1 < (int32_t)P.rlpairs.size() && P.rlpairs[g1].p_off == P.rlpairs[g0].p_off; g1++) {
                    const RLPair &pr = P.rlpairs[g1];
                    const int32_t *ri = s->rl_relind.data() + pr.ri_off;
                    // target rows mP - 1 - relind[r] of the pair's rows, ascending in r
                    lo = std::min(lo, pr.mP - 1 - ri[0]);
                    hi = std::max(hi, pr.mP - 1 - ri[pr.s - pr.c_begin - 1]);
                }
                for (int32_t r = lo; r <= hi; r += kRLSlabRows)
                    P.rlslabs.push_back(RLSlab{g0, g1 - g0, r, std::min(hi + 1, r + kRLSlabRows)});
            }
            p.rlo_cnt = (int32_t)P.rlslabs.size() - p.rlo_off;
            if (s->test_det_short_slab && p.rlo_cnt && !P.rlslabs.empty()) {
                RLSlab &last = P.rlslabs.back();  // its last row is a touched row (the group's hi)
                if (last.row1 - last.row0 > 1 && P.rlslabs.size() == (size_t)p.rlo_cnt) last.row1--;
            }
        }
    }
}

}  // namespace

int det_plan_check(const sc_symbolic *s, int64_t *bad_level) {
    for (int precision : {SC_FP64, SC_TF32}) {
        Plan P;
        build_plan(s, precision, P, false);
        for (size_t lv = 0; lv < P.levels.size(); lv++) {
            const LevelPlan &p = P.levels[lv];
            *bad_level = (int64_t)lv;
            auto split_in = [&](int32_t off, int32_t cnt) {
                for (int32_t i = off; i < off + cnt; i++)
                    if (P.gemm[i].ks >= 0) return true;
                return false;
            };
            for (const ProdLists *pl : {&p.crit, &p.rest})
                if (split_in(pl->gemm_off, pl->gemm_cnt) || split_in(pl->tc_off, pl->tc_cnt) ||
                    split_in(pl->tc64_off, pl->tc64_cnt) || split_in(pl->tc256_off, pl->tc256_cnt))
                    return 13;
            if (split_in(p.rlg_off, p.rlg_cnt)) return 13;
            if (!p.rlp_cnt) continue;
            // slabs: inside the level's pairs, one target each, sources ascending (pool offsets
            // follow the level's source order), groups disjoint and ascending, a group's row
            // ranges non-empty, ascending and disjoint
            const int32_t pe = p.rlp_off + p.rlp_cnt;
            for (int32_t q = p.rlo_off; q < p.rlo_off + p.rlo_cnt; q++) {
                const RLSlab &sl = P.rlslabs[q];
                if (sl.npairs < 1 || sl.pair0 < p.rlp_off || sl.pair0 + sl.npairs > pe || sl.row0 >= sl.row1) return 13;
                for (int32_t i = sl.pair0 + 1; i < sl.pair0 + sl.npairs; i++)
                    if (P.rlpairs[i].p_off != P.rlpairs[sl.pair0].p_off || P.rlpairs[i].u_off <= P.rlpairs[i - 1].u_off)
                        return 13;
                if (q > p.rlo_off) {
                    const RLSlab &pv = P.rlslabs[q - 1];
                    if (pv.pair0 == sl.pair0 ? (pv.npairs != sl.npairs || pv.row1 > sl.row0)
                                             : pv.pair0 + pv.npairs > sl.pair0)
                        return 13;
                }
            }
            // every target row of every pair lies in a slab of the pair's group
            int32_t q = p.rlo_off;
            for (int32_t i = p.rlp_off; i < pe; i++) {
                while (q < p.rlo_off + p.rlo_cnt && P.rlslabs[q].pair0 + P.rlslabs[q].npairs <= i) q++;
                if (q == p.rlo_off + p.rlo_cnt || P.rlslabs[q].pair0 > i) return 13;
                int32_t qe = q;
                while (qe < p.rlo_off + p.rlo_cnt && P.rlslabs[qe].pair0 == P.rlslabs[q].pair0) qe++;
                const RLPair &pr = P.rlpairs[i];
                const int32_t *ri = s->rl_relind.data() + pr.ri_off;
                for (int32_t r = 0, k = q; r < pr.s - pr.c_begin; r++) {
                    const int32_t row = pr.mP - 1 - ri[r];
                    while (k < qe && P.rlslabs[k].row1 <= row) k++;
                    if (k == qe || P.rlslabs[k].row0 > row) return 13;
                }
            }
        }
    }
    *bad_level = -1;
    return 0;
}

int plan_stats(const sc_symbolic *s, int precision, int64_t *out, int nout) {
    Plan P;
    build_plan(s, precision, P, false);
    int64_t small_tasks = 0, tile_tasks = 0;
    for (const LevelPlan &l : P.levels) small_tasks += l.small_cnt + l.rls_cnt;
    tile_tasks = (int64_t)P.tasks.size() - small_tasks;
    int64_t tc_tiles = 0, simt_tiles = 0, split_tiles = 0, tc256_tiles = 0;
    for (const LevelPlan &l : P.levels) {
        tc256_tiles += l.crit.tc256_cnt + l.rest.tc256_cnt;
        tc_tiles += l.crit.tc_cnt + l.crit.tc64_cnt + l.crit.tc256_cnt + l.rest.tc_cnt + l.rest.tc64_cnt +
                    l.rest.tc256_cnt;
        simt_tiles += l.crit.gemm_cnt + l.rest.gemm_cnt + l.rlg_cnt;
    }
    for (const GemmTile &g : P.gemm) split_tiles += g.ks >= 0;
    int64_t v[] = {(int64_t)P.levels.size(), (int64_t)P.cd.size(), (int64_t)P.tasks.size(), small_tasks, tile_tasks,
                   simt_tiles, tc_tiles, (int64_t)P.trsm.size(), (int64_t)P.rlpairs.size(), (int64_t)P.loops.size(),
                   (int64_t)P.thin.size(), split_tiles, (int64_t)P.rlslabs.size(), tc256_tiles};
    for (int i = 0; i < nout && i < (int)(sizeof(v) / sizeof(v[0])); i++) out[i] = v[i];
    return SC_OK;
}

int numeric_create(sc_symbolic *s, int precision, sc_numeric **out) {
    if (precision < SC_FP64 || precision > SC_TF32X3) return -3;
    if (s->poisoned) return SC_ERR_INTERNAL;
    int rc = set_smem_attrs();
    if (rc) return rc;
    auto h = new sc_numeric();
    h->sym = s;
    s->refs++;  // released by numeric_free, also on the error paths below
    h->precision = precision;
    h->elt = precision == SC_FP64 ? 8 : 4;
    h->use_graph = s->opt.use_graph != 0;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (h->num_sms < 1) h->num_sms = 1;
    }
    int64_t &bytes = h->device_bytes;
    auto fail = [&](int code) {
        numeric_free(h);
        return code;
    };
    if (cudaMalloc(&h->d_lnz, (size_t)s->lnz_size * h->elt) != cudaSuccess) return fail(SC_ERR_OOM);
    bytes += s->lnz_size * (int64_t)h->elt;
    if (cudaMalloc(&h->d_pool, (size_t)std::max<int64_t>(1, s->rl_pool_max) * h->elt) != cudaSuccess)
        return fail(SC_ERR_OOM);
    bytes += std::max<int64_t>(1, s->rl_pool_max) * (int64_t)h->elt;
    if ((rc = upload(h->d_valmap, s->valmap, bytes))) return fail(rc);
    if (cudaMalloc((void **)&h->d_values, std::max<size_t>(1, s->valmap.size()) * sizeof(double)) != cudaSuccess)
        return fail(SC_ERR_OOM);
    bytes += (int64_t)s->valmap.size() * 8;
    {
        std::vector<int64_t> dp(s->n);
        for (int64_t k = 0; k < s->n; k++) dp[k] = s->colptr[s->perm[k]];  // diagonal is first in its column
        if ((rc = upload(h->d_diagpos, dp, bytes))) return fail(rc);
    }
    if (cudaMalloc((void **)&h->d_adiag, (size_t)s->n * sizeof(double)) != cudaSuccess) return fail(SC_ERR_OOM);
    if (cudaMalloc((void **)&h->d_info, 2 * sizeof(int32_t)) != cudaSuccess) return fail(SC_ERR_OOM);
    if (cudaMalloc((void **)&h->d_err, sizeof(int32_t)) != cudaSuccess) return fail(SC_ERR_OOM);
    if (precision == SC_TF32X3) {
        // split copies of the factor: zero once, so padding columns stay zero
        for (float **p : {&h->d_hi, &h->d_lo}) {
            if (cudaMalloc((void **)p, (size_t)s->lnz_size * sizeof(float)) != cudaSuccess) return fail(SC_ERR_OOM);
            if (cudaMemset(*p, 0, (size_t)s->lnz_size * sizeof(float)) != cudaSuccess) return fail(SC_ERR_CUDA);
            bytes += s->lnz_size * 4;
        }
    }
    if (precision == SC_TF32 || precision == SC_TF32X3) {
        // TF32: maps over the factor; TF32x3: maps over hi, then maps over lo
        std::vector<CUtensorMap> maps, maps_lo;
        std::vector<int32_t> tmap_of_sn;
        if ((rc = tc_encode_maps(s, precision == SC_TF32 ? (float *)h->d_lnz : h->d_hi, maps, tmap_of_sn)))
            return fail(rc);
        h->nmaps = (int32_t)(maps.size() / 2);
        if (precision == SC_TF32X3) {
            if ((rc = tc_encode_maps(s, h->d_lo, maps_lo, tmap_of_sn))) return fail(rc);
            maps.insert(maps.end(), maps_lo.begin(), maps_lo.end());
        }
        if ((rc = upload(h->d_tmaps, maps, bytes))) return fail(rc);
        if ((rc = upload(h->d_tmap_of_sn, tmap_of_sn, bytes))) return fail(rc);
    }
    Plan P;
    // one persistent launch per level: SIMT precisions, RLB schedule
    const Knobs kn = knobs_of(s->tune);
    h->fused = kn.fused && s->opt.variant == SC_RLB && (precision == SC_FP64 || precision == SC_FP32);
    // lookahead needs concurrent work: the captured graph's branches, or the fused launches
    h->lookahead = (h->use_graph || h->fused) && s->opt.variant == SC_RLB && kn.lookahead;
    build_plan(s, precision, P, h->lookahead);
    if (h->fused) {
        build_flow(P, h->lookahead);
        h->flow_tail_off = P.flow_tail_off;
        h->flow_tail_cnt = P.flow_tail_cnt;
        const size_t nch = s->chunks.size();
        std::vector<int32_t> need(nch, 1), task_chunk(P.tasks.size()), sn_chunk(s->nsuper);
        for (const TrsmTile &t : P.trsm) need[t.chunk]++;
        for (size_t i = 0; i < P.tasks.size(); i++) {
            const Task &t = P.tasks[i];
            task_chunk[i] = s->chunk_of_col[s->sup_ptr[t.src] + t.kx0 + t.k - 1];
        }
        for (int64_t J = 0; J < s->nsuper; J++) sn_chunk[J] = s->chunk_of_col[s->sup_ptr[J + 1] - 1];
        if ((rc = upload(h->d_flow, P.flow, bytes))) return fail(rc);
        if ((rc = upload(h->d_flow_need, need, bytes))) return fail(rc);
        if ((rc = upload(h->d_task_chunk, task_chunk, bytes))) return fail(rc);
        if ((rc = upload(h->d_sn_chunk, sn_chunk, bytes))) return fail(rc);
        const size_t words = nch * kFlowStride + P.levels.size() + 1;
        if (cudaMalloc((void **)&h->d_flow_ctr, words * sizeof(int32_t)) != cudaSuccess) return fail(SC_ERR_OOM);
        bytes += (int64_t)(words * sizeof(int32_t));
    }
    if (precision != SC_FP64) {
        if (cudaMalloc(&h->d_inv, (size_t)std::max<int64_t>(1, P.inv_size) * sizeof(float)) != cudaSuccess)
            return fail(SC_ERR_OOM);
        bytes += P.inv_size * 4;
    }
    std::copy(P.class_flops, P.class_flops + kProfClasses, h->class_flops);
    h->plans = P.levels;
    h->ntasks = (int32_t)P.tasks.size();
    if ((rc = upload(h->d_chunks, P.cd, bytes))) return fail(rc);
    if ((rc = upload(h->d_potrf, P.potrf, bytes))) return fail(rc);
    if ((rc = upload(h->d_trsm, P.trsm, bytes))) return fail(rc);
    if ((rc = upload(h->d_gemm, P.gemm, bytes))) return fail(rc);
    if ((rc = upload(h->d_small, P.small, bytes))) return fail(rc);
    if ((rc = upload(h->d_thin, P.thin, bytes))) return fail(rc);
    if ((rc = upload(h->d_tasks, P.tasks, bytes))) return fail(rc);
    if ((rc = upload(h->d_rlpairs, P.rlpairs, bytes))) return fail(rc);
    if ((rc = upload(h->d_rlslabs, P.rlslabs, bytes))) return fail(rc);
    if ((rc = upload(h->d_rlrelind, s->rl_relind, bytes))) return fail(rc);
    if ((rc = upload(h->d_loops, P.loops, bytes))) return fail(rc);
    {
        std::vector<SnDev> snd(s->nsuper);
        for (int64_t J = 0; J < s->nsuper; J++)
            snd[J] = SnDev{s->lnz_off[J], s->lnz_ld[J], (int32_t)(s->gl_ptr[J + 1] - s->gl_ptr[J]), s->sup_ptr[J],
                           s->sup_ptr[J + 1] - s->sup_ptr[J], (int32_t)s->blk_ptr[J + 1], 0};
        std::vector<BlkDev> bd(s->blk_first.size());
        for (int64_t J = 0; J < s->nsuper; J++) {
            int64_t b0 = s->blk_ptr[J], b1 = s->blk_ptr[J + 1];
            int32_t q = s->sup_ptr[J + 1] - s->sup_ptr[J];
            for (int64_t b = b0; b < b1; b++) {
                bd[b] = BlkDev{q, s->blk_size[b], s->blk_first[b], s->blk_owner[b], 0, 0, 0};
                q += s->blk_size[b];
            }
            for (int64_t pq = s->rb_pair_ptr[J]; pq < s->rb_pair_ptr[J + 1]; pq++) {
                int64_t cnt = s->rb_val_ptr[pq + 1] - s->rb_val_ptr[pq];
                int64_t bs = b1 - cnt;
                for (int64_t b = bs; b < b1 && s->blk_owner[b] == s->rb_pair_P[pq]; b++) {
                    bd[b].rb = s->rb_val_ptr[pq];
                    bd[b].bs = (int32_t)bs;
                }
            }
        }
        if ((rc = upload(h->d_sn, snd, bytes))) return fail(rc);
        if ((rc = upload(h->d_blk, bd, bytes))) return fail(rc);
        if ((rc = upload(h->d_rbval, s->rb_val, bytes))) return fail(rc);
    }
    *out = h;
    return SC_OK;
}

int numeric_factor(sc_numeric *h, const double *values, int on_device, cudaStream_t st, sc_factor_info *info) {
    const sc_symbolic *s = h->sym;
    int64_t nnz = (int64_t)s->valmap.size();
    h->last_stream = st;
    if (h->stall_factor_chunk >= 0) {
        // test hook: this factorization's units that read the chunk wait for one
        // more POTRF / TRSM completion than will come; their bounded waits give up
        const int32_t c = h->stall_factor_chunk;
        h->stall_factor_chunk = -1;
        if (!h->fused || c >= (int32_t)s->chunks.size()) return SC_ERR_UNSUPPORTED;
        int32_t need = 0;
        SC_CUDA(cudaMemcpy(&need, h->d_flow_need + c, sizeof(need), cudaMemcpyDeviceToHost));
        const int32_t raised = need + 1;
        SC_CUDA(cudaMemcpy(h->d_flow_need + c, &raised, sizeof(raised), cudaMemcpyHostToDevice));
        const int rc = numeric_factor(h, values, on_device, st, info);
        cudaStreamSynchronize(st);
        SC_CUDA(cudaMemcpy(h->d_flow_need + c, &need, sizeof(need), cudaMemcpyHostToDevice));
        return rc;
    }
    SC_CUDA(cudaMemcpyAsync(h->d_values, values, nnz * sizeof(double),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    SC_CUDA(cudaEventCreate(&e0));
    SC_CUDA(cudaEventCreate(&e1));
    SC_CUDA(cudaEventRecord(e0, st));
    int rc = SC_OK;
    if (h->use_graph) {
        if (!h->gexec) {
            // captured once on the handle's own stream (the legacy default stream
            // cannot be captured), then replayed on the caller's stream
            if (!h->cap_stream) SC_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            if (!h->cap_stream2) SC_CUDA(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
            if (!h->ev_fork) SC_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            if (!h->ev_join) SC_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
            cudaStream_t st3 = nullptr;
            if (h->lookahead) {
                if (!h->cap_stream3) SC_CUDA(cudaStreamCreateWithFlags(&h->cap_stream3, cudaStreamNonBlocking));
                if (!h->ev_trsm) SC_CUDA(cudaEventCreateWithFlags(&h->ev_trsm, cudaEventDisableTiming));
                for (auto &e : h->ev_rest)
                    if (!e) SC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                st3 = h->cap_stream3;
            }
            cudaGraph_t g;
            SC_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = h->precision == SC_FP64 ? run_levels<double>(h, h->cap_stream, nullptr, h->cap_stream2, st3)
                                         : run_levels<float>(h, h->cap_stream, nullptr, h->cap_stream2, st3);
            cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
            if (rc) return rc;
            SC_CUDA(ce);
            SC_CUDA(cudaGraphInstantiate(&h->gexec, g, 0));
            cudaGraphDestroy(g);
        }
        SC_CUDA(cudaGraphLaunch(h->gexec, st));
    } else {
        rc = h->precision == SC_FP64 ? run_levels<double>(h, st) : run_levels<float>(h, st);
        if (rc) return rc;
    }
    SC_CUDA(cudaEventRecord(e1, st));
    int32_t hinfo[2], herr = 0;
    SC_CUDA(cudaMemcpyAsync(hinfo, h->d_info, sizeof(hinfo), cudaMemcpyDeviceToHost, st));
    SC_CUDA(cudaMemcpyAsync(&herr, h->d_err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    SC_CUDA(cudaStreamSynchronize(st));
    if (herr) return SC_ERR_TIMEOUT;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int64_t failed = 0;
    if (hinfo[0] != 0x7f7f7f7f) failed = (int64_t)s->perm[hinfo[0] - 1] + 1;
    if (info) {
        info->failed_col = failed;
        info->precision = h->precision;
        info->pivot_fallbacks = hinfo[1];
        info->flops = s->flops;
        info->factor_ms = ms;
        info->device_bytes = h->device_bytes;
        info->kernel_launches = h->kernel_launches;
    }
    return failed ? (int)std::min<int64_t>(failed, INT32_MAX) : SC_OK;
}

int numeric_profile(sc_numeric *h, const double *values, int on_device, cudaStream_t st, double *ms, double *flops,
                    int32_t *launches) {
    const sc_symbolic *s = h->sym;
    int64_t nnz = (int64_t)s->valmap.size();
    h->last_stream = st;
    SC_CUDA(cudaMemcpyAsync(h->d_values, values, nnz * sizeof(double),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    Prof prof;
    prof.st = st;
    int rc = h->precision == SC_FP64 ? run_levels<double>(h, st, &prof) : run_levels<float>(h, st, &prof);
    SC_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < kProfClasses; c++) {
        ms[c] = 0.0;
        flops[c] = h->class_flops[c];
        launches[c] = 0;
    }
    for (auto &e : prof.ev) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e.second.first, e.second.second);
        ms[e.first] += t;
        launches[e.first]++;
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    return rc;
}

int numeric_export_L(const sc_numeric *h, double *out) {
    const sc_symbolic *s = h->sym;
    if (h->last_stream) SC_CUDA(cudaStreamSynchronize(h->last_stream));
    std::vector<unsigned char> buf((size_t)s->lnz_size * h->elt);
    SC_CUDA(cudaMemcpy(buf.data(), h->d_lnz, buf.size(), cudaMemcpyDeviceToHost));
    int64_t o = 0;
    for (int64_t J = 0; J < s->nsuper; J++) {
        int32_t w = s->sup_ptr[J + 1] - s->sup_ptr[J];
        int64_t m = s->gl_ptr[J + 1] - s->gl_ptr[J];
        for (int64_t r = 0; r < m; r++)
            for (int32_t c = 0; c < w; c++) {
                int64_t e = s->lnz_off[J] + r * s->lnz_ld[J] + c;
                double v = h->elt == 8 ? ((const double *)buf.data())[e] : (double)((const float *)buf.data())[e];
                out[o++] = r >= c ? v : 0.0;
            }
    }
    return SC_OK;
}

void numeric_free(sc_numeric *h) {
    if (!h) return;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    for (auto &g : h->sg)
        if (g) cudaGraphExecDestroy(g);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
    if (h->cap_stream3) cudaStreamDestroy(h->cap_stream3);
    for (cudaEvent_t e : {h->ev_fork, h->ev_join, h->ev_trsm, h->ev_rest[0], h->ev_rest[1]})
        if (e) cudaEventDestroy(e);
    void *ptrs[] = {h->d_lnz, h->d_pool, h->d_valmap, h->d_values, h->d_diagpos, h->d_adiag, h->d_info,
                    h->d_chunks, h->d_potrf, h->d_trsm, h->d_gemm, h->d_small, h->d_tasks, h->d_rlpairs,
                    h->d_rlslabs, h->d_rlrelind, h->d_glbind, h->d_perm, h->d_csr_ptr, h->d_csr_col, h->d_csr_val,
                    h->d_csr_map, h->d_counters, h->d_xw, h->d_solve_tiles, h->d_sn, h->d_blk, h->d_rbval,
                    h->d_loops, h->d_tmaps, h->d_tmap_of_sn, h->d_err, h->d_inv, h->d_x, h->d_r, h->d_b, h->d_xbest, h->d_y, h->d_z, h->d_acc, h->d_red,
                    h->d_dep_ptr, h->d_dep, h->d_sync, h->d_serr, h->d_hi, h->d_lo, h->d_thin,
                    h->d_cgz, h->d_cgp, h->d_cgq, h->d_cgs, h->d_solve_units, h->d_flow, h->d_flow_ctr,
                    h->d_flow_need, h->d_task_chunk, h->d_sn_chunk};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->sym) h->sym->refs--;
    delete h;
}

}  // namespace sc
