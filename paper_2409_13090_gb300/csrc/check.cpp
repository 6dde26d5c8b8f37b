// Host-side check of the device schedule (sc_check_schedule in include/sc.h):
// recomputes, from the symbolic structures alone, every address range the
// factor kernels derive from a Task, a device-loop item or an RL assembly pair,
// and the level order those ranges rely on. It stands in for device-side bounds
// checks: nothing here touches the GPU.
#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "sc_internal.h"

namespace {

using namespace sc;

enum Violation : int64_t {
    kOk = 0,
    kSrcRange = 1,      // A or B rows / columns outside the source panel
    kTgtRange = 2,      // C outside the target panel or its columns
    kTrapezoid = 3,     // C not in the lower trapezoid of the target
    kNotAncestor = 4,   // target neither the source (in-panel update) nor an ancestor of it
    kOrder = 5,         // source columns not factored yet, or target already factored
    kCrit = 6,          // critical / other classification does not match the target's chunk level
    kRun = 7,           // a run B' does not map to consecutive rows of P
    kPool = 8,          // RL product outside the level's pool
    kRelind = 9,        // RL assembly entry outside Lnz(P) or above its diagonal
    kExclusive = 10,    // a plain (non-atomic) update outside the source's own panel
    kMap = 11,          // a target row / column is not the position in glbind(P) of the source's row
    kTcK = 12,          // a product the tensor-core precisions route to tcgen05 would multiply
                        // panel columns past its inner dimension (its K is not a whole number of
                        // MMA steps and real columns of the panel follow it)
};

struct Checker {
    const sc_symbolic *s;
    std::vector<int32_t> clevel;      // chunk -> level
    std::vector<int32_t> first_lv;    // supernode -> level of its first chunk
    std::vector<int32_t> last_lv;     // supernode -> level of its last chunk
    std::vector<int32_t> by_off;      // supernodes sorted by Lnz offset
    Knobs kn;                         // the handle's launch-plan settings

    explicit Checker(const sc_symbolic *s_) : s(s_), kn(knobs_of(s_->tune)) {
        clevel.assign(s->chunks.size(), -1);
        for (size_t lv = 0; lv < s->levels.size(); lv++)
            for (int32_t c : s->levels[lv].chunks) clevel[c] = (int32_t)lv;
        first_lv.assign(s->nsuper, 1 << 30);
        last_lv.assign(s->nsuper, -1);
        for (size_t c = 0; c < s->chunks.size(); c++) {
            const int32_t J = s->chunks[c].sn;
            first_lv[J] = std::min(first_lv[J], clevel[c]);
            last_lv[J] = std::max(last_lv[J], clevel[c]);
        }
        by_off.resize(s->nsuper);
        for (int64_t J = 0; J < s->nsuper; J++) by_off[J] = (int32_t)J;
        std::sort(by_off.begin(), by_off.end(), [&](int32_t a, int32_t b) { return s->lnz_off[a] < s->lnz_off[b]; });
    }
    int64_t m_of(int32_t J) const { return s->gl_ptr[J + 1] - s->gl_ptr[J]; }
    const int32_t *gl(int32_t J) const { return s->glbind.data() + s->gl_ptr[J]; }
    // rows [jr, jr + cnt) of glbind(J) are rows [pr, pr + cnt) of glbind(P): the
    // definition of where a product entry lands (the relind maps are not used)
    bool same_rows(int32_t J, int64_t jr, int32_t P, int64_t pr, int64_t cnt) const {
        const int32_t *a = gl(J) + jr, *b = gl(P) + pr;
        for (int64_t i = 0; i < cnt; i++)
            if (a[i] != b[i]) return false;
        return true;
    }
    int32_t n_of(int32_t J) const { return s->sup_ptr[J + 1] - s->sup_ptr[J]; }
    int32_t col_level(int32_t global_col) const { return clevel[s->chunk_of_col[global_col]]; }
    bool is_ancestor(int32_t P, int32_t J) const {
        for (int32_t a = s->sup_parent[J]; a >= 0; a = s->sup_parent[a])
            if (a == P) return true;
        return false;
    }
    // supernode whose panel holds element offset off, or -1
    int32_t owner_of(int64_t off) const {
        auto it = std::upper_bound(by_off.begin(), by_off.end(), off,
                                   [&](int64_t v, int32_t J) { return v < s->lnz_off[J]; });
        if (it == by_off.begin()) return -1;
        const int32_t P = *(it - 1);
        return off < s->lnz_off[P] + m_of(P) * s->lnz_ld[P] ? P : -1;
    }

    int64_t task(const Task &t, int32_t lv, bool rl, int64_t pool) const {
        const int32_t J = t.src;
        if (J < 0 || J >= s->nsuper || t.m < 1 || t.n < 1 || t.k < 1) return kSrcRange;
        const int64_t offJ = s->lnz_off[J], ldJ = s->lnz_ld[J], mJ = m_of(J);
        const int32_t nJ = n_of(J);
        if (t.lds != ldJ || t.kx0 < 0 || t.kx0 + t.k > nJ || t.a_row < 0 || t.a_row + t.m > mJ || t.b_row < 0 ||
            t.b_row + t.n > mJ || t.a_off != offJ + t.a_row * ldJ + t.kx0 || t.b_off != offJ + t.b_row * ldJ + t.kx0)
            return kSrcRange;
        // the columns read are factored at this level or before
        if (col_level(s->sup_ptr[J] + t.kx0 + t.k - 1) > lv) return kOrder;
        // tensor-core tiles (TF32 / TF32x3 plans) multiply K in whole MMA steps:
        // the columns consumed past kx0 + k must be the panel's zero padding
        if (tc_route_width(t, nJ, kn.tc_min_k, kn.tc_wide_n, s->test_tc_ignore_tail)) {
            const int64_t consumed = (int64_t)t.kx0 + (t.k + kTcKStep - 1) / kTcKStep * kTcKStep;
            if (consumed > t.kx0 + t.k && t.kx0 + t.k < nJ) return kTcK;
        }
        const bool lower = t.flags & kTaskLower;
        if (t.flags & kTaskStoreU) {
            if (!rl || t.ldc < t.n || t.c_off < 0 || t.c_off + (int64_t)(t.m - 1) * t.ldc + t.n > pool) return kPool;
            return kOk;
        }
        const int32_t P = owner_of(t.c_off);
        if (P < 0) return kTgtRange;
        const int64_t local = t.c_off - s->lnz_off[P], ldP = s->lnz_ld[P];
        const int64_t row0 = local / ldP, col0 = local % ldP;
        if (t.ldc != ldP || col0 + t.n > n_of(P) || row0 + t.m > m_of(P)) return kTgtRange;
        if (lower ? row0 != col0 : row0 < col0 + t.n) return kTrapezoid;
        if (!same_rows(J, t.a_row, P, row0, t.m) || !same_rows(J, t.b_row, P, col0, t.n)) return kMap;
        if (P == J) {
            if (!(t.flags & kTaskExclusive) || col0 < t.kx0 + t.k) return kNotAncestor;
        } else {
            if (t.flags & kTaskExclusive) return kExclusive;
            if (!is_ancestor(P, J)) return kNotAncestor;
            if (first_lv[P] <= lv) return kOrder;
        }
        const int32_t tcol = s->sup_ptr[P] + (int32_t)col0;
        if (col_level(tcol) <= lv) return kOrder;
        if (!rl) {
            if (t.tcol != tcol) return kCrit;
            const bool crit = (t.flags & kTaskCrit) != 0;
            if (crit != (col_level(tcol) == lv + 1)) return kCrit;
        }
        return kOk;
    }

    // One device-loop item: the SYRK on B (when r_lo == b) and the runs B'
    // starting in [max(r_lo, b + 1), r_hi), as the loop kernels walk them.
    int64_t item(const LoopItem &it, int32_t lv, int64_t &products) const {
        const int32_t J = it.sn;
        if (J < 0 || J >= s->nsuper) return kSrcRange;
        const int64_t b0 = s->blk_ptr[J], b1 = s->blk_ptr[J + 1];
        if (it.b < b0 || it.b >= b1 || it.r_lo < it.b || it.r_hi > b1 || it.r_lo > it.r_hi) return kSrcRange;
        if (last_lv[J] != lv) return kOrder;
        const int32_t nJ = n_of(J);
        const int64_t mJ = m_of(J);
        std::vector<int64_t> pos(b1 - b0);
        int64_t q = nJ;
        for (int64_t b = b0; b < b1; b++) {
            pos[b - b0] = q;
            q += s->blk_size[b];
        }
        if (q != mJ) return kSrcRange;
        const int32_t P = s->blk_owner[it.b];
        if (!is_ancestor(P, J)) return kNotAncestor;
        if (first_lv[P] <= lv) return kOrder;
        // the (J, P) pair and its relindB entries
        int64_t pq = -1;
        for (int64_t x = s->rb_pair_ptr[J]; x < s->rb_pair_ptr[J + 1]; x++)
            if (s->rb_pair_P[x] == P) pq = x;
        if (pq < 0) return kRun;
        const int32_t *rb = s->rb_val.data() + s->rb_val_ptr[pq];
        const int64_t bs = b1 - (s->rb_val_ptr[pq + 1] - s->rb_val_ptr[pq]);
        if (it.b < bs) return kRun;
        const int64_t mP = m_of(P);
        const int32_t colB = s->blk_first[it.b] - s->sup_ptr[P], nb = s->blk_size[it.b];
        if (colB < 0 || colB + nb > n_of(P)) return kTgtRange;
        if (pos[it.b - b0] + nb > mJ) return kSrcRange;
        if (!same_rows(J, pos[it.b - b0], P, colB, nb)) return kMap;
        if (it.r_lo == it.b) {
            if (mP - 1 - rb[it.b - bs] != colB) return kTrapezoid;
            products++;
        }
        int64_t r = it.r_lo == it.b ? it.b + 1 : it.r_lo;
        while (r < it.r_hi) {
            int64_t e = r;
            int64_t rows = s->blk_size[r];
            while (e + 1 < b1 && s->blk_first[e + 1] == s->blk_first[e] + s->blk_size[e]) {
                e++;
                rows += s->blk_size[e];
            }
            if (r < bs || e >= b1) return kRun;
            const int64_t rowP = mP - 1 - rb[r - bs];
            if (rowP < 0 || rowP + rows > mP) return kTgtRange;
            if (rowP < colB + nb) return kTrapezoid;
            if (pos[r - b0] + rows > mJ) return kSrcRange;
            if (!same_rows(J, pos[r - b0], P, rowP, rows)) return kMap;
            for (int64_t x = r; x <= e; x++)
                if (mP - 1 - rb[x - bs] != rowP + (s->blk_first[x] - s->blk_first[r])) return kRun;
            products++;
            r = e + 1;
        }
        return kOk;
    }

    // RL assembly: entry (r, c) of U_J, c_begin <= c <= r < s, goes to
    // Lnz(P)[m_P - 1 - ri[r]][m_P - 1 - ri[c]].
    int64_t pair(const RLPair &p, int32_t J, int64_t pool, int64_t &entries) const {
        if (p.c_begin < 0 || p.c_end > p.s || p.c_begin >= p.c_end || p.u_off < 0 ||
            p.u_off + (int64_t)p.s * p.s > pool)
            return kPool;
        const int32_t P = owner_of(p.p_off);
        if (P < 0 || p.p_off != s->lnz_off[P] || p.ldp != s->lnz_ld[P] || p.mP != m_of(P) || p.fP != s->sup_ptr[P])
            return kTgtRange;
        if (p.ri_off < 0 || p.ri_off + (p.s - p.c_begin) > (int64_t)s->rl_relind.size()) return kRelind;
        const int32_t *ri = s->rl_relind.data() + p.ri_off;
        const int32_t nrows = p.s - p.c_begin, ncols = p.c_end - p.c_begin;
        if (J < 0 || p.s != m_of(J) - n_of(J) || !is_ancestor(P, J)) return kNotAncestor;
        const int32_t *SJ = gl(J) + n_of(J);  // row r of U_J is global row SJ[r]
        for (int32_t x = 0; x < nrows; x++) {
            const int64_t row = p.mP - 1 - (int64_t)ri[x];
            if (row < 0 || row >= p.mP) return kRelind;
            if (gl(P)[row] != SJ[p.c_begin + x]) return kMap;
            if (x < ncols && row >= n_of(P)) return kRelind;  // an assembled column lies inside P
            if (x > 0 && ri[x] >= ri[x - 1]) return kRelind;  // rows ascend in P as in U_J
        }
        entries += (int64_t)ncols * nrows;
        return kOk;
    }
};

}  // namespace

extern "C" int sc_check_schedule(const sc_symbolic *s, int64_t *out, int nout) {
    if (!s) return -1;
    if (nout > 0 && !out) return -2;
    try {
        Checker ck(s);
        int64_t tasks = 0, products = 0, entries = 0, bad_level = -1, bad_kind = 0;
        for (size_t lv = 0; lv < s->levels.size() && !bad_kind; lv++) {
            const Level &L = s->levels[lv];
            for (const Task &t : L.tasks) {
                tasks++;
                if ((bad_kind = ck.task(t, (int32_t)lv, false, 0))) break;
            }
            for (size_t i = 0; !bad_kind && i < L.rl_tasks.size(); i++) {
                tasks++;
                bad_kind = ck.task(L.rl_tasks[i], (int32_t)lv, true, L.rl_pool);
            }
            for (size_t i = 0; !bad_kind && i < L.loops.size(); i++)
                bad_kind = ck.item(L.loops[i], (int32_t)lv, products);
            if (!bad_kind && !L.rl_pairs.empty()) {
                std::vector<std::pair<int64_t, int32_t>> u_of;  // pool offset of U_J -> J
                for (const Task &t : L.rl_tasks) u_of.emplace_back(t.c_off, t.src);
                std::sort(u_of.begin(), u_of.end());
                for (size_t i = 0; !bad_kind && i < L.rl_pairs.size(); i++) {
                    auto it = std::lower_bound(u_of.begin(), u_of.end(), std::make_pair(L.rl_pairs[i].u_off, INT32_MIN));
                    const int32_t J = it != u_of.end() && it->first == L.rl_pairs[i].u_off ? it->second : -1;
                    bad_kind = ck.pair(L.rl_pairs[i], J, L.rl_pool, entries);
                }
            }
            if (bad_kind) bad_level = (int64_t)lv;
        }
        if (!bad_kind && s->opt.deterministic) bad_kind = det_plan_check(s, &bad_level);
        int64_t v[] = {tasks, products, entries, bad_level, bad_kind};
        for (int i = 0; i < nout && i < 5; i++) out[i] = v[i];
        return bad_kind ? SC_ERR_INTERNAL : SC_OK;
    } catch (...) {
        return SC_ERR_OOM;
    }
}

// Test hook: plants one mistake in the schedule of s so that a test can see
// sc_check_schedule find it. The handle is marked unusable: sc_factor and
// sc_tune refuse it.
extern "C" int sc_test_perturb_schedule(sc_symbolic *s, int kind) {
    if (!s) return -1;
    if (kind < 1 || kind > 6) return -2;
    if (kind == 6) {  // a deterministic plan whose first assembly slab misses a touched row
        for (const auto &L : s->levels)
            if (!L.rl_pairs.empty() && s->opt.deterministic) {
                s->test_det_short_slab = true;
                s->poisoned = true;
                return SC_OK;
            }
        return SC_ERR_UNSUPPORTED;
    }
    if (kind == 5) {  // tensor-core routing without the K-tail rule: only matters where a K tail exists
        const Knobs kn = knobs_of(s->tune);
        for (auto &L : s->levels)
            for (const Task &t : L.tasks) {
                const int32_t nJ = s->sup_ptr[t.src + 1] - s->sup_ptr[t.src];
                if (t.k % kTcKStep != 0 && t.kx0 + t.k < nJ && tc_route_width(t, nJ, kn.tc_min_k, kn.tc_wide_n, true)) {
                    s->test_tc_ignore_tail = true;
                    s->poisoned = true;
                    return SC_OK;
                }
            }
        return SC_ERR_UNSUPPORTED;
    }
    for (auto &L : s->levels) {
        for (Task &t : L.tasks) {
            const bool inpanel = t.flags & kTaskExclusive;
            if (kind == 1 && !inpanel && !(t.flags & kTaskLower)) {  // a GEMM target one row too high
                t.c_off -= t.ldc;
                s->poisoned = true;
                return SC_OK;
            }
            if (kind == 2 && (t.flags & kTaskCrit)) {  // a critical product marked as other
                t.flags &= ~kTaskCrit;
                s->poisoned = true;
                return SC_OK;
            }
            if (kind == 3 && inpanel) {  // an in-panel update reading one column too many
                t.k += 1;
                s->poisoned = true;
                return SC_OK;
            }
        }
        if (kind == 4)
            for (LoopItem &it : L.loops) {  // an item reaching past J's blocks
                it.r_hi = (int32_t)s->blk_ptr[it.sn + 1] + 1;
                s->poisoned = true;
                return SC_OK;
            }
    }
    return SC_ERR_UNSUPPORTED;  // no entry of that kind in this schedule
}
