// Level schedule of the numeric factorization (host side, precision independent).
//
// Every supernode J is cut into chunks of at most `chunk` columns. Chunks form
// a tree: chunk k of J is the child of chunk k+1 of J, and J's last chunk is a
// child of the first chunk of p(J). A chunk's level is its height in that tree,
// so all work of one level is independent and runs in one launch sequence.
//
// Per level:
//   - cdiv of each chunk: POTRF of its diagonal block, TRSM of the rows below;
//   - for a chunk that is not the last of J: trailing updates inside J,
//     deferred in levels (a chunk updates the rest of its 256-column macro
//     panel, K = chunk width; a macro panel's last chunk updates the rest of its
//     outer block, K = 256, and an outer block's last chunk every later column,
//     K = the outer width; with an outer width of 256 the macro panel's last
//     chunk updates all later columns at once; the default is 512);
//   - for J's last chunk (all of L_{*,J} is final):
//       RLB (Alg. 5): for every ancestor P, every block B of J inside P:
//         SYRK  L_{B,B}  -= L_{B,J} L_{B,J}^T
//         GEMM  L_{B',B} -= L_{B',J} L_{B,J}^T  for every maximal B' below B
//       each straight into Lnz(P) at the offsets given by relindB(J,P);
//       RL (Alg. 4): U_J = -L_{S,J} L_{S,J}^T into a pooled buffer,
//         then for each ancestor P the columns of U_J lying in P are added
//         into Lnz(P) through relind(J,P).
#include <algorithm>

#include "sc_internal.h"

namespace sc {

int build_schedule(sc_symbolic *s) {
    const int64_t ns = s->nsuper;
    const Knobs kn = knobs_of(s->tune);
    int32_t W = s->opt.chunk;
    if (W < 1) W = 64;
    if (W > 64) W = 64;
    s->chunks.clear();
    std::vector<int32_t> first_chunk(ns), last_chunk(ns);
    std::vector<int32_t> clevel;
    s->chunk_of_col.assign(s->n, 0);
    // children lists of the supernodal tree
    std::vector<int32_t> maxchild(ns, -1);  // max level over children's last chunks
    for (int64_t J = 0; J < ns; J++) {
        int32_t nJ = s->sup_ptr[J + 1] - s->sup_ptr[J];
        int32_t base = maxchild[J] + 1;
        first_chunk[J] = (int32_t)s->chunks.size();
        int32_t k = 0;
        for (int32_t c0 = 0; c0 < nJ; c0 += W, k++) {
            int32_t w = std::min(W, nJ - c0);
            s->chunks.push_back(Chunk{(int32_t)J, c0, w, c0 + w >= nJ ? 1 : 0});
            clevel.push_back(base + k);
            for (int32_t c = c0; c < c0 + w; c++) s->chunk_of_col[s->sup_ptr[J] + c] = (int32_t)s->chunks.size() - 1;
        }
        last_chunk[J] = (int32_t)s->chunks.size() - 1;
        int32_t P = s->sup_parent[J];
        if (P >= 0) maxchild[P] = std::max(maxchild[P], clevel[last_chunk[J]]);
    }
    int32_t nlev = 0;
    for (int32_t l : clevel) nlev = std::max(nlev, l + 1);
    s->levels.assign(nlev, Level{});
    for (size_t c = 0; c < s->chunks.size(); c++) {
        Level &L = s->levels[clevel[c]];
        L.chunks.push_back((int32_t)c);
        if (s->chunks[c].last) L.last_chunks.push_back((int32_t)c);
    }

    const bool rl = s->opt.variant == SC_RL;
    s->rl_relind.clear();
    s->rl_pool_max = 0;
    std::vector<int32_t> cur, nxt;
    for (int32_t lv = 0; lv < nlev; lv++) {
        Level &L = s->levels[lv];
        for (int32_t c : L.chunks) {
            const Chunk &ch = s->chunks[c];
            int32_t J = ch.sn;
            int32_t nJ = s->sup_ptr[J + 1] - s->sup_ptr[J];
            int64_t mJ = s->gl_ptr[J + 1] - s->gl_ptr[J];
            int32_t ldJ = s->lnz_ld[J];
            int64_t offJ = s->lnz_off[J];
            if (!ch.last) {
                // trailing updates inside J, deferred in levels of width W (the chunk),
                // Wm (macro panel) and Wd (outer block; Wd = Wm: two levels only): the
                // chunk ending at column e updates, with K = the width of the largest
                // level block ending at e, the columns from e to the end of the next
                // level's block (to nJ after an outer block). Every column before a
                // chunk is then applied to it before its POTRF. Targets lie in Lnz(J).
                const int32_t Wm = W * std::max(1, 256 / W);
                const int32_t Wd = Wm * std::max(1, kn.defer_width / Wm);
                const int32_t r0 = ch.c0 + ch.w;
                // the update of the next chunk's columns is split off, so the next
                // level's POTRF waits only for it (kTaskCrit, set below)
                auto lower_update = [&](int32_t c_first, int32_t c_end, int32_t kx0, int32_t K) {
                    const int32_t split = std::min(c_end, r0 + std::min(W, nJ - r0));
                    for (int32_t part = 0; part < 2; part++) {
                        const int32_t a = part == 0 ? c_first : split, e = part == 0 ? split : c_end;
                        if (a >= e) continue;
                        Task t;
                        t.a_off = offJ + (int64_t)a * ldJ + kx0;
                        t.b_off = t.a_off;
                        t.c_off = offJ + (int64_t)a * ldJ + a;
                        t.lds = ldJ;
                        t.ldc = ldJ;
                        t.m = (int32_t)(mJ - a);
                        t.n = e - a;
                        t.k = K;
                        t.flags = kTaskLower | kTaskExclusive;
                        t.src = J;
                        t.a_row = t.b_row = a;
                        t.kx0 = kx0;
                        t.tcol = s->sup_ptr[J] + a;
                        L.tasks.push_back(t);
                    }
                };
                if (r0 % Wm != 0) lower_update(r0, std::min(nJ, (r0 / Wm + 1) * Wm), ch.c0, ch.w);
                else if (Wd > Wm && r0 % Wd != 0) lower_update(r0, std::min(nJ, (r0 / Wd + 1) * Wd), r0 - Wm, Wm);
                else lower_update(r0, nJ, r0 - (Wd > Wm ? Wd : Wm), Wd > Wm ? Wd : Wm);
                continue;
            }
            int64_t b0 = s->blk_ptr[J], b1 = s->blk_ptr[J + 1];
            if (b1 == b0) continue;
            // position in glbind(J) of each block's first row
            std::vector<int64_t> bpos(b1 - b0);
            {
                int64_t q = nJ;
                for (int64_t b = b0; b < b1; b++) {
                    bpos[b - b0] = q;
                    q += s->blk_size[b];
                }
            }
            if (!rl) {
                // Alg. 5's loops over J's ancestors and blocks: large (B, B') products become tiled tasks;
                // the rest run on the device in items of bounded cost, each item
                // one block B and a range of the runs B' below it.
                const int64_t kLoopBudget = kn.loop_budget;
                for (int64_t q = s->rb_pair_ptr[J]; q < s->rb_pair_ptr[J + 1]; q++) {
                    int32_t P = s->rb_pair_P[q];
                    const int32_t *rb = s->rb_val.data() + s->rb_val_ptr[q];
                    int64_t cnt = s->rb_val_ptr[q + 1] - s->rb_val_ptr[q];
                    int64_t bs = b1 - cnt;  // first block at or above P
                    int32_t fP = s->sup_ptr[P];
                    int64_t mP = s->gl_ptr[P + 1] - s->gl_ptr[P];
                    int32_t ldP = s->lnz_ld[P];
                    int64_t offP = s->lnz_off[P];
                    for (int64_t b = bs; b < b1 && s->blk_owner[b] == P; b++) {
                        int64_t posB = mP - 1 - rb[b - bs];
                        int32_t colB = s->blk_first[b] - fP;
                        if (posB != colB) return SC_ERR_INTERNAL;
                        int32_t nb = s->blk_size[b];
                        LoopItem item{(int32_t)J, (int32_t)b, (int32_t)b, (int32_t)b};
                        int64_t cost = 0;
                        bool open = false;  // item holds work
                        long long tri = (long long)nb * (nb + 1) / 2;
                        if (tile_task(tri, nJ, kn.tile_min_entries, kn.tile_min_k)) {
                            Task t;
                            t.a_off = offJ + bpos[b - b0] * ldJ;
                            t.b_off = t.a_off;
                            t.c_off = offP + posB * ldP + colB;
                            t.lds = ldJ;
                            t.ldc = ldP;
                            t.m = t.n = nb;
                            t.k = nJ;
                            t.flags = kTaskLower;
                            t.src = J;
                            t.a_row = t.b_row = (int32_t)bpos[b - b0];
                            t.kx0 = 0;
                            t.tcol = fP + colB;
                            L.tasks.push_back(t);
                            item.r_lo = (int32_t)b + 1;  // no SYRK in the device loop
                        } else {
                            cost += tri * (nJ + 4);
                            open = true;
                            L.loop_flops += 2.0 * (double)tri * nJ;
                        }
                        // maximal blocks B' below B: runs of blocks whose rows abut
                        int64_t r = b + 1;
                        while (r < b1) {
                            int64_t e = r;
                            int32_t rows = s->blk_size[e];
                            while (e + 1 < b1 && s->blk_first[e + 1] == s->blk_first[e] + s->blk_size[e]) {
                                e++;
                                rows += s->blk_size[e];
                            }
                            if (tile_task((long long)rows * nb, nJ, kn.tile_min_entries, kn.tile_min_k)) {
                                Task g;
                                g.a_off = offJ + bpos[r - b0] * ldJ;
                                g.b_off = offJ + bpos[b - b0] * ldJ;
                                g.c_off = offP + (mP - 1 - rb[r - bs]) * ldP + colB;
                                g.lds = ldJ;
                                g.ldc = ldP;
                                g.m = rows;
                                g.n = nb;
                                g.k = nJ;
                                g.flags = 0;
                                g.src = J;
                                g.a_row = (int32_t)bpos[r - b0];
                                g.b_row = (int32_t)bpos[b - b0];
                                g.kx0 = 0;
                                g.tcol = fP + colB;
                                L.tasks.push_back(g);
                                // a tiled run ends the current item; the next item starts after it
                                if (open) {
                                    item.r_hi = (int32_t)r;
                                    L.loops.push_back(item);
                                }
                                item = LoopItem{(int32_t)J, (int32_t)b, (int32_t)(e + 1), (int32_t)(e + 1)};
                                cost = 0;
                                open = false;
                            } else {
                                int64_t c = (int64_t)rows * nb * (nJ + 4);
                                if (open && cost + c > kLoopBudget) {
                                    item.r_hi = (int32_t)r;
                                    L.loops.push_back(item);
                                    item = LoopItem{(int32_t)J, (int32_t)b, (int32_t)r, (int32_t)r};
                                    cost = 0;
                                }
                                cost += c;
                                open = true;
                                L.loop_flops += 2.0 * (double)rows * nb * nJ;
                            }
                            r = e + 1;
                        }
                        if (open) {
                            item.r_hi = (int32_t)b1;
                            L.loops.push_back(item);
                        }
                    }
                }
            } else {
                // RL: U_J = -L_{S,J} L_{S,J}^T into the level's pool
                int32_t sJ = (int32_t)(mJ - nJ);
                Task t;
                t.a_off = offJ + (int64_t)nJ * ldJ;
                t.b_off = t.a_off;
                t.c_off = L.rl_pool;
                t.lds = ldJ;
                t.ldc = sJ;
                t.m = t.n = sJ;
                t.k = nJ;
                t.flags = kTaskLower | kTaskStoreU;
                t.src = J;
                t.a_row = t.b_row = nJ;
                t.kx0 = 0;
                t.tcol = 0;
                L.rl_tasks.push_back(t);
                int64_t u_off = L.rl_pool;
                L.rl_pool += (int64_t)sJ * sJ;
                // walk the ancestors: relind(J,P) = relind(J,C) o relind(C,P) (Alg. 4's composition)
                const int32_t *S = s->glbind.data() + s->gl_ptr[J] + nJ;
                int32_t P = s->sup_parent[J];
                cur.assign(s->relind.begin() + s->ri_ptr[J], s->relind.begin() + s->ri_ptr[J + 1]);
                int32_t start = 0;  // rows of S_J still to be assembled: start..sJ-1
                int32_t C = J;
                while (start < sJ && P >= 0) {
                    if (C != J) {
                        int64_t lenCP = s->ri_ptr[C + 1] - s->ri_ptr[C];
                        nxt.resize(cur.size());
                        if (compose_relind(cur.data(), (int64_t)cur.size(), s->relind.data() + s->ri_ptr[C], lenCP,
                                           nxt.data()))
                            return SC_ERR_INTERNAL;
                        cur.swap(nxt);
                    }
                    int32_t fP = s->sup_ptr[P], lP = s->sup_ptr[P + 1] - 1;
                    int32_t cb = start, ce = start;
                    while (ce < sJ && S[ce] <= lP) ce++;
                    if (ce > cb) {
                        if (S[cb] < fP) return SC_ERR_INTERNAL;
                        RLPair pr;
                        pr.u_off = u_off;
                        pr.p_off = s->lnz_off[P];
                        pr.ri_off = (int64_t)s->rl_relind.size();
                        pr.s = sJ;
                        pr.c_begin = cb;
                        pr.c_end = ce;
                        pr.ldp = s->lnz_ld[P];
                        pr.mP = (int32_t)(s->gl_ptr[P + 1] - s->gl_ptr[P]);
                        pr.fP = fP;
                        pr.pad = 0;
                        s->rl_relind.insert(s->rl_relind.end(), cur.begin(), cur.end());
                        L.rl_pairs.push_back(pr);
                        // remove the assembled columns (Alg. 4)
                        cur.erase(cur.begin(), cur.begin() + (ce - cb));
                        start = ce;
                    }
                    C = P;
                    P = s->sup_parent[P];
                }
            }
        }
        s->rl_pool_max = std::max(s->rl_pool_max, L.rl_pool);
    }
    // a product is critical when its target lies in a chunk of the next level
    for (int32_t lv = 0; lv < nlev; lv++)
        for (Task &t : s->levels[lv].tasks)
            if (clevel[s->chunk_of_col[t.tcol]] == lv + 1) t.flags |= kTaskCrit;
    return SC_OK;
}

}  // namespace sc
