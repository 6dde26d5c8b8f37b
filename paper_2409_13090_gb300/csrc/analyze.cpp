// Host symbolic analysis of libsc (Sec. 1 steps 1-2, Sec. 2.1.2, Sec. 3.1 of
// arXiv 2409.13090): ordering, elimination tree, postorder, column counts,
// fundamental supernodes, supernodal elimination tree, partition refinement
// within supernodes, relind(J,p(J)), blocks and relindB(J,P) (Alg. 5), levels,
// factor-storage layout and the map from A's entries into it.
//
// Algorithms (chosen for O(nnz(L)) or better cost on multi-million-row inputs):
//   - nested dissection on a grid with an explicit work stack, or on the
//     matrix graph by level structures, optionally with multilevel bisection
//     (heavy-edge coarsening, seeded growth, FM refinement);
//   - elimination tree by Liu's algorithm with path compression;
//   - column counts by marking the row subtrees of the elimination tree;
//   - supernode structures by a union over child supernodes only;
//   - partition refinement with an in-place, array-based partition;
//   - relindB(J,P) by composition with relind(C,P), as Alg. 5 composes them.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <memory>
#include <numeric>
#include <queue>
#include <set>
#include <system_error>
#include <thread>

#include "sc_internal.h"

namespace sc {

namespace {

// Runs body(lo, hi) over [0, n) in blocks of `block`, taken from a shared
// counter by up to `threads` threads (the caller is one of them); the blocks
// must write disjoint data. Without a thread to be had the caller does the
// remaining blocks alone. An exception in a block stops the taking of new
// blocks and is rethrown to the caller once every thread has ended.
template <class F>
void parallel_blocks(int64_t n, int64_t block, int threads, const F &body) {
    std::atomic<int64_t> next{0};
    std::atomic<bool> failed{false};
    std::exception_ptr first;  // written once, by the thread that sets failed
    auto work = [&] {
        for (int64_t lo = next.fetch_add(block); lo < n && !failed.load(); lo = next.fetch_add(block)) {
            try {
                body(lo, std::min(n, lo + block));
            } catch (...) {
                if (!failed.exchange(true)) first = std::current_exception();
            }
        }
    };
    std::vector<std::thread> pool;
    const int64_t extra = std::min<int64_t>(threads, (n + block - 1) / block) - 1;
    for (int64_t t = 0; t < extra; t++) {
        try {
            pool.emplace_back(work);
        } catch (const std::system_error &) {
            break;
        }
    }
    work();
    for (auto &t : pool) t.join();
    if (first) std::rethrow_exception(first);
}

int validate(int64_t n, const int64_t *colptr, const int32_t *rowind) {
    if (n <= 0 || n > INT32_MAX - 1) return -1;
    if (!colptr) return -2;
    if (!rowind) return -3;
    if (colptr[0] != 0) return -2;
    for (int64_t j = 0; j < n; j++) {
        if (colptr[j + 1] <= colptr[j]) return -2;  // every column holds its diagonal
        if (rowind[colptr[j]] != j) return -3;      // diagonal present and first
        for (int64_t p = colptr[j] + 1; p < colptr[j + 1]; p++)
            if (rowind[p] <= rowind[p - 1] || rowind[p] >= n) return -3;
    }
    return SC_OK;
}

// Geometric nested dissection: a box of volume <= leaf is emitted in
// lexicographic order (x fastest); otherwise the longest axis (ties: x, y, z)
// is split at m = lo + len/2 and the order is left box, right box, plane m.
void grid_nd(int nx, int ny, int nz, int leaf, std::vector<int32_t> &perm) {
    struct Box { int lo[3], hi[3]; bool sep; };
    perm.clear();
    perm.reserve((size_t)nx * ny * nz);
    std::vector<Box> st;
    st.push_back(Box{{0, 0, 0}, {nx, ny, nz}, false});
    while (!st.empty()) {
        Box b = st.back();
        st.pop_back();
        int len[3] = {b.hi[0] - b.lo[0], b.hi[1] - b.lo[1], b.hi[2] - b.lo[2]};
        if (len[0] <= 0 || len[1] <= 0 || len[2] <= 0) continue;
        int64_t vol = (int64_t)len[0] * len[1] * len[2];
        if (b.sep || vol <= leaf) {
            for (int z = b.lo[2]; z < b.hi[2]; z++)
                for (int y = b.lo[1]; y < b.hi[1]; y++)
                    for (int x = b.lo[0]; x < b.hi[0]; x++) perm.push_back(x + nx * (y + ny * z));
            continue;
        }
        int ax = 0;
        for (int d = 1; d < 3; d++)
            if (len[d] > len[ax]) ax = d;
        int m = b.lo[ax] + len[ax] / 2;
        Box left = b, right = b, sep = b;
        left.hi[ax] = m;
        right.lo[ax] = m + 1;
        sep.lo[ax] = m;
        sep.hi[ax] = m + 1;
        sep.sep = true;
        // processed in the order left, right, separator (stack: push reversed)
        st.push_back(sep);
        st.push_back(right);
        st.push_back(left);
    }
}

// Full symmetric adjacency (no diagonal) of the lower-triangle CSC input.
// Multilevel bisection of a small weighted graph (local ids 0..n-1, adjacency
// lists sorted by neighbour id), every choice integer and tie-broken by id:
//  * coarsening: heavy-edge matching, vertices visited in increasing id, each
//    unmatched vertex takes the unmatched neighbour of largest edge weight
//    (ties: smaller vertex weight, then smaller id); coarse ids in visiting
//    order; repeated while more than 40 vertices remain (at most 30 times) and
//    a step keeps at most 95 % of the vertices;
//  * initial partition on the coarsest graph: from each of its first 32
//    vertices, breadth-first growth (neighbours in increasing id) of part 0
//    until it holds half the weight, then FM refinement; the smallest cut wins
//    (ties: better balance, then the earlier seed);
//  * uncoarsening: the partition is projected and refined again at every level;
//  * FM refinement: up to 8 passes; a pass moves, one at a time, the unlocked
//    boundary vertex of largest gain (cut decrease; ties smaller id) whose
//    move keeps every part at most 55 % of the weight, locks it, and stops
//    after 25 moves without a new best; it then returns to its best prefix.
//    Passes end when one finds no improvement.
namespace ml {

struct WGraph {
    std::vector<int64_t> vw;
    std::vector<std::vector<std::pair<int32_t, int64_t>>> adj;  // (neighbour, edge weight), ascending
    int32_t n() const { return (int32_t)vw.size(); }
};

constexpr int kCoarseMin = 40, kMaxLevels = 30, kSeeds = 32, kPasses = 8, kStall = 25;
constexpr int64_t kMinSet = 64;  // smaller sets take the level split only

WGraph coarsen(const WGraph &g, std::vector<int32_t> &cmap) {
    const int32_t n = g.n();
    std::vector<int32_t> match(n, -1);
    cmap.assign(n, -1);
    int32_t nc = 0;
    for (int32_t v = 0; v < n; v++) {
        if (match[v] >= 0) continue;
        int32_t best = -1;
        int64_t bw = 0;
        for (const auto &[u, w] : g.adj[v]) {
            if (match[u] >= 0 || u == v) continue;
            if (best < 0 || w > bw || (w == bw && g.vw[u] < g.vw[best])) {
                best = u;
                bw = w;
            }
        }
        if (best >= 0) {
            match[v] = best;
            match[best] = v;
            cmap[v] = cmap[best] = nc;
        } else {
            match[v] = v;
            cmap[v] = nc;
        }
        nc++;
    }
    WGraph c;
    c.vw.assign(nc, 0);
    c.adj.resize(nc);
    std::vector<std::vector<int32_t>> members(nc);
    for (int32_t v = 0; v < n; v++) {
        c.vw[cmap[v]] += g.vw[v];
        members[cmap[v]].push_back(v);
    }
    std::vector<int64_t> acc(nc, 0);
    std::vector<int32_t> touched;
    for (int32_t a = 0; a < nc; a++) {
        touched.clear();
        for (int32_t v : members[a])
            for (const auto &[u, w] : g.adj[v]) {
                const int32_t b = cmap[u];
                if (b == a) continue;
                if (acc[b] == 0) touched.push_back(b);
                acc[b] += w;
            }
        std::sort(touched.begin(), touched.end());
        for (int32_t b : touched) {
            c.adj[a].emplace_back(b, acc[b]);
            acc[b] = 0;
        }
    }
    return c;
}

int64_t cut_of(const WGraph &g, const std::vector<int8_t> &part) {
    int64_t c = 0;
    for (int32_t v = 0; v < g.n(); v++)
        for (const auto &[u, w] : g.adj[v])
            if (part[u] != part[v]) c += w;
    return c / 2;
}

void fm_refine(const WGraph &g, std::vector<int8_t> &part, int64_t maxw) {
    const int32_t n = g.n();
    const bool small = n <= 128;  // candidates found by a scan instead of an ordered set
    int64_t W[2] = {0, 0};
    for (int32_t v = 0; v < n; v++) W[part[v]] += g.vw[v];
    std::vector<int64_t> gain(n), ext(n);
    std::vector<char> locked(n);
    for (int pass = 0; pass < kPasses; pass++) {
        std::set<std::pair<int64_t, int32_t>> cand;  // (-gain, id) of unlocked boundary vertices
        for (int32_t v = 0; v < n; v++) {
            int64_t e = 0, i = 0;
            for (const auto &[u, w] : g.adj[v]) (part[u] != part[v] ? e : i) += w;
            ext[v] = e;
            gain[v] = e - i;
            locked[v] = 0;
            if (e > 0 && !small) cand.emplace(-gain[v], v);
        }
        std::vector<int32_t> moves;
        int64_t cum = 0, best = 0;
        size_t best_len = 0;
        int stall = 0;
        while (stall < kStall) {
            int32_t v = -1;
            if (small) {  // the same choice by a scan: largest gain, then smallest id
                for (int32_t u = 0; u < n; u++)
                    if (!locked[u] && ext[u] > 0 && W[1 - part[u]] + g.vw[u] <= maxw &&
                        (v < 0 || gain[u] > gain[v]))
                        v = u;
            } else {
                for (const auto &[ng, id] : cand)
                    if (W[1 - part[id]] + g.vw[id] <= maxw) {
                        v = id;
                        break;
                    }
            }
            if (v < 0) break;
            if (!small) cand.erase({-gain[v], v});
            const int8_t src = part[v], dst = 1 - src;
            cum += gain[v];
            part[v] = dst;
            W[src] -= g.vw[v];
            W[dst] += g.vw[v];
            locked[v] = 1;
            moves.push_back(v);
            gain[v] = -gain[v];
            for (const auto &[u, w] : g.adj[v]) {
                if (!small && !locked[u] && ext[u] > 0) cand.erase({-gain[u], u});
                if (part[u] == dst) {
                    gain[u] -= 2 * w;
                    ext[u] -= w;
                } else {
                    gain[u] += 2 * w;
                    ext[u] += w;
                }
                if (!small && !locked[u] && ext[u] > 0) cand.emplace(-gain[u], u);
            }
            if (cum > best) {
                best = cum;
                best_len = moves.size();
                stall = 0;
            } else {
                stall++;
            }
        }
        for (size_t q = moves.size(); q > best_len; q--) {
            const int32_t v = moves[q - 1];
            const int8_t src = part[v];
            part[v] = 1 - src;
            W[src] -= g.vw[v];
            W[1 - src] += g.vw[v];
        }
        if (best <= 0) break;
    }
}

std::vector<int8_t> bfs_grow(const WGraph &g, int32_t seed, int64_t half) {
    const int32_t n = g.n();
    std::vector<int8_t> part(n, 1);
    std::vector<char> seen(n, 0);
    std::vector<int32_t> queue{seed};
    seen[seed] = 1;
    int64_t got = 0;
    for (size_t h = 0; h < queue.size() && got < half; h++) {
        const int32_t v = queue[h];
        part[v] = 0;
        got += g.vw[v];
        for (const auto &[u, w] : g.adj[v])
            if (!seen[u]) {
                seen[u] = 1;
                queue.push_back(u);
            }
    }
    return part;
}

std::vector<int8_t> bisect(const WGraph &g0) {
    std::vector<WGraph> graphs;
    std::vector<std::vector<int32_t>> cmaps;
    graphs.push_back(g0);
    while (graphs.back().n() > kCoarseMin && (int)cmaps.size() < kMaxLevels) {
        std::vector<int32_t> cmap;
        WGraph c = coarsen(graphs.back(), cmap);
        if ((double)c.n() > 0.95 * (double)graphs.back().n()) break;
        cmaps.push_back(std::move(cmap));
        graphs.push_back(std::move(c));
    }
    int64_t total = 0;
    for (int64_t w : g0.vw) total += w;
    const int64_t maxw = (11 * total + 19) / 20;
    const WGraph &gc = graphs.back();
    std::vector<int8_t> part;
    int64_t best_cut = 0, best_bal = 0;
    for (int32_t seed = 0; seed < std::min<int32_t>(gc.n(), kSeeds); seed++) {
        std::vector<int8_t> p = bfs_grow(gc, seed, (total + 1) / 2);
        fm_refine(gc, p, maxw);
        int64_t w0 = 0;
        for (int32_t v = 0; v < gc.n(); v++)
            if (p[v] == 0) w0 += gc.vw[v];
        const int64_t cut = cut_of(gc, p), bal = std::llabs(total - 2 * w0);
        if (part.empty() || cut < best_cut || (cut == best_cut && bal < best_bal)) {
            part = std::move(p);
            best_cut = cut;
            best_bal = bal;
        }
    }
    for (size_t l = cmaps.size(); l > 0; l--) {
        const std::vector<int32_t> &cmap = cmaps[l - 1];
        std::vector<int8_t> fine(cmap.size());
        for (size_t v = 0; v < cmap.size(); v++) fine[v] = part[cmap[v]];
        part = std::move(fine);
        fm_refine(graphs[l - 1], part, maxw);
    }
    return part;
}

// Minimum vertex cover of the cut edges (König): a maximum matching between
// the boundary layers b0 (part 0, ascending) and b1, found by augmenting paths
// (Kuhn: each vertex of b0 in increasing order starts a depth-first search
// over its part-1 neighbours in increasing order, each part-1 vertex visited
// at most once per search); then Z = the vertices reachable from the
// unmatched vertices of b0 by alternating paths (any cut edge from part 0,
// matching edges from part 1), and the cover is (b0 minus Z) with (b1 in Z).
std::vector<int32_t> min_cover(const WGraph &g, const std::vector<int8_t> &part, const std::vector<int32_t> &b0) {
    const int32_t n = g.n();
    std::vector<int32_t> mate(n, -1), seen(n, -1);
    struct Frame {
        int32_t v;
        size_t next;
    };
    std::vector<Frame> stack;
    for (int32_t root : b0) {
        stack.assign(1, Frame{root, 0});
        bool found = false;
        while (!stack.empty() && !found) {
            Frame &f = stack.back();
            const auto &adj = g.adj[f.v];
            bool descended = false;
            while (f.next < adj.size()) {
                const int32_t u = adj[f.next].first;
                if (part[u] != 1 || seen[u] == root) {
                    f.next++;
                    continue;
                }
                seen[u] = root;
                if (mate[u] < 0) {
                    found = true;  // augment along the stack: each frame takes its current neighbour
                    break;
                }
                stack.push_back(Frame{mate[u], 0});
                descended = true;
                break;
            }
            if (found || descended) continue;
            stack.pop_back();
            if (!stack.empty()) stack.back().next++;
        }
        if (found)
            for (const Frame &f : stack) {
                const int32_t u = g.adj[f.v][f.next].first;
                mate[u] = f.v;
                mate[f.v] = u;
            }
    }
    std::vector<char> z(n, 0);
    std::vector<int32_t> todo;
    for (int32_t v : b0)
        if (mate[v] < 0) {
            z[v] = 1;
            todo.push_back(v);
        }
    while (!todo.empty()) {
        const int32_t v = todo.back();
        todo.pop_back();
        for (const auto &[u, w] : g.adj[v]) {
            if (part[u] != 1 || z[u]) continue;
            z[u] = 1;
            const int32_t x = mate[u];
            if (x >= 0 && !z[x]) {
                z[x] = 1;
                todo.push_back(x);
            }
        }
    }
    std::vector<int32_t> cover;
    for (int32_t v = 0; v < n; v++) {
        const bool boundary0 = part[v] == 0 && mate[v] >= 0;  // matched b0 vertices: the unmatched are in Z
        if ((boundary0 && !z[v]) || (part[v] == 1 && z[v])) cover.push_back(v);
    }
    return cover;
}

}  // namespace ml

// Nested dissection of a general graph (no coordinates), a stand-in for the
// paper's METIS ordering on inputs without a grid. For a vertex set S (sorted):
// |S| <= leaf: emit S ascending. Otherwise split S into the connected
// components of G[S] (found from their smallest vertex, in that order) and
// order each alone; a connected S is split by a breadth-first level structure
// from a pseudo-peripheral root (start at min S; up to 8 times move to the
// vertex of the last level with the fewest neighbours in S, ties to the smaller
// index, while that raises the eccentricity): the first level k with
// 2 |L_0 .. L_k| >= |S| is the separator, and the order is ND(levels < k),
// ND(levels > k), then level k ascending. Neighbours are visited ascending.
// With `multilevel`, a connected S of at least 64 vertices is also bisected
// by ml::bisect (unit weights) and its vertex separator taken as the smaller
// of the two boundary layers (ties: part 0's); that split is used when both
// remaining parts are non-empty and its separator is smaller than the level
// separator.
class GraphND {
  public:
    // threads: the top ceil(log2(threads)) levels of splits order their two
    // halves on two threads (halves of at least kForkMin vertices). Every
    // subproblem depends only on its own vertex set, so the order is the same
    // for any thread count.
    GraphND(int64_t n, const std::vector<int64_t> &ptr, const std::vector<int32_t> &adj, int leaf,
            std::vector<int32_t> &out, bool multilevel, int threads)
        : n_(n), ptr_(ptr), adj_(adj), leaf_(leaf), out_(out), inset_(new std::atomic<int32_t>[n]), seen_(n, 0),
          loc_(n, -1), multilevel_(multilevel) {
        for (int64_t v = 0; v < n; v++) inset_[v].store(0, std::memory_order_relaxed);
        while ((1 << fork_depth_) < threads) fork_depth_++;
    }

    // The order of all n vertices, written to out (resized to n).
    void run() {
        std::vector<int32_t> all(n_);
        std::iota(all.begin(), all.end(), 0);
        out_.assign(n_, -1);
        order(std::move(all), 0, 0);
    }

  private:
    static constexpr int64_t kForkMin = 2048;

    // A subproblem stamps its own vertices in inset_ and reads the stamps of
    // their neighbours, which a concurrent subproblem may be writing: relaxed
    // atomics (stamps are unique, so another set's stamp never matches).
    // seen_ and loc_ are read and written only at the subproblem's own vertices.
    bool in_set(int32_t u, int32_t st) const { return inset_[u].load(std::memory_order_relaxed) == st; }

    // Orders the vertex set S (sorted) into out_[off, off + |S|).
    void order(std::vector<int32_t> S, int64_t off, int depth) {
        if ((int64_t)S.size() <= leaf_) {
            std::copy(S.begin(), S.end(), out_.begin() + off);
            return;
        }
        const int32_t st = set_stamp_.fetch_add(1) + 1;
        for (int32_t v : S) inset_[v].store(st, std::memory_order_relaxed);
        // connected components of G[S]
        std::vector<std::vector<int32_t>> comps;
        const int32_t cs = seen_stamp_.fetch_add(1) + 1;
        for (int32_t v : S) {
            if (seen_[v] == cs) continue;
            std::vector<int32_t> comp{v};
            seen_[v] = cs;
            for (size_t h = 0; h < comp.size(); h++)
                for (int64_t p = ptr_[comp[h]]; p < ptr_[comp[h] + 1]; p++) {
                    const int32_t u = adj_[p];
                    if (in_set(u, st) && seen_[u] != cs) {
                        seen_[u] = cs;
                        comp.push_back(u);
                    }
                }
            std::sort(comp.begin(), comp.end());
            comps.push_back(std::move(comp));
        }
        if (comps.size() > 1) {
            for (auto &c : comps) {
                const int64_t size = (int64_t)c.size();
                order(std::move(c), off, depth);
                off += size;
            }
            return;
        }
        // pseudo-peripheral root and its level structure
        int32_t r = S[0];
        std::vector<std::vector<int32_t>> L = levels(r, st);
        for (int it = 0; it < 8; it++) {
            int32_t cand = -1, cdeg = 0;
            for (int32_t v : L.back()) {
                int32_t d = 0;
                for (int64_t p = ptr_[v]; p < ptr_[v + 1]; p++) d += in_set(adj_[p], st);
                if (cand < 0 || d < cdeg || (d == cdeg && v < cand)) {
                    cand = v;
                    cdeg = d;
                }
            }
            std::vector<std::vector<int32_t>> Lc = levels(cand, st);
            if (Lc.size() <= L.size()) break;
            r = cand;
            L = std::move(Lc);
        }
        size_t k = 0;
        int64_t cum = 0;
        for (; k < L.size(); k++) {
            cum += (int64_t)L[k].size();
            if (2 * cum >= (int64_t)S.size()) break;
        }
        std::vector<int32_t> left, right, sep = L[k];
        if (!multilevel_ || (int64_t)S.size() < ml::kMinSet || !ml_split(S, st, sep.size(), left, right, sep)) {
            for (size_t q = 0; q < L.size(); q++) {
                if (q < k) left.insert(left.end(), L[q].begin(), L[q].end());
                else if (q > k) right.insert(right.end(), L[q].begin(), L[q].end());
            }
        }
        std::sort(left.begin(), left.end());
        std::sort(right.begin(), right.end());
        std::sort(sep.begin(), sep.end());
        const int64_t nl = (int64_t)left.size(), nr = (int64_t)right.size();
        std::copy(sep.begin(), sep.end(), out_.begin() + off + nl + nr);
        S.clear();
        S.shrink_to_fit();
        if (depth < fork_depth_ && nl >= kForkMin && nr >= kForkMin) {
            std::exception_ptr err;
            std::thread t;
            try {
                t = std::thread([&] {
                    try {
                        order(std::move(left), off, depth + 1);
                    } catch (...) {
                        err = std::current_exception();
                    }
                });
            } catch (const std::system_error &) {  // no thread to be had: this one does both halves
                order(std::move(left), off, depth + 1);
                order(std::move(right), off + nl, depth + 1);
                return;
            }
            try {
                order(std::move(right), off + nl, depth + 1);
            } catch (...) {
                t.join();
                throw;
            }
            t.join();
            if (err) std::rethrow_exception(err);
            return;
        }
        order(std::move(left), off, depth + 1);
        order(std::move(right), off + nl, depth + 1);
    }

    // The multilevel split of the connected set S (sorted, stamped st): fills
    // left / right / sep and returns true when its separator is smaller than
    // level_sep vertices and both parts are non-empty.
    bool ml_split(const std::vector<int32_t> &S, int32_t st, size_t level_sep, std::vector<int32_t> &left,
                  std::vector<int32_t> &right, std::vector<int32_t> &sep) {
        const int32_t m = (int32_t)S.size();
        ml::WGraph g;
        g.vw.assign(m, 1);
        g.adj.resize(m);
        for (int32_t i = 0; i < m; i++) loc_[S[i]] = i;
        for (int32_t i = 0; i < m; i++)
            for (int64_t p = ptr_[S[i]]; p < ptr_[S[i] + 1]; p++)
                if (in_set(adj_[p], st)) g.adj[i].emplace_back(loc_[adj_[p]], 1);
        const std::vector<int8_t> part = ml::bisect(g);
        std::vector<int32_t> b[2];
        for (int32_t i = 0; i < m; i++)
            for (const auto &[u, w] : g.adj[i])
                if (part[u] != part[i]) {
                    b[part[i]].push_back(i);
                    break;
                }
        const int side = b[0].size() <= b[1].size() ? 0 : 1;
        std::vector<char> in_sep(m, 0);
        const std::vector<int32_t> cover = ml::min_cover(g, part, b[0]);
        for (int32_t i : cover.size() < b[side].size() ? cover : b[side]) in_sep[i] = 1;
        std::vector<int32_t> p0, p1, sp;
        for (int32_t i = 0; i < m; i++)
            (in_sep[i] ? sp : part[i] == 0 ? p0 : p1).push_back(S[i]);
        if (sp.empty() || p0.empty() || p1.empty() || level_sep <= sp.size()) return false;
        left = std::move(p0);
        right = std::move(p1);
        sep = std::move(sp);
        return true;
    }

    // breadth-first levels of G[S] (S = vertices stamped st) from root
    std::vector<std::vector<int32_t>> levels(int32_t root, int32_t st) {
        const int32_t bs = seen_stamp_.fetch_add(1) + 1;
        std::vector<std::vector<int32_t>> L{{root}};
        seen_[root] = bs;
        while (true) {
            std::vector<int32_t> next;
            for (int32_t v : L.back())
                for (int64_t p = ptr_[v]; p < ptr_[v + 1]; p++) {
                    const int32_t u = adj_[p];
                    if (in_set(u, st) && seen_[u] != bs) {
                        seen_[u] = bs;
                        next.push_back(u);
                    }
                }
            if (next.empty()) break;
            L.push_back(std::move(next));
        }
        return L;
    }

    const int64_t n_;
    const std::vector<int64_t> &ptr_;
    const std::vector<int32_t> &adj_;
    int64_t leaf_;
    std::vector<int32_t> &out_;
    std::unique_ptr<std::atomic<int32_t>[]> inset_;
    std::vector<int32_t> seen_, loc_;
    bool multilevel_;
    int fork_depth_ = 0;
    std::atomic<int32_t> set_stamp_{0}, seen_stamp_{0};
};

void build_adjacency(int64_t n, const int64_t *colptr, const int32_t *rowind, std::vector<int64_t> &ptr,
                     std::vector<int32_t> &adj) {
    ptr.assign(n + 1, 0);
    for (int64_t j = 0; j < n; j++)
        for (int64_t p = colptr[j] + 1; p < colptr[j + 1]; p++) {
            ptr[rowind[p] + 1]++;
            ptr[j + 1]++;
        }
    for (int64_t j = 0; j < n; j++) ptr[j + 1] += ptr[j];
    adj.resize(ptr[n]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t j = 0; j < n; j++)
        for (int64_t p = colptr[j] + 1; p < colptr[j + 1]; p++) {
            int32_t i = rowind[p];
            adj[fill[i]++] = (int32_t)j;
            adj[fill[j]++] = i;
        }
}

// Liu's elimination-tree algorithm with path compression, for the ordering
// perm (new -> old). parent[] in new labels, -1 for roots.
void etree_liu(int64_t n, const std::vector<int64_t> &aptr, const std::vector<int32_t> &adj,
               const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm, std::vector<int32_t> &parent) {
    parent.assign(n, -1);
    std::vector<int32_t> anc(n, -1);
    for (int64_t i = 0; i < n; i++) {
        int32_t io = perm[i];
        for (int64_t p = aptr[io]; p < aptr[io + 1]; p++) {
            int32_t k = iperm[adj[p]];
            if (k >= i) continue;
            int32_t r = k;
            while (anc[r] != -1 && anc[r] != i) {
                int32_t t = anc[r];
                anc[r] = (int32_t)i;
                r = t;
            }
            if (anc[r] == -1) {
                anc[r] = (int32_t)i;
                parent[r] = (int32_t)i;
            }
        }
    }
}

// Postorder: DFS from the roots in ascending order, children in ascending
// order; post[k] = the k-th vertex to finish.
void postorder(int64_t n, const std::vector<int32_t> &parent, std::vector<int32_t> &post) {
    std::vector<int32_t> head(n, -1), next(n, -1);
    for (int64_t j = n - 1; j >= 0; j--)
        if (parent[j] >= 0) {
            next[j] = head[parent[j]];
            head[parent[j]] = (int32_t)j;
        }
    post.clear();
    post.reserve(n);
    std::vector<int32_t> stack;
    std::vector<int32_t> cur(n);
    for (int64_t r = 0; r < n; r++) {
        if (parent[r] != -1) continue;
        stack.push_back((int32_t)r);
        cur[r] = head[r];
        while (!stack.empty()) {
            int32_t v = stack.back();
            int32_t c = cur[v];
            if (c != -1) {
                cur[v] = next[c];
                cur[c] = head[c];
                stack.push_back(c);
            } else {
                post.push_back(v);
                stack.pop_back();
            }
        }
    }
}

// Partition refinement of one supernode (the PR method cited in Sec. 1 and
// Sec. 3.1; its steps are not printed in the paper). Start from the parts
// [all columns, ascending]; for each set R (a descendant's rows inside this
// supernode, descendants in ascending order), split every part X that R cuts
// into X n R and X \ R, kept adjacent; X n R goes last when R meets a part
// after X and none before it, first otherwise; each part stays ascending.
// sets: local column indices. Output order[pos] = local column at position pos.
void refine(int32_t size, const std::vector<std::vector<int32_t>> &sets, std::vector<int32_t> &order) {
    order.resize(size);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int32_t> where(size), part_of(size, 0);
    std::iota(where.begin(), where.end(), 0);
    std::vector<int32_t> pstart{0}, pend{size};
    std::vector<int32_t> cnt(1, 0);
    std::vector<char> inR(size, 0);
    std::vector<int32_t> touched, tmp_in, tmp_out;
    for (const auto &R : sets) {
        touched.clear();
        for (int32_t x : R) {
            inR[x] = 1;
            int32_t p = part_of[where[x]];
            if (cnt[p]++ == 0) touched.push_back(p);
        }
        std::sort(touched.begin(), touched.end(), [&](int32_t a, int32_t b) { return pstart[a] < pstart[b]; });
        for (size_t t = 0; t < touched.size(); t++) {
            int32_t p = touched[t];
            int32_t s = pstart[p], e = pend[p];
            if (cnt[p] == e - s) continue;
            bool before = t > 0, after = t + 1 < touched.size();
            tmp_in.clear();
            tmp_out.clear();
            for (int32_t q = s; q < e; q++) (inR[order[q]] ? tmp_in : tmp_out).push_back(order[q]);
            const std::vector<int32_t> &first = (after && !before) ? tmp_out : tmp_in;
            const std::vector<int32_t> &second = (after && !before) ? tmp_in : tmp_out;
            int32_t q = s;
            for (int32_t x : first) { order[q] = x; where[x] = q; q++; }
            int32_t split = q;
            for (int32_t x : second) { order[q] = x; where[x] = q; q++; }
            int32_t np = (int32_t)pstart.size();
            pstart.push_back(split);
            pend.push_back(e);
            cnt.push_back(0);
            pend[p] = split;
            for (int32_t r = split; r < e; r++) part_of[r] = np;
        }
        for (int32_t p : touched) cnt[p] = 0;
        for (int32_t x : R) inR[x] = 0;
    }
}

// Supernode merging (Sec. 3.1): merge, one pair at a time, the child-parent
// pair adding the least new fill, while the total added fill stays within
// frac x the fundamental storage. A pair (X, p(X)) qualifies when X ends on the
// column just before p(X) starts (merged supernodes stay consecutive); the
// storage of w columns with m rows is w m - w (w - 1) / 2; merging X into P
// yields w = |X| + |P|, m = |X| + m_P; ties go to the smaller first column.
// Candidates live in an ordered set keyed by (fill, first column) and are
// re-keyed when a merge changes them. The merged supernode keeps P's rows
// below its last column (S_X lies inside P's columns and S_P).
void merge_supernodes(int64_t n, double frac, std::vector<int32_t> &sup_ptr, std::vector<int32_t> &sup_of,
                      const std::vector<int64_t> &cc, const std::vector<int32_t> &parent) {
    // A fundamental supernode X with last column l has |S_X| = cc[l] - 1 rows
    // below it, the first of them parent[l] (the etree parent of l); merging a
    // child into P changes neither P's last column nor its structure, so the
    // sizes and the parent column are all the merging needs.
    const int64_t ns = (int64_t)sup_ptr.size() - 1;
    auto trap = [](int64_t w, int64_t m) { return w * m - w * (w - 1) / 2; };
    // owner of a column: find() over the merges from its fundamental supernode
    // (rep[X] = the supernode X was merged into, path-halved)
    std::vector<int32_t> f(ns), l(ns), rep(ns);
    std::iota(rep.begin(), rep.end(), 0);
    auto find = [&](int32_t X) {
        while (rep[X] != X) {
            rep[X] = rep[rep[X]];
            X = rep[X];
        }
        return X;
    };
    auto own = [&](int32_t j) { return find(sup_of[j]); };
    std::vector<int64_t> w(ns), m(ns);
    std::vector<char> alive(ns, 1);
    int64_t S0 = 0;
    for (int64_t X = 0; X < ns; X++) {
        f[X] = sup_ptr[X];
        l[X] = sup_ptr[X + 1] - 1;
        w[X] = l[X] - f[X] + 1;
        m[X] = w[X] + (cc[l[X]] - 1);
        S0 += trap(w[X], m[X]);
    }
    auto parent_now = [&](int64_t X) -> int32_t {
        const int32_t r = parent[l[X]];
        return r < 0 ? -1 : own(r);
    };
    // Candidates ordered by (fill, first column), with lazy deletion: an entry
    // whose key is no longer X's current key is dropped when it comes to the
    // top. Fills below kSmall (most merges) sit in one bucket per fill, each a
    // min-heap of (first column, X); larger fills in one heap of (fill, first
    // column, X). The first valid entry of the lowest non-empty bucket, else
    // of the large heap, is the least current candidate. (fill >= 0: the
    // merged trapezoid holds X's columns padded to P's rows plus P itself.)
    typedef std::pair<int64_t, int32_t> Key;  // (fill, first column)
    typedef std::pair<Key, int32_t> Entry;
    typedef std::pair<int32_t, int32_t> Small;  // (first column, X)
    constexpr int64_t kSmall = 64;
    std::vector<std::vector<Small>> bucket(kSmall);
    int64_t lo = kSmall;  // buckets below lo are empty
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> large;
    std::vector<Key> key(ns, Key(-1, -1));
    auto refresh = [&](int32_t X) {
        key[X] = Key(-1, -1);
        if (!alive[X]) return;
        int32_t P = parent_now(X);
        if (P < 0 || l[X] + 1 != f[P]) return;
        int64_t fill = trap(w[X] + w[P], w[X] + m[P]) - trap(w[X], m[X]) - trap(w[P], m[P]);
        key[X] = Key(fill, f[X]);
        if (fill >= 0 && fill < kSmall) {
            bucket[fill].emplace_back(f[X], X);
            std::push_heap(bucket[fill].begin(), bucket[fill].end(), std::greater<Small>());
            lo = std::min(lo, fill);
        } else {
            large.push({key[X], X});
        }
    };
    // the least current candidate (X = -1: none); stale entries on the way are dropped
    auto least = [&](Key &k) -> int32_t {
        for (; lo < kSmall; lo++) {
            std::vector<Small> &h = bucket[lo];
            while (!h.empty()) {
                const int32_t X = h.front().second;
                if (alive[X] && key[X] == Key(lo, h.front().first)) {
                    k = key[X];
                    return X;
                }
                std::pop_heap(h.begin(), h.end(), std::greater<Small>());
                h.pop_back();
            }
        }
        while (!large.empty()) {
            const int32_t X = large.top().second;
            if (alive[X] && key[X] == large.top().first) {
                k = key[X];
                return X;
            }
            large.pop();
        }
        return -1;
    };
    auto drop = [&](const Key &k) {  // removes the entry least() returned
        if (k.first >= 0 && k.first < kSmall) {
            std::vector<Small> &h = bucket[k.first];
            std::pop_heap(h.begin(), h.end(), std::greater<Small>());
            h.pop_back();
        } else {
            large.pop();
        }
    };
    for (int32_t X = 0; X < ns; X++) refresh(X);
    int64_t added = 0;
    while (true) {
        Key k;
        const int32_t X = least(k);
        if (X < 0) break;
        int64_t fill = k.first;
        if ((double)(added + fill) > frac * (double)S0) break;
        int32_t P = parent_now(X);
        drop(k);
        key[X] = Key(-1, -1);
        added += fill;
        alive[X] = 0;
        rep[X] = P;
        m[P] += w[X];
        w[P] += w[X];
        f[P] = f[X];
        refresh(P);
        if (f[P] > 0) {
            int32_t C = own(f[P] - 1);
            if (alive[C] && parent_now(C) == P) refresh(C);
        }
    }
    // the surviving supernodes in column order
    std::vector<int32_t> nptr;
    for (int32_t X = 0; X < ns; X++)
        if (alive[X]) nptr.push_back(f[X]);
    nptr.push_back((int32_t)n);
    const int64_t nn = (int64_t)nptr.size() - 1;
    for (int64_t J = 0; J < nn; J++)
        for (int32_t j = nptr[J]; j < nptr[J + 1]; j++) sup_of[j] = (int32_t)J;
    sup_ptr.swap(nptr);
}

}  // namespace

int compose_relind(const int32_t *rJC, int64_t lenJC, const int32_t *rCP, int64_t lenCP, int32_t *out) {
    if (!rJC) return -1;
    if (lenJC < 0) return -2;
    if (!rCP) return -3;
    if (lenCP < 0) return -4;
    if (!out) return -5;
    for (int64_t k = 0; k < lenJC; k++) {
        int64_t d = rJC[k];
        if (d < 0 || d >= lenCP) return -1;
        out[k] = rCP[lenCP - 1 - d];
    }
    return SC_OK;
}

int analyze_impl(int64_t n, const int64_t *colptr, const int32_t *rowind, const sc_options &o, sc_symbolic **out) {
    int rc = validate(n, colptr, rowind);
    if (rc) return rc;
    auto s = std::make_unique<sc_symbolic>();
    s->n = n;
    s->opt = o;
    s->opt.tune = nullptr;
    if (o.tune) s->tune = *o.tune;
    int64_t nnzA = colptr[n];
    const int threads =
        o.threads > 0 ? o.threads : (int)std::min(64u, std::max(1u, std::thread::hardware_concurrency()));
    s->colptr.assign(colptr, colptr + n + 1);
    s->rowind.assign(rowind, rowind + nnzA);

    // ---- step 1: ordering
    std::vector<int32_t> p0;
    if (o.ordering == SC_ORDER_GRID_ND) {
        if ((int64_t)o.grid[0] * o.grid[1] * o.grid[2] != n || o.grid[0] <= 0 || o.grid[1] <= 0 || o.grid[2] <= 0 ||
            o.nd_leaf < 1)
            return -4;
        grid_nd(o.grid[0], o.grid[1], o.grid[2], o.nd_leaf, p0);
    } else if (o.ordering == SC_ORDER_USER) {
        if (!o.user_perm) return -4;
        p0.assign(o.user_perm, o.user_perm + n);
        std::vector<char> seen(n, 0);
        for (int64_t k = 0; k < n; k++) {
            if (p0[k] < 0 || p0[k] >= n || seen[p0[k]]) return -4;
            seen[p0[k]] = 1;
        }
    } else if (o.ordering == SC_ORDER_NATURAL) {
        p0.resize(n);
        std::iota(p0.begin(), p0.end(), 0);
    } else if (o.ordering != SC_ORDER_GRAPH_ND && o.ordering != SC_ORDER_GRAPH_ML) {
        return -4;
    }
    std::vector<int64_t> aptr;
    std::vector<int32_t> adj;
    build_adjacency(n, colptr, rowind, aptr, adj);
    if (o.ordering == SC_ORDER_GRAPH_ND || o.ordering == SC_ORDER_GRAPH_ML) {
        if (o.nd_leaf < 1) return -4;
        GraphND(n, aptr, adj, o.nd_leaf, p0, o.ordering == SC_ORDER_GRAPH_ML, threads).run();
        for (int64_t k = 0; k < n; k++)
            if (p0[k] < 0) return SC_ERR_INTERNAL;
    }
    std::vector<int32_t> ip0(n);
    for (int64_t k = 0; k < n; k++) ip0[p0[k]] = (int32_t)k;

    // ---- elimination tree and postorder
    std::vector<int32_t> par0;
    etree_liu(n, aptr, adj, p0, ip0, par0);
    std::vector<int32_t> post;
    postorder(n, par0, post);
    std::vector<int32_t> p1(n), ip1(n), newof(n);
    for (int64_t k = 0; k < n; k++) {
        p1[k] = p0[post[k]];
        newof[post[k]] = (int32_t)k;
    }
    for (int64_t k = 0; k < n; k++) ip1[p1[k]] = (int32_t)k;
    std::vector<int32_t> parent(n);
    for (int64_t k = 0; k < n; k++) parent[k] = par0[post[k]] < 0 ? -1 : newof[par0[post[k]]];

    // ---- column counts in O(nnz(A) alpha) by the row-subtree leaf method of
    // Gilbert, Ng and Peyton (1994). cc[j] counts the rows i >= j whose row
    // subtree T_r(i) (the union of the etree paths from each j' < i with
    // A_ij' != 0, up to i) contains j. For a subtree T rooted at i with leaves
    // l_1 < ... < l_k in postorder, the weights +1 at every leaf, -1 at
    // lca(l_t-1, l_t) and -1 at parent(i) sum to [j in T] over the etree
    // subtree of any j; so cc[j] is the subtree sum of the weights of all rows.
    // With the columns visited in postorder, j is a leaf of T_r(i) when no
    // earlier neighbour of row i lies in j's subtree [first[j], j]; the lca of
    // the previous leaf and j is the lowest unfinished ancestor of the previous
    // leaf (a disjoint-set forest that links each finished column to its parent).
    std::vector<int64_t> cc(n, 0);
    {
        std::vector<int32_t> first(n, -1), prevnbr(n, -1), prevleaf(n, -1), anc(n);
        for (int64_t j = 0; j < n; j++)
            for (int64_t k = j; k >= 0 && first[k] < 0; k = parent[k]) first[k] = (int32_t)j;
        for (int64_t j = 0; j < n; j++) anc[j] = (int32_t)j;
        auto find = [&](int32_t x) {
            int32_t r = x;
            while (anc[r] != r) r = anc[r];
            while (anc[x] != r) {
                const int32_t nx = anc[x];
                anc[x] = r;
                x = nx;
            }
            return r;
        };
        auto visit = [&](int32_t i, int32_t j) {  // entry (i, j), i >= j, of the postordered A
            if (first[j] > prevnbr[i]) {          // j is a leaf of T_r(i)
                cc[j]++;
                if (prevleaf[i] >= 0) cc[find(prevleaf[i])]--;
                prevleaf[i] = j;
            }
            prevnbr[i] = j;
        };
        for (int64_t j = 0; j < n; j++) {
            visit((int32_t)j, (int32_t)j);
            const int32_t jo = p1[j];
            for (int64_t p = aptr[jo]; p < aptr[jo + 1]; p++) {
                const int32_t i = ip1[adj[p]];
                if (i > j) visit(i, (int32_t)j);
            }
            if (parent[j] >= 0) {
                cc[parent[j]]--;
                anc[j] = parent[j];
            }
        }
        for (int64_t j = 0; j < n; j++)
            if (parent[j] >= 0) cc[parent[j]] += cc[j];
    }

    // ---- fundamental supernodes
    std::vector<int32_t> nchild(n, 0);
    for (int64_t j = 0; j < n; j++)
        if (parent[j] >= 0) nchild[parent[j]]++;
    std::vector<int32_t> &sup_ptr = s->sup_ptr;
    sup_ptr.clear();
    for (int64_t j = 0; j < n; j++) {
        bool joins = j > 0 && parent[j - 1] == j && nchild[j] == 1 && cc[j - 1] == cc[j] + 1;
        if (!joins) sup_ptr.push_back((int32_t)j);
    }
    sup_ptr.push_back((int32_t)n);
    int64_t ns = (int64_t)sup_ptr.size() - 1;
    s->nsuper = ns;
    std::vector<int32_t> &sup_of = s->sup_of;
    sup_of.resize(n);
    for (int64_t J = 0; J < ns; J++)
        for (int32_t j = sup_ptr[J]; j < sup_ptr[J + 1]; j++) sup_of[j] = (int32_t)J;

    // ---- optional supernode merging (Sec. 3.1), before the structures and the
    // reordering within supernodes
    if (o.merge_frac > 0.0) {
        merge_supernodes(n, o.merge_frac, sup_ptr, sup_of, cc, parent);
        ns = (int64_t)sup_ptr.size() - 1;
        s->nsuper = ns;
    }

    // ---- supernode structures S_J (pre-PR labels), union over child supernodes
    std::vector<int64_t> sptr(ns + 1, 0);
    std::vector<int32_t> srows;
    srows.reserve(n * 4);
    std::vector<int32_t> spar(ns, -1);
    std::vector<int32_t> chead(ns, -1), cnext(ns, -1), ctail(ns, -1);
    {
        // S_J = (rows of A in J's columns, and the S_C of J's child supernodes) below J's
        // last column. The children's lists are sorted, so with few children they are
        // merged into the sorted entries of A; with many, marked and sorted at once.
        std::vector<int32_t> mark(n, -1);
        std::vector<int32_t> lst, tmp;
        for (int64_t J = 0; J < ns; J++) {
            int32_t f = sup_ptr[J], l = sup_ptr[J + 1] - 1;
            int nchildren = 0;
            for (int32_t C = chead[J]; C != -1; C = cnext[C]) nchildren++;
            lst.clear();
            for (int32_t j = f; j <= l; j++) {
                int32_t jo = p1[j];
                for (int64_t p = aptr[jo]; p < aptr[jo + 1]; p++) {
                    int32_t i = ip1[adj[p]];
                    if (i > l && mark[i] != J) {
                        mark[i] = (int32_t)J;
                        lst.push_back(i);
                    }
                }
            }
            if (nchildren <= 4) {
                std::sort(lst.begin(), lst.end());
                for (int32_t C = chead[J]; C != -1; C = cnext[C]) {
                    const int32_t *a = srows.data() + sptr[C], *ae = srows.data() + sptr[C + 1];
                    a = std::upper_bound(a, ae, l);
                    tmp.clear();
                    size_t q = 0;
                    while (a < ae || q < lst.size()) {
                        int32_t v;
                        if (q == lst.size() || (a < ae && *a < lst[q])) v = *a++;
                        else if (a == ae || lst[q] < *a) v = lst[q++];
                        else {
                            v = *a++;
                            q++;
                        }
                        tmp.push_back(v);
                    }
                    lst.swap(tmp);
                }
            } else {
                for (int32_t C = chead[J]; C != -1; C = cnext[C])
                    for (int64_t p = sptr[C]; p < sptr[C + 1]; p++) {
                        int32_t i = srows[p];
                        if (i > l && mark[i] != J) {
                            mark[i] = (int32_t)J;
                            lst.push_back(i);
                        }
                    }
                std::sort(lst.begin(), lst.end());
            }
            srows.insert(srows.end(), lst.begin(), lst.end());
            sptr[J + 1] = (int64_t)srows.size();
            // consistency with the column counts: S_J is the structure of J's last
            // column; the other columns' structures lie inside J's (equal for
            // fundamental supernodes, smaller where merging added zeros)
            int64_t m = (l - f + 1) + (int64_t)lst.size();
            if (cc[l] != m - (l - f)) return SC_ERR_INTERNAL;
            for (int32_t j = f; j < l; j++)
                if (cc[j] > m - (j - f) || (o.merge_frac <= 0.0 && cc[j] != m - (j - f))) return SC_ERR_INTERNAL;
            if (!lst.empty()) {
                int32_t P = sup_of[lst[0]];
                spar[J] = P;
                if (chead[P] == -1) chead[P] = (int32_t)J; else cnext[ctail[P]] = (int32_t)J;
                ctail[P] = (int32_t)J;
            }
        }
    }

    // sum over columns of |L_{*,j}|^2 of the true (fundamental) structure
    s->flops = 0.0;
    for (int64_t j = 0; j < n; j++) s->flops += (double)cc[j] * (double)cc[j];

    // ---- partition refinement within supernodes (on the pre-PR structure)
    std::vector<int32_t> p3 = p1;
    if (o.pr) {
        // R = S_J n P for each descendant J, grouped by P, ascending J
        std::vector<int64_t> nsets(ns + 1, 0);
        for (int64_t J = 0; J < ns; J++) {
            int32_t last = -1;
            for (int64_t p = sptr[J]; p < sptr[J + 1]; p++) {
                int32_t P = sup_of[srows[p]];
                if (P != last) { nsets[P + 1]++; last = P; }
            }
        }
        for (int64_t P = 0; P < ns; P++) nsets[P + 1] += nsets[P];
        std::vector<int64_t> set_owner_fill(nsets.begin(), nsets.end() - 1);
        std::vector<int64_t> set_lo(nsets[ns]), set_hi(nsets[ns]);
        for (int64_t J = 0; J < ns; J++) {
            int64_t p = sptr[J];
            while (p < sptr[J + 1]) {
                int32_t P = sup_of[srows[p]];
                int64_t q = p;
                while (q < sptr[J + 1] && sup_of[srows[q]] == P) q++;
                int64_t slot = set_owner_fill[P]++;
                set_lo[slot] = p;
                set_hi[slot] = q;
                p = q;
            }
        }
        // each P reorders only its own columns: blocks of supernodes on the host threads
        parallel_blocks(ns, 64, threads, [&](int64_t P0, int64_t P1) {
            std::vector<std::vector<int32_t>> sets;
            std::vector<int32_t> order;
            for (int64_t P = P0; P < P1; P++) {
                int32_t f = sup_ptr[P], size = sup_ptr[P + 1] - f;
                if (size < 2 || nsets[P + 1] == nsets[P]) continue;
                sets.clear();
                for (int64_t q = nsets[P]; q < nsets[P + 1]; q++) {
                    sets.emplace_back();
                    for (int64_t p = set_lo[q]; p < set_hi[q]; p++) sets.back().push_back(srows[p] - f);
                }
                refine(size, sets, order);
                for (int32_t k = 0; k < size; k++) p3[f + k] = p1[f + order[k]];
            }
        });
    }
    // labels after PR
    std::vector<int32_t> lab(n);  // lab[pre-PR label] = final label
    {
        std::vector<int32_t> ip3(n);
        for (int64_t k = 0; k < n; k++) ip3[p3[k]] = (int32_t)k;
        for (int64_t k = 0; k < n; k++) lab[k] = ip3[p1[k]];
    }
    s->perm = p3;
    s->iperm.resize(n);
    for (int64_t k = 0; k < n; k++) s->iperm[p3[k]] = (int32_t)k;

    // ---- glbind(J) = J's columns followed by the relabelled S_J, ascending
    s->gl_ptr.assign(ns + 1, 0);
    for (int64_t J = 0; J < ns; J++)
        s->gl_ptr[J + 1] = s->gl_ptr[J] + (sup_ptr[J + 1] - sup_ptr[J]) + (sptr[J + 1] - sptr[J]);
    s->glbind.resize(s->gl_ptr[ns]);
    parallel_blocks(ns, 256, threads, [&](int64_t J0, int64_t J1) {
        for (int64_t J = J0; J < J1; J++) {
            int64_t w = s->gl_ptr[J];
            for (int32_t j = sup_ptr[J]; j < sup_ptr[J + 1]; j++) s->glbind[w++] = j;
            int64_t b = w;
            for (int64_t p = sptr[J]; p < sptr[J + 1]; p++) s->glbind[w++] = lab[srows[p]];
            std::sort(s->glbind.begin() + b, s->glbind.begin() + w);
        }
    });
    s->sup_parent = spar;
    s->nnzL = 0;
    for (int64_t J = 0; J < ns; J++) {
        int64_t m = s->gl_ptr[J + 1] - s->gl_ptr[J];
        for (int32_t c = 0; c < sup_ptr[J + 1] - sup_ptr[J]; c++) s->nnzL += m - c;
    }
    // column elimination tree of the final ordering
    etree_liu(n, aptr, adj, s->perm, s->iperm, s->cparent);

    // ---- relind(J, p(J)) through a position map of glbind(P) (Sec. 2.1.2)
    s->ri_ptr.assign(ns + 1, 0);
    for (int64_t J = 0; J < ns; J++) s->ri_ptr[J + 1] = s->ri_ptr[J] + (spar[J] >= 0 ? sptr[J + 1] - sptr[J] : 0);
    s->relind.resize(s->ri_ptr[ns]);
    {
        std::vector<int32_t> dist(n, -1);
        for (int64_t P = 0; P < ns; P++) {
            if (chead[P] == -1) continue;
            int64_t m = s->gl_ptr[P + 1] - s->gl_ptr[P];
            for (int64_t q = 0; q < m; q++) dist[s->glbind[s->gl_ptr[P] + q]] = (int32_t)(m - 1 - q);
            for (int32_t J = chead[P]; J != -1; J = cnext[J]) {
                int64_t nJ = sup_ptr[J + 1] - sup_ptr[J];
                int64_t w = s->ri_ptr[J];
                for (int64_t p = s->gl_ptr[J] + nJ; p < s->gl_ptr[J + 1]; p++) {
                    int32_t d = dist[s->glbind[p]];
                    if (d < 0) return SC_ERR_INTERNAL;
                    s->relind[w++] = d;
                }
            }
            for (int64_t q = 0; q < m; q++) dist[s->glbind[s->gl_ptr[P] + q]] = -1;
        }
    }

    // ---- blocks: maximal runs of consecutive rows of S_J, cut at supernode boundaries
    s->blk_ptr.assign(ns + 1, 0);
    for (int64_t J = 0; J < ns; J++) {
        int64_t nJ = sup_ptr[J + 1] - sup_ptr[J];
        int32_t prev = -2;
        for (int64_t p = s->gl_ptr[J] + nJ; p < s->gl_ptr[J + 1]; p++) {
            int32_t i = s->glbind[p];
            if (i == prev + 1 && sup_of[i] == sup_of[prev]) {
                s->blk_size.back()++;
            } else {
                s->blk_first.push_back(i);
                s->blk_size.push_back(1);
                s->blk_owner.push_back(sup_of[i]);
            }
            prev = i;
        }
        s->blk_ptr[J + 1] = (int64_t)s->blk_first.size();
    }

    // ---- relindB(J, P): extracted from relind(J, p(J)) (Alg. 5), then
    //      composed with relind(C, P) for each further ancestor
    s->rb_pair_ptr.assign(ns + 1, 0);
    s->rb_val_ptr.assign(1, 0);
    {
        std::vector<int32_t> cur, nxt;
        std::vector<int64_t> bpos;  // position in S_J of each block's first row
        for (int64_t J = 0; J < ns; J++) {
            int64_t b0 = s->blk_ptr[J], b1 = s->blk_ptr[J + 1];
            if (b1 > b0) {
                int64_t nJ = sup_ptr[J + 1] - sup_ptr[J];
                // extract: relind of each block's top row
                cur.clear();
                int64_t q = 0;
                for (int64_t b = b0; b < b1; b++) {
                    cur.push_back(s->relind[s->ri_ptr[J] + q]);
                    q += s->blk_size[b];
                }
                (void)nJ;
                int32_t top = s->blk_owner[b1 - 1];
                int64_t first_blk = b0;  // blocks at or above the current P
                int32_t C = (int32_t)J;
                for (int32_t P = spar[J]; P >= 0; P = spar[P]) {
                    if (P != spar[J]) {
                        // compose for the blocks lying below C: relindB(J,P) = relindB(J,C) o relind(C,P)
                        int32_t lC = sup_ptr[C + 1] - 1;
                        int64_t k0 = 0;
                        while (first_blk + k0 < b1 && s->blk_first[first_blk + k0] <= lC) k0++;
                        int64_t lenCP = s->ri_ptr[C + 1] - s->ri_ptr[C];
                        nxt.resize(cur.size() - k0);
                        int r = compose_relind(cur.data() + k0, (int64_t)nxt.size(), s->relind.data() + s->ri_ptr[C], lenCP,
                                               nxt.data());
                        if (r) return SC_ERR_INTERNAL;
                        cur.swap(nxt);
                        first_blk += k0;
                    }
                    s->rb_pair_P.push_back(P);
                    s->rb_val.insert(s->rb_val.end(), cur.begin(), cur.end());
                    s->rb_val_ptr.push_back((int64_t)s->rb_val.size());
                    if (P == top) break;
                    C = P;
                }
            }
            s->rb_pair_ptr[J + 1] = (int64_t)s->rb_pair_P.size();
        }
    }

    // ---- levels: height in the supernodal elimination tree
    s->level.assign(ns, 0);
    for (int64_t J = 0; J < ns; J++)
        if (spar[J] >= 0 && s->level[spar[J]] < s->level[J] + 1) s->level[spar[J]] = s->level[J] + 1;

    // ---- factor storage: J holds m_J rows of ld_J entries (row-major), at lnz_off[J].
    //      Wide panels get ld a multiple of 4 and 128-byte aligned bases (tensor-memory copies).
    s->lnz_off.resize(ns);
    s->lnz_ld.resize(ns);
    int64_t off = 0;
    for (int64_t J = 0; J < ns; J++) {
        int32_t w = sup_ptr[J + 1] - sup_ptr[J];
        int64_t m = s->gl_ptr[J + 1] - s->gl_ptr[J];
        int32_t ld = w >= 16 ? (w + 3) / 4 * 4 : w;
        int64_t align = w >= 16 ? 32 : 4;
        off = (off + align - 1) / align * align;
        s->lnz_off[J] = off;
        s->lnz_ld[J] = ld;
        off += m * ld;
    }
    s->lnz_size = (off + 31) / 32 * 32;

    // ---- map of A's entries into Lnz
    s->valmap.resize(nnzA);
    std::atomic<bool> missing{false};
    parallel_blocks(n, 4096, threads, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; c++)
            for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
                int32_t a = s->iperm[rowind[p]], b = s->iperm[c];
                int32_t col = std::min(a, b), row = std::max(a, b);
                int32_t J = sup_of[col];
                int32_t f = sup_ptr[J];
                int64_t m = s->gl_ptr[J + 1] - s->gl_ptr[J];
                const int32_t *g = s->glbind.data() + s->gl_ptr[J];
                int64_t pos = std::lower_bound(g, g + m, row) - g;
                if (pos >= m || g[pos] != row) {
                    missing.store(true, std::memory_order_relaxed);
                    return;
                }
                s->valmap[p] = s->lnz_off[J] + pos * s->lnz_ld[J] + (col - f);
            }
    });
    if (missing.load()) return SC_ERR_INTERNAL;

    // ---- full symmetric CSR of A (caller's ordering) for the FP64 residual
    s->csr_ptr.assign(n + 1, 0);
    for (int64_t c = 0; c < n; c++)
        for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
            s->csr_ptr[rowind[p] + 1]++;
            if (rowind[p] != c) s->csr_ptr[c + 1]++;
        }
    for (int64_t i = 0; i < n; i++) s->csr_ptr[i + 1] += s->csr_ptr[i];
    s->csr_col.resize(s->csr_ptr[n]);
    s->csr_map.resize(s->csr_ptr[n]);
    {
        std::vector<int64_t> fill(s->csr_ptr.begin(), s->csr_ptr.end() - 1);
        for (int64_t c = 0; c < n; c++)
            for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
                int32_t i = rowind[p];
                s->csr_col[fill[i]] = (int32_t)c;
                s->csr_map[fill[i]++] = p;
                if (i != c) {
                    s->csr_col[fill[c]] = i;
                    s->csr_map[fill[c]++] = p;
                }
            }
    }

    rc = build_schedule(s.get());
    if (rc) return rc;
    *out = s.release();
    return SC_OK;
}

}  // namespace sc
