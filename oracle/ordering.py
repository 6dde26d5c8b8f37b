"""General-graph nested dissection orderings of the oracle: TEST INFRASTRUCTURE.

Plain Python on sets and dicts, written from the definitions below (the paper
orders with METIS, Sec. 3.1, which is not available; these are the stand-ins
whose exact output the library must reproduce). Small graphs only.

nd_graph(A, leaf): ND(S), S a vertex set of the graph of A:
  * |S| <= leaf: the vertices of S in increasing order;
  * G[S] disconnected: ND of each connected component, the components taken
    in order of their smallest vertex;
  * otherwise the level split: r = min S and L_0, L_1, ... the breadth-first
    levels of G[S] from r; at most 8 times, let c be the vertex of the last
    level with the fewest neighbours in S (ties: smaller index); if the levels
    from c are more than those from r, take c as r, else stop. The separator
    is the first level L_k with 2 |L_0 u ... u L_k| >= |S|, and
    ND(S) = ND(L_0..L_{k-1}), ND(L_{k+1}..), then L_k in increasing order.

nd_graph_ml(A, leaf): as nd_graph, but a connected S of at least 64 vertices
is also bisected by the multilevel scheme below (unit weights on G[S],
vertices renumbered 0.. in increasing order); its separator is the minimum
vertex cover of the cut edges (see _min_cover) when that is smaller than the
smaller boundary layer (the vertices of one part with a neighbour in the
other; ties: part 0's), else that layer. That split, ND(part 0 minus sep),
ND(part 1 minus sep), sep, is used when both parts keep a vertex and its
separator is smaller than the level separator.

Multilevel bisection of a weighted graph (vertex weights vw, edge weights):
  * coarsening, while more than 40 vertices remain and fewer than 30 levels
    were made: visit vertices in increasing id; an unmatched vertex is matched
    with its unmatched neighbour of largest edge weight (ties: smaller vertex
    weight, then smaller id), or alone; coarse vertices are numbered in visiting
    order, weights summed, parallel edges merged by summing; stop (discarding
    the step) when it keeps more than 95 % of the vertices;
  * initial partition of the coarsest graph, for each seed among its first 32
    vertices: breadth-first growth from the seed (neighbours in increasing id)
    putting vertices into part 0 until its weight reaches ceil(W / 2), then FM
    refinement; keep the smallest cut (ties: smaller |W - 2 w0|, then the
    earlier seed);
  * project back level by level, refining with FM at each;
  * FM refinement, part weights bounded by floor((11 W + 19) / 20): up to 8
    passes; a pass computes every gain (edge weight to the other part minus to
    its own), then repeatedly moves the unlocked vertex with a neighbour in the
    other part, of largest gain (ties: smaller id), whose move respects the
    bound, and locks it, until 25 moves in a row bring no new best cumulative
    gain or no vertex qualifies; it then undoes the moves after the best
    prefix; the passes stop after one whose best cumulative gain is not
    positive.
"""
from __future__ import annotations

import sys

import numpy as np

COARSE_MIN, MAX_LEVELS, SEEDS, PASSES, STALL = 40, 30, 32, 8, 25
ML_MIN_SET = 64


def _neighbours(A):
    nbr = [set() for _ in range(A.n)]
    for j in range(A.n):
        for p in range(int(A.colptr[j]), int(A.colptr[j + 1])):
            i = int(A.rowind[p])
            if i != j:
                nbr[i].add(j)
                nbr[j].add(i)
    return nbr


# ----------------------------------------------------------------- multilevel

def _coarsen(vw, adj):
    n = len(vw)
    match = [None] * n
    cmap = [None] * n
    nc = 0
    for v in range(n):
        if match[v] is not None:
            continue
        best = None
        for u in sorted(adj[v]):
            if match[u] is not None or u == v:
                continue
            if best is None or adj[v][u] > adj[v][best] or (adj[v][u] == adj[v][best] and vw[u] < vw[best]):
                best = u
        if best is None:
            match[v] = v
            cmap[v] = nc
        else:
            match[v], match[best] = best, v
            cmap[v] = cmap[best] = nc
        nc += 1
    cvw = [0] * nc
    cadj = [dict() for _ in range(nc)]
    for v in range(n):
        cvw[cmap[v]] += vw[v]
        for u, w in adj[v].items():
            a, b = cmap[v], cmap[u]
            if a != b:
                cadj[a][b] = cadj[a].get(b, 0) + w
    return cmap, cvw, cadj


def _cut(adj, part):
    return sum(w for v in range(len(adj)) for u, w in adj[v].items() if part[u] != part[v]) // 2


def _fm(vw, adj, part, maxw):
    n = len(vw)
    W = [0, 0]
    for v in range(n):
        W[part[v]] += vw[v]
    for _ in range(PASSES):
        gain = [sum(w if part[u] != part[v] else -w for u, w in adj[v].items()) for v in range(n)]
        ext = [sum(w for u, w in adj[v].items() if part[u] != part[v]) for v in range(n)]
        locked = [False] * n
        moves, cum, best, best_len, stall = [], 0, 0, 0, 0
        while stall < STALL:
            pick = None
            for v in range(n):
                if locked[v] or ext[v] == 0 or W[1 - part[v]] + vw[v] > maxw:
                    continue
                if pick is None or gain[v] > gain[pick]:
                    pick = v
            if pick is None:
                break
            v = pick
            src, dst = part[v], 1 - part[v]
            cum += gain[v]
            part[v] = dst
            W[src] -= vw[v]
            W[dst] += vw[v]
            locked[v] = True
            moves.append(v)
            gain[v] = -gain[v]
            for u, w in adj[v].items():
                if part[u] == dst:
                    gain[u] -= 2 * w
                    ext[u] -= w
                else:
                    gain[u] += 2 * w
                    ext[u] += w
            if cum > best:
                best, best_len, stall = cum, len(moves), 0
            else:
                stall += 1
        for v in reversed(moves[best_len:]):
            W[part[v]] -= vw[v]
            part[v] = 1 - part[v]
            W[part[v]] += vw[v]
        if best <= 0:
            break
    return part


def _grow(vw, adj, seed, half):
    part = [1] * len(vw)
    seen = {seed}
    queue = [seed]
    got = 0
    h = 0
    while h < len(queue) and got < half:
        v = queue[h]
        h += 1
        part[v] = 0
        got += vw[v]
        for u in sorted(adj[v]):
            if u not in seen:
                seen.add(u)
                queue.append(u)
    return part


def _bisect(vw, adj):
    stack = []
    cvw, cadj = vw, adj
    while len(cvw) > COARSE_MIN and len(stack) < MAX_LEVELS:
        cmap, nvw, nadj = _coarsen(cvw, cadj)
        if len(nvw) > 0.95 * len(cvw):
            break
        stack.append((cmap, cvw, cadj))
        cvw, cadj = nvw, nadj
    total = sum(vw)
    maxw = (11 * total + 19) // 20
    best = None
    for seed in range(min(len(cvw), SEEDS)):
        p = _fm(cvw, cadj, _grow(cvw, cadj, seed, (total + 1) // 2), maxw)
        w0 = sum(cvw[v] for v in range(len(cvw)) if p[v] == 0)
        key = (_cut(cadj, p), abs(total - 2 * w0), seed)
        if best is None or key < best[0]:
            best = (key, p)
    part = best[1]
    for cmap, fvw, fadj in reversed(stack):
        part = _fm(fvw, fadj, [part[cmap[v]] for v in range(len(fvw))], maxw)
    return part


def _min_cover(adj, part, b0):
    """Minimum vertex cover of the cut edges (Konig's theorem): a maximum
    matching between the part-0 boundary b0 and part 1 by augmenting paths
    (each v of b0 in increasing order starts a depth-first search over its
    part-1 neighbours in increasing order, every part-1 vertex entered at most
    once per search); Z = the vertices reachable from the unmatched vertices
    of b0 by alternating paths; the cover is (b0 - Z) with (part 1 in Z)."""
    mate = {}

    def augment(v, seen):
        for u in sorted(adj[v]):
            if part[u] != 1 or u in seen:
                continue
            seen.add(u)
            if u not in mate or augment(mate[u], seen):
                mate[u], mate[v] = v, u
                return True
        return False

    for v in b0:
        augment(v, set())
    z = {v for v in b0 if v not in mate}
    todo = list(z)
    while todo:
        v = todo.pop()
        for u in adj[v]:
            if part[u] == 1 and u not in z:
                z.add(u)
                if u in mate and mate[u] not in z:
                    z.add(mate[u])
                    todo.append(mate[u])
    return {v for v in b0 if v not in z} | {u for u in z if part[u] == 1}


# ----------------------------------------------------------------- recursion

def _nested_dissection(A, leaf, multilevel, ml_min=ML_MIN_SET):
    nbr = _neighbours(A)

    def levels(r, S):
        seen = {r}
        out = [{r}]
        while True:
            nxt = set()
            for v in out[-1]:
                nxt |= (nbr[v] & S) - seen
            if not nxt:
                return out
            seen |= nxt
            out.append(nxt)

    def components(S):
        left = set(S)
        comps = []
        while left:
            comp = set().union(*levels(min(left), S))
            comps.append(comp)
            left -= comp
        return comps

    def level_split(S):
        lv = levels(min(S), S)
        for _ in range(8):
            c = min(lv[-1], key=lambda v: (len(nbr[v] & S), v))
            lc = levels(c, S)
            if len(lc) <= len(lv):
                break
            lv = lc
        total = 0
        for k, level in enumerate(lv):
            total += len(level)
            if 2 * total >= len(S):
                break
        below = set().union(*lv[:k]) if k > 0 else set()
        above = set().union(*lv[k + 1:]) if k + 1 < len(lv) else set()
        return below, above, lv[k]

    def multilevel_split(S):
        verts = sorted(S)
        loc = {g: i for i, g in enumerate(verts)}
        adj = [{loc[u]: 1 for u in nbr[g] if u in loc} for g in verts]
        part = _bisect([1] * len(verts), adj)
        bnd = [[i for i in range(len(verts)) if part[i] == side and any(part[u] != side for u in adj[i])]
               for side in (0, 1)]
        sep = set(bnd[0] if len(bnd[0]) <= len(bnd[1]) else bnd[1])
        cover = _min_cover(adj, part, bnd[0])
        if len(cover) < len(sep):
            sep = cover
        p0 = {verts[i] for i in range(len(verts)) if part[i] == 0 and i not in sep}
        p1 = {verts[i] for i in range(len(verts)) if part[i] == 1 and i not in sep}
        return p0, p1, {verts[i] for i in sep}

    def nd(S):
        if len(S) <= leaf:
            return sorted(S)
        comps = components(S)
        if len(comps) > 1:
            return [v for c in comps for v in nd(c)]
        first, second, sep = level_split(S)
        if multilevel and len(S) >= ml_min:
            p0, p1, msep = multilevel_split(S)
            if msep and p0 and p1 and len(msep) < len(sep):
                first, second, sep = p0, p1, msep
        return nd(first) + nd(second) + sorted(sep)

    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        perm = nd(set(range(A.n)))
    finally:
        sys.setrecursionlimit(old)
    return np.asarray(perm, dtype=np.int32)


def nd_graph(A, leaf: int = 8) -> np.ndarray:
    """Level-structure nested dissection of the graph of A, perm[new] = old."""
    return _nested_dissection(A, leaf, False)


def nd_graph_ml(A, leaf: int = 8) -> np.ndarray:
    """Nested dissection with the smaller of the level and multilevel separators."""
    return _nested_dissection(A, leaf, True)
