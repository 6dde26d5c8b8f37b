"""Pins of the oracle against facts fixed by the paper and by mathematics (CPU only).

- the paper's worked example (Figs. 1-3, Sec. 2.1.2, Sec. 2.2.2), from tests/golden/;
- closed forms: tridiagonal, dense, arrowhead, k x k grid in natural order;
- column structure against brute-force structural elimination (n <= 200);
- numeric factor against dense Cholesky (a textbook library routine) on small
  matrices, entries outside the pattern exactly zero, ||A - L L^T|| / ||A||;
- solve: backward error, and the closed form x = b / d for a diagonal matrix;
- nested dissection: hand-derived order on a 3 x 3 grid;
- PR invariants: storage and flops unchanged, permutation only inside supernodes.
"""
import numpy as np
import pytest

import oracle
from paper_2409_13090_gb300 import inputs


def _example(golden):
    ents = [(i - 1, j - 1) for i, j in golden["A_strict_lower_pattern"]["entries"]]
    return inputs.from_lower_pattern(golden["n"], ents, seed=3)


def _seg(arr, ptr, k):
    return arr[ptr[k]:ptr[k + 1]].tolist()


# --------------------------------------------------------------------------- worked example

def test_worked_example_symbolic(golden):
    A = _example(golden)
    s = oracle.Oracle(A, None, pr=False).symbolic()
    assert s.perm.tolist() == list(range(9))  # postorder of Fig. 3's tree is the identity
    sets = [list(range(s.sup_ptr[J] + 1, s.sup_ptr[J + 1] + 1)) for J in range(s.nsuper)]
    assert sets == golden["supernodes"]["sets"]
    assert [(p + 1) if p >= 0 else 0 for p in s.cparent] == golden["etree_parent"]["parent"]
    assert [g + 1 for g in _seg(s.glbind, s.gl_ptr, 0)] == golden["glbind"]["J1"]
    assert [g + 1 for g in _seg(s.glbind, s.gl_ptr, 1)] == golden["glbind"]["J2"]
    assert [(p + 1) if p >= 0 else 0 for p in s.sup_parent] == golden["supernodal_parent"]["parent"]
    assert _seg(s.relind, s.ri_ptr, 0) == golden["relind"]["J1_J3"]
    assert _seg(s.relind, s.ri_ptr, 1) == golden["relind"]["J2_J3"]
    for J, key in ((0, "J1"), (1, "J2")):
        blocks = [list(range(f + 1, f + 1 + z)) for f, z in zip(_seg(s.blk_first, s.blk_ptr, J), _seg(s.blk_size, s.blk_ptr, J))]
        assert blocks == golden["blocks"][key]
    for J, key in ((0, "J1_J3"), (1, "J2_J3")):
        q0, q1 = s.rb_pair_ptr[J], s.rb_pair_ptr[J + 1]
        assert q1 - q0 == 1 and s.rb_pair_P[q0] == 2
        assert s.rb_val[s.rb_val_ptr[q0]:s.rb_val_ptr[q0 + 1]].tolist() == golden["relindB"][key]
    # the updates J1 -> J3 of Sec. 1: blocks {5,6} and {9}; B' = {9} lies below B = {5,6}
    assert golden["rlb_updates_J1_to_J3"]["syrk"] == [[5, 6], [9]]
    # pattern of L = A's pattern plus the fill of Fig. 1
    cp, rows = oracle.Oracle(A, None, pr=False).columns()
    pat = {(int(r) + 1, j + 1) for j in range(9) for r in rows[cp[j]:cp[j + 1]] if r != j}
    want = {tuple(e) for e in golden["A_strict_lower_pattern"]["entries"]} | {tuple(e) for e in golden["fill"]["entries"]}
    assert pat == want


def test_levels_are_heights_in_the_supernodal_tree(golden):
    """level(J) = height of J in the supernodal elimination tree (leaves 0, a
    parent one above its highest child), by hand: the worked example (J1, J2
    are leaves below J3), a chain, an arrowhead (leaves under one root), and a
    tree whose branches differ in length, where height and depth disagree."""
    s = oracle.Oracle(_example(golden), None, pr=False).symbolic()
    assert s.level.tolist() == [0, 0, 1]
    # tridiagonal, natural order: supernodes {0}, ..., {n-3}, {n-2, n-1}, a chain
    n = 10
    s = oracle.Oracle(inputs.from_lower_pattern(n, [(j + 1, j) for j in range(n - 1)], seed=1), None,
                      pr=False).symbolic()
    assert s.nsuper == n - 1 and s.level.tolist() == list(range(n - 1))
    # arrowhead (dense last row): every other column is a leaf under the last one
    s = oracle.Oracle(inputs.from_lower_pattern(n, [(n - 1, j) for j in range(n - 1)], seed=1), None,
                      pr=False).symbolic()
    assert s.level.tolist() == [0] * (n - 1) + [1]
    # columns 0 - 1 - 2 - 4 and 3 - 4, then 4 - 5: etree 0->1->2->4, 3->4, 4->5;
    # supernodes {0} {1} {2} {3} {4, 5}; heights 0 1 2 0 3 (depths would be 3 2 1 1 0)
    s = oracle.Oracle(inputs.from_lower_pattern(6, [(1, 0), (2, 1), (4, 2), (4, 3), (5, 4)], seed=1), None,
                      pr=False).symbolic()
    assert s.sup_ptr.tolist() == [0, 1, 2, 3, 4, 6]
    assert [int(p) for p in s.sup_parent] == [1, 2, 4, 4, -1]
    assert s.level.tolist() == [0, 1, 2, 0, 3]


def test_worked_example_pr(golden):
    A = _example(golden)
    s = oracle.Oracle(A, None, pr=True).symbolic()
    old_to_new = {int(k): v for k, v in golden["pr_relabel"]["old_to_new"].items()}
    for new0, old0 in enumerate(s.perm.tolist()):
        if old0 >= 4:
            assert old_to_new[old0 + 1] == new0 + 1
        else:
            assert old0 == new0
    assert s.blk_ptr[1] - s.blk_ptr[0] == golden["pr_blocks"]["J1"]
    assert s.blk_ptr[2] - s.blk_ptr[1] == golden["pr_blocks"]["J2"]
    # supernodes and storage carried over unchanged
    assert s.sup_ptr.tolist() == [0, 2, 4, 9]
    assert s.nnzL == oracle.Oracle(A, None, pr=False).symbolic().nnzL


def test_worked_example_numeric(golden):
    A = _example(golden)
    for pr in (False, True):
        o = oracle.Oracle(A, None, pr=pr)
        assert o.factor() == 0
        s = o.symbolic()
        M = inputs.dense_from_lower(A)[np.ix_(s.perm, s.perm)]
        Ld = np.linalg.cholesky(M)
        Ls = _dense_L(o)
        assert np.abs(Ls - Ld).max() <= 1e-13 * np.abs(Ld).max()


# --------------------------------------------------------------------------- helpers

def _dense_L(o):
    cp, rows = o.columns()
    lv = o.L_columns()
    n = len(cp) - 1
    L = np.zeros((n, n))
    for j in range(n):
        L[rows[cp[j]:cp[j + 1]], j] = lv[cp[j]:cp[j + 1]]
    return L


def _pattern_mask(o):
    cp, rows = o.columns()
    n = len(cp) - 1
    m = np.zeros((n, n), bool)
    for j in range(n):
        m[rows[cp[j]:cp[j + 1]], j] = True
    return m


def _brute_force_pattern(M):
    """Structural elimination on a dense boolean matrix (fill of Gaussian elimination)."""
    n = M.shape[0]
    S = (M != 0)
    S = np.tril(S | S.T)
    for j in range(n):
        rows = np.nonzero(S[j + 1:, j])[0] + j + 1
        for a in rows:
            S[a, rows[rows <= a]] = True
    return S


# --------------------------------------------------------------------------- closed forms

def test_tridiagonal_closed_form():
    n = 50
    A = inputs.from_lower_pattern(n, [(i + 1, i) for i in range(n - 1)])
    o = oracle.Oracle(A, None, pr=False)
    s = o.symbolic()
    assert s.nnzL == 2 * n - 1
    assert s.cparent.tolist() == list(range(1, n)) + [-1]
    sizes = np.diff(s.sup_ptr).tolist()
    assert sizes == [1] * (n - 2) + [2]


def test_dense_closed_form():
    n = 30
    A = inputs.from_lower_pattern(n, [(i, j) for j in range(n) for i in range(j + 1, n)])
    s = oracle.Oracle(A, None, pr=True).symbolic()
    assert s.nsuper == 1 and s.nnzL == n * (n + 1) // 2
    assert s.flops == sum(c * c for c in range(1, n + 1))


def test_arrowhead_closed_form():
    n = 40
    A = inputs.from_lower_pattern(n, [(n - 1, j) for j in range(n - 1)])
    s = oracle.Oracle(A, None, pr=False).symbolic()
    assert s.nnzL == 2 * n - 1


@pytest.mark.parametrize("k", [3, 5, 8, 12])
def test_grid_natural_band_closed_form(k):
    # In natural order the factor fills the row envelope: row i of a point with
    # y >= 1 spans k+1 columns, the first grid row spans 2 (1 for the corner), so
    # nnz(L) = (n - k)(k + 1) + 2(k - 1) + 1 = n(k + 1) - k^2 + k - 1.
    A = inputs.laplacian_2d(k, k)
    n = k * k
    s = oracle.Oracle(A, None, pr=False).symbolic()
    assert s.nnzL == n * (k + 1) - k * k + k - 1


def test_nd_hand_order():
    # 3x3 grid, leaf 1: split x at 1 -> left column {x=0}, right {x=2}, separator {x=1};
    # each column box splits y at 1 -> (y=0), (y=2), separator (y=1).
    assert oracle.nd_grid(3, 3, 1, leaf=1).tolist() == [0, 6, 3, 2, 8, 5, 1, 4, 7]


def test_nd_is_permutation_and_top_separator():
    perm = oracle.nd_grid(64, 64, 1, leaf=8)
    assert sorted(perm.tolist()) == list(range(64 * 64))
    top = perm[-64:]
    assert set((top % 64).tolist()) == {32}  # the last 64 points are the plane x = 32
    p3 = oracle.nd_grid(6, 5, 4, leaf=8)
    assert sorted(p3.tolist()) == list(range(120))


# --------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("pr", [False, True])
def test_structure_vs_brute_force(seed, pr):
    n = 60 + 35 * seed
    A = inputs.random_spd(n, 0.04, seed)
    rng = np.random.default_rng(seed)
    perm0 = rng.permutation(n).astype(np.int32)
    o = oracle.Oracle(A, perm0, pr=pr)
    s = o.symbolic()
    M = inputs.dense_from_lower(A)[np.ix_(s.perm, s.perm)]
    bf = _brute_force_pattern(M)
    mask = _pattern_mask(o)
    if not pr:
        assert np.array_equal(mask, bf)
    else:
        assert not np.any(bf & ~mask)  # the true pattern lies inside the supernodal one
        assert mask.sum() == oracle.Oracle(A, perm0, pr=False).symbolic().nnzL


@pytest.mark.parametrize("case", ["rand", "grid2d", "grid3d", "st27"])
@pytest.mark.parametrize("pr", [False, True])
def test_numeric_vs_dense_cholesky(case, pr):
    if case == "rand":
        A = inputs.random_spd(150, 0.03, 11)
        perm0 = None
    elif case == "grid2d":
        A = inputs.laplacian_2d(12, 13, shift=0.01)
        perm0 = oracle.nd_grid(12, 13, 1, 4)
    elif case == "grid3d":
        A = inputs.diffusion_3d_7pt(5, 6, 5, seed=4, shift=1e-2)
        perm0 = oracle.nd_grid(5, 6, 5, 8)
    else:
        A = inputs.stencil_3d_27pt(5, 5, 5, seed=5)
        perm0 = oracle.nd_grid(5, 5, 5, 8)
    o = oracle.Oracle(A, perm0, pr=pr)
    assert o.factor() == 0
    s = o.symbolic()
    M = inputs.dense_from_lower(A)[np.ix_(s.perm, s.perm)]
    Ld = np.linalg.cholesky(M)
    Ls = _dense_L(o)
    mask = _pattern_mask(o)
    assert np.all(Ld[~mask] == 0.0) or np.abs(Ld[~mask]).max() <= 1e-15 * np.abs(Ld).max()
    assert np.linalg.norm(Ls - Ld) <= 1e-12 * np.linalg.norm(Ld)
    assert np.linalg.norm(M - Ls @ Ls.T) <= 1e-14 * np.linalg.norm(M)


def test_solve_backward_error_and_diagonal_closed_form():
    A = inputs.diffusion_3d_7pt(6, 6, 6, seed=9, shift=1e-3)
    o = oracle.Oracle(A, oracle.nd_grid(6, 6, 6, 8), pr=True)
    assert o.factor() == 0
    B = inputs.rhs(A.n, 3, 1)
    X = o.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14
    # diagonal matrix: x = b / d exactly
    n = 17
    D = inputs.from_lower_pattern(n, [])
    D.values[:] = np.arange(1, n + 1, dtype=float) ** 2
    od = oracle.Oracle(D, None, pr=True)
    assert od.factor() == 0
    b = inputs.rhs(n, 2, 2)
    x = od.solve(b)
    # x = (b / d^(1/2)) / d^(1/2): two correctly rounded divisions, within 2 ulps of b / d
    want = b / D.values[:, None]
    assert np.all(np.abs(x - want) <= 2 * np.finfo(float).eps * np.abs(want))


def test_not_positive_definite_reports_column():
    A = inputs.laplacian_2d(6, 6)
    o = oracle.Oracle(A, None, pr=False)
    s = o.symbolic()
    # make the diagonal of original column 20 very negative: the first non-positive
    # pivot is met at that column's position in the final ordering, or before it
    v = A.values.copy()
    diag_pos = A.colptr[20]
    v[diag_pos] = -100.0
    info = o.factor(v)
    assert info >= 1
    new_pos = int(np.nonzero(s.perm == info - 1)[0][0])
    assert new_pos <= int(np.nonzero(s.perm == 20)[0][0])


def test_pr_invariants():
    A = inputs.diffusion_3d_7pt(10, 9, 8, seed=1)
    perm0 = oracle.nd_grid(10, 9, 8, 8)
    s0 = oracle.Oracle(A, perm0, pr=False).symbolic()
    s1 = oracle.Oracle(A, perm0, pr=True).symbolic()
    assert s0.nnzL == s1.nnzL and s0.flops == s1.flops
    assert np.array_equal(s0.sup_ptr, s1.sup_ptr) and np.array_equal(s0.gl_ptr, s1.gl_ptr)
    for J in range(s0.nsuper):
        a, b = s0.sup_ptr[J], s0.sup_ptr[J + 1]
        assert sorted(s0.perm[a:b].tolist()) == sorted(s1.perm[a:b].tolist())
    assert len(s1.blk_first) <= len(s0.blk_first)


def test_relindB_is_distance_of_block_top_from_bottom():
    """relindB(J, P) entry = m_P - 1 - position of the block's first row in glbind(P)."""
    A = inputs.stencil_3d_27pt(6, 6, 6, seed=2)
    s = oracle.Oracle(A, oracle.nd_grid(6, 6, 6, 8), pr=True).symbolic()
    for J in range(s.nsuper):
        firsts = _seg(s.blk_first, s.blk_ptr, J)
        for q in range(s.rb_pair_ptr[J], s.rb_pair_ptr[J + 1]):
            P = s.rb_pair_P[q]
            g = _seg(s.glbind, s.gl_ptr, P)
            sel = [f for f in firsts if f >= s.sup_ptr[P]]
            vals = s.rb_val[s.rb_val_ptr[q]:s.rb_val_ptr[q + 1]].tolist()
            assert vals == [len(g) - 1 - g.index(f) for f in sel]


# --------------------------------------------------------------------------- supernode merging (Sec. 3.1)

def test_merge_worked_example_by_hand(golden):
    """At a 12.5 % budget: S0 = 9 + 9 + 15 = 33, budget 4.125. J1 is not adjacent to J3;
    J2 -> J3 adds 7*7 - 21 - 9 - 15 = 4 <= 4.125 and merges; J1 -> (J2 u J3) would then
    add 9*9 - 36 - 9 - 28 = 8, past the budget."""
    ents = [(i - 1, j - 1) for i, j in golden["A_strict_lower_pattern"]["entries"]]
    A = inputs.from_lower_pattern(9, ents)
    s = oracle.Oracle(A, None, pr=False, merge=0.125).symbolic()
    assert s.sup_ptr.tolist() == [0, 2, 9]
    assert s.nnzL == 33 + 4
    assert s.flops == oracle.Oracle(A, None, pr=False).symbolic().flops  # metric stays fundamental
    s = oracle.Oracle(A, None, pr=False, merge=4.0 / 33.0 - 1e-9).symbolic()  # budget just below 4
    assert s.sup_ptr.tolist() == [0, 2, 4, 9]


def test_merge_chain_by_hand():
    """Tridiagonal n = 8: fundamental supernodes {0}..{5},{6,7}, storage 15, budget 1.875.
    Every adjacent pair adds exactly 1; the tie goes to the smallest first column, so
    {0} merges into {1}; the next merge would reach 2 > 1.875."""
    n = 8
    A = inputs.from_lower_pattern(n, [(i + 1, i) for i in range(n - 1)])
    s = oracle.Oracle(A, None, pr=False, merge=0.125).symbolic()
    assert s.sup_ptr.tolist() == [0, 2, 3, 4, 5, 6, 8]
    s = oracle.Oracle(A, None, pr=False, merge=10.0).symbolic()
    assert s.nsuper == 1 and s.nnzL == n * (n + 1) // 2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_merge_invariants_and_numeric(seed):
    A = inputs.diffusion_3d_7pt(7, 6, 5, seed=seed, shift=1e-2)
    perm0 = oracle.nd_grid(7, 6, 5, 8)
    f = oracle.Oracle(A, perm0, pr=True).symbolic()
    o = oracle.Oracle(A, perm0, pr=True, merge=0.125)
    m = o.symbolic()
    assert m.nsuper < f.nsuper and m.flops == f.flops
    assert f.nnzL <= m.nnzL <= f.nnzL * 1.125
    # merged partition coarsens the fundamental one (same postorder, up to PR inside supernodes)
    assert set(m.sup_ptr.tolist()) <= set(f.sup_ptr.tolist())
    assert o.factor() == 0
    M = inputs.dense_from_lower(A)[np.ix_(m.perm, m.perm)]
    Ld = np.linalg.cholesky(M)
    Ls = _dense_L(o)
    assert np.linalg.norm(Ls - Ld) <= 1e-12 * np.linalg.norm(Ld)
    assert not np.any(_brute_force_pattern(M) & ~_pattern_mask(o))


def test_backward_error_hand_example():
    """A = [[4,1],[1,3]], b = [1,2], x = [0.1,0.6]: r = [0, 0.1], ||A||_inf = 5,
    eta = 0.1 / (5 * 0.6 + 2) = 0.02."""
    A = inputs.SparseSym(2, np.array([0, 2, 3], np.int64), np.array([0, 1, 1], np.int32), np.array([4.0, 1.0, 3.0]))
    eta = oracle.backward_error(A, np.array([[1.0], [2.0]]), np.array([[0.1], [0.6]]))
    assert abs(eta[0] - 0.02) <= 1e-15


# --------------------------------------------------------------------------- general-graph ND

def test_nd_graph_hand_orders():
    # path 0-1-...-6, leaf 1: levels from 0 are singletons (from 6 no more levels),
    # the separator is the first level with 2*4 >= 7, i.e. vertex 3; each half of
    # three splits at its middle vertex.
    path = inputs.from_lower_pattern(7, [(i + 1, i) for i in range(6)])
    assert oracle.nd_graph(path, leaf=1).tolist() == [0, 2, 1, 4, 6, 5, 3]
    # star with centre 0, leaf 1: levels from 0 are {0},{1..6}; from leaf 1 they are
    # {1},{0},{2..6} (deeper, so the root moves to 1); from 2 no deeper. Separator:
    # 2*1 < 7, 2*2 < 7, 2*7 >= 7 -> {2..6}; the rest {0,1} splits at 0.
    star = inputs.from_lower_pattern(7, [(i, 0) for i in range(1, 7)])
    assert oracle.nd_graph(star, leaf=1).tolist() == [1, 0, 2, 3, 4, 5, 6]
    # two disjoint paths 0-2-4 and 1-3-5, leaf 1: components taken by smallest vertex
    two = inputs.from_lower_pattern(6, [(2, 0), (4, 2), (3, 1), (5, 3)])
    assert oracle.nd_graph(two, leaf=1).tolist() == [0, 4, 2, 1, 5, 3]
    # a leaf at least n keeps the natural order
    assert oracle.nd_graph(star, leaf=7).tolist() == list(range(7))


def test_nd_graph_is_a_dissection():
    # each separator splits: eliminating in ND order never creates fill between
    # vertices of the two sides, so on a 2D grid the fill is far below the
    # natural (banded) order and of the order of the geometric ND.
    A = inputs.laplacian_2d(24, 24)
    perm = oracle.nd_graph(A, leaf=8)
    assert sorted(perm.tolist()) == list(range(A.n))
    nnz_nd = oracle.Oracle(A, perm, pr=False).symbolic().nnzL
    nnz_nat = oracle.Oracle(A, None, pr=False).symbolic().nnzL
    nnz_geo = oracle.Oracle(A, oracle.nd_grid(24, 24, 1, 8), pr=False).symbolic().nnzL
    assert nnz_nd < 0.75 * nnz_nat, (nnz_nd, nnz_nat)
    assert nnz_nd < 1.6 * nnz_geo, (nnz_nd, nnz_geo)
    # the last vertices form a separator: removing them disconnects the grid
    D = inputs.dense_from_lower(A) != 0
    top = perm[-24:]
    keep = np.setdiff1d(np.arange(A.n), top)
    sub = D[np.ix_(keep, keep)]
    seen = {0}
    stack = [0]
    while stack:
        v = stack.pop()
        for u in np.nonzero(sub[v])[0].tolist():
            if u not in seen:
                seen.add(u)
                stack.append(u)
    assert len(seen) < len(keep)


@pytest.mark.parametrize("case", ["grid3d", "rand"])
def test_llt_probe_on_the_oracle_factor(case):
    """The size-independent check used on full-size GPU factors: the oracle's
    FP64 factor gives rounding-level residuals, and one wrong entry of L (a
    planted mistake) is seen."""
    from tests.factor_props import llt_probe
    if case == "grid3d":
        A = inputs.diffusion_3d_7pt(12, 11, 10, seed=4)
        perm0 = oracle.nd_grid(12, 11, 10, 8)
    else:
        A = inputs.random_spd(400, 0.02, 8)
        perm0 = None
    o = oracle.Oracle(A, perm0, pr=True, merge=0.125)
    assert o.factor() == 0
    s = o.symbolic()
    view = {"perm": s.perm, "sup_ptr": s.sup_ptr, "gl_ptr": s.gl_ptr, "glbind": s.glbind}
    L = o.L_supernodal()
    assert llt_probe(A, view, L) <= 1e-14
    bad = L.copy()
    k = int(np.argmax(np.abs(bad)))
    bad[k] *= 1.01
    assert llt_probe(A, view, bad) > 1e-4


@pytest.mark.parametrize("case", ["grid3d", "rand"])
def test_llt_probe_device_agrees_with_host_probe(case):
    """The in-place probe used on factors too large for the host (torch gather /
    index_add over the storage layout, here on a CPU tensor in the library's
    padded panel layout built from the oracle's factor): the same residual as
    the host probe, rounding-level on the oracle's factor, and a planted wrong
    entry seen."""
    torch = pytest.importorskip("torch")
    from tests.factor_props import llt_probe, llt_probe_device
    if case == "grid3d":
        A = inputs.diffusion_3d_7pt(12, 11, 10, seed=4)
        perm0 = oracle.nd_grid(12, 11, 10, 8)
    else:
        A = inputs.random_spd(400, 0.02, 8)
        perm0 = None
    o = oracle.Oracle(A, perm0, pr=True, merge=0.125)
    assert o.factor() == 0
    s = o.symbolic()
    view = {"perm": s.perm, "sup_ptr": s.sup_ptr, "gl_ptr": s.gl_ptr, "glbind": s.glbind}
    L = o.L_supernodal()
    # padded storage: each panel's rows 3 entries longer than its width, junk in
    # the padding and above the diagonal (neither is part of L)
    ns = len(s.sup_ptr) - 1
    w = np.diff(s.sup_ptr).astype(np.int64)
    m = np.diff(s.gl_ptr).astype(np.int64)
    ld = w + 3
    off = np.zeros(ns, np.int64)
    off[1:] = np.cumsum(m * ld)[:-1]
    store = np.full(int((m * ld).sum()), 7.0)
    q = 0
    for J in range(ns):
        blk = L[q:q + m[J] * w[J]].reshape(m[J], w[J]).copy()
        q += m[J] * w[J]
        blk[np.triu_indices(w[J], 1)] = 5.0
        store[off[J]:off[J] + m[J] * ld[J]].reshape(m[J], ld[J])[:, :w[J]] = blk
    dview = {"lnz": torch.tensor(store), "panel_off": off, "panel_ld": ld.astype(np.int32)}
    r_dev = llt_probe_device(A, view, dview, nprobe=2, group_entries=997)
    assert r_dev <= 1e-14
    assert abs(r_dev - llt_probe(A, view, L, nprobe=2)) <= 1e-15
    k = int(np.argmax(np.abs(L)))
    bad = L.copy()
    bad[k] *= 1.01
    # the same entry in the padded storage
    J = int(np.searchsorted(np.cumsum(m * w), k, side="right"))
    kk = k - int((m * w)[:J].sum())
    dview["lnz"][int(off[J] + (kk // w[J]) * ld[J] + kk % w[J])] *= 1.01
    assert llt_probe_device(A, view, dview, nprobe=2) > 1e-4
    assert abs(llt_probe_device(A, view, dview, nprobe=2) - llt_probe(A, view, bad, nprobe=2)) <= 1e-12


def test_nd_graph_ml_hand_orders():
    """Two 10-cliques joined by the edge 9-10, leaf 10, the multilevel split
    tried on every set (the library tries it from 64 vertices up). The
    multilevel bisection (20 vertices: no coarsening) grows part 0 from vertex
    0 over its clique {0..9} (cut 1, nothing for FM to gain); the boundary
    layers are {9} and {10}, so the separator is {9}, smaller than the level
    separator {1..9} (levels from 0 are {0}, {1..9}, {10}, {11..19}; from 11 no
    deeper). The level-structure order keeps {1..9}; so does nd_graph_ml, whose
    20-vertex set is below the multilevel threshold."""
    from oracle import ordering as od
    K = lambda off: [(i + off, j + off) for j in range(10) for i in range(j + 1, 10)]
    bar = inputs.from_lower_pattern(20, K(0) + K(10) + [(10, 9)])
    assert od._nested_dissection(bar, 10, True, ml_min=1).tolist() == list(range(9)) + list(range(10, 20)) + [9]
    level_order = [0] + list(range(10, 20)) + list(range(1, 10))
    assert oracle.nd_graph(bar, 10).tolist() == level_order
    assert oracle.nd_graph_ml(bar, 10).tolist() == level_order


def test_multilevel_building_blocks_by_hand():
    from oracle import ordering as od
    # heavy-edge matching: 0 takes 2 (weight 5 over 1); 1 stays alone; the two
    # unit edges 0-1 and 2-1 merge into one coarse edge of weight 2
    assert od._coarsen([1, 1, 1], [{1: 1, 2: 5}, {0: 1, 2: 1}, {0: 5, 1: 1}]) == ([0, 1, 0], [2, 1], [{1: 2}, {0: 2}])
    # path 0-1-2-3 cut 3 ways by [0,1,0,1], parts bounded by 3: vertex 1 (gain 2,
    # the smaller of the two best) moves first; the next moves bring nothing and
    # are undone; the second pass finds no gain
    path4 = [{1: 1}, {0: 1, 2: 1}, {1: 1, 3: 1}, {2: 1}]
    assert od._fm([1] * 4, path4, [0, 1, 0, 1], 3) == [0, 0, 0, 1]
    # cut edges a-c, a-r, a-s, p-c, q-c with a, p, q = 0, 1, 2 (part 0) and
    # c, r, s = 3, 4, 5: Kuhn matches 0-3, then 1 re-routes 0 to 4 and takes 3,
    # 2 finds nothing; alternating paths from 2 reach 3 and 1; the cover
    # {0, 3} is smaller than either boundary layer (3 vertices each)
    adj6 = [{3: 1, 4: 1, 5: 1}, {3: 1}, {3: 1}, {0: 1, 1: 1, 2: 1}, {0: 1}, {0: 1}]
    assert od._min_cover(adj6, [0, 0, 0, 1, 1, 1], [0, 1, 2]) == {0, 3}
    # growth from vertex 2 of a 6-path until 3 vertices: 2, then 1 and 3
    path6 = [{1: 1}, {0: 1, 2: 1}, {1: 1, 3: 1}, {2: 1, 4: 1}, {3: 1, 5: 1}, {4: 1}]
    assert od._grow([1] * 6, path6, 2, 3) == [1, 0, 0, 0, 1, 1]


def test_nd_graph_ml_finds_the_plane_of_a_27_point_cube():
    """On a 27-point 12^3 cube (no coordinates) the top separator is the axis
    plane z = 6 (144 vertices, the smallest balanced separator), where the
    level structure gives a cube shell; the fill is within 15 % of the
    geometric ND's."""
    from oracle import ordering as od
    A = inputs.stencil_3d_27pt(12, 12, 12, seed=3)
    nbr = od._neighbours(A)
    adj = [{u: 1 for u in nbr[g]} for g in range(A.n)]
    part = od._bisect([1] * A.n, adj)
    b0 = [i for i in range(A.n) if part[i] == 0 and any(part[u] == 1 for u in adj[i])]
    b1 = [i for i in range(A.n) if part[i] == 1 and any(part[u] == 0 for u in adj[i])]
    sep = np.array(b0 if len(b0) <= len(b1) else b1)
    assert len(sep) == 144 and len(np.unique(sep // 144)) == 1
    f_ml = oracle.Oracle(A, oracle.nd_graph_ml(A, 8), pr=False).symbolic().flops
    f_geo = oracle.Oracle(A, oracle.nd_grid(12, 12, 12, 8), pr=False).symbolic().flops
    f_bfs = oracle.Oracle(A, oracle.nd_graph(A, 8), pr=False).symbolic().flops
    assert f_ml <= 1.15 * f_geo and f_ml < 0.5 * f_bfs, (f_ml, f_geo, f_bfs)
