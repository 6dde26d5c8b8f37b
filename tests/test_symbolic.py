"""Host symbolic analysis of libsc against the oracle's separately written pass (CPU only).

Bit-exact on every array: ordering (ND + postorder + PR), supernodes, supernodal
parents, glbind, relind(J,p(J)), blocks, relindB(J,P) (the library composes it
as in Alg. 5, the oracle searches glbind(P) directly), levels, column etree.
"""
import re
import os

import numpy as np
import pytest

import oracle
import paper_2409_13090_gb300 as sc
from paper_2409_13090_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ["perm", "sup_ptr", "sup_parent", "gl_ptr", "glbind", "ri_ptr", "relind", "blk_ptr", "blk_first",
        "blk_size", "blk_owner", "rb_pair_ptr", "rb_pair_P", "rb_val_ptr", "rb_val", "level", "cparent"]


@pytest.fixture(scope="module", autouse=True)
def built():
    sc.build()


def _compare(A, *, grid=None, user_perm=None, pr=True, leaf=8, merge=0.0, graph_nd=False, graph_ml=False):
    if graph_nd or graph_ml:
        perm0 = (oracle.nd_graph_ml if graph_ml else oracle.nd_graph)(A, leaf)
        lib_sym = sc.Symbolic(A, ordering="graph_ml" if graph_ml else "graph_nd", nd_leaf=leaf, pr=pr, merge=merge)
    elif grid is not None:
        perm0 = oracle.nd_grid(*grid, leaf)
        lib_sym = sc.Symbolic(A, ordering="grid_nd", grid=grid, nd_leaf=leaf, pr=pr, merge=merge)
    elif user_perm is not None:
        perm0 = user_perm
        lib_sym = sc.Symbolic(A, ordering="user", user_perm=user_perm, pr=pr, merge=merge)
    else:
        perm0 = None
        lib_sym = sc.Symbolic(A, ordering="natural", pr=pr, merge=merge)
    o = oracle.Oracle(A, perm0, pr=pr, merge=merge).symbolic()
    v = lib_sym.view()
    for k in KEYS:
        assert np.array_equal(v[k], getattr(o, k)), k
    chk = lib_sym.check_schedule()
    assert chk["ok"], chk
    assert v["nnzL"] == o.nnzL and v["flops"] == o.flops and v["nsuper"] == o.nsuper
    return v


def test_worked_example_through_library(golden):
    ents = [(i - 1, j - 1) for i, j in golden["A_strict_lower_pattern"]["entries"]]
    A = inputs.from_lower_pattern(9, ents)
    v = sc.Symbolic(A, pr=False).view()
    assert v["sup_ptr"].tolist() == [0, 2, 4, 9]
    assert v["relind"].tolist() == golden["relind"]["J1_J3"] + golden["relind"]["J2_J3"]
    assert v["rb_val"].tolist() == golden["relindB"]["J1_J3"] + golden["relindB"]["J2_J3"]
    v = sc.Symbolic(A, pr=True).view()
    assert (v["blk_ptr"][1:3] - v["blk_ptr"][0:2]).tolist() == [1, 1]
    _compare(A, pr=False)
    _compare(A, pr=True)


def test_relind_composition_example(golden):
    g = golden["relind_composition"]
    assert sc.sc_relind_compose(g["relind_J_C"], g["relind_C_P"]).tolist() == g["relind_J_P"]


def test_indmap_example(golden):
    # relative indices of glbind(J3) with respect to itself: distance from the bottom
    g = golden["indmap_J3"]
    rows = g["rows"]
    assert [len(rows) - 1 - i for i in range(len(rows))] == g["values"]


@pytest.mark.parametrize("pr", [False, True])
def test_workload1_full(pr):
    A, _ = inputs.workload(1)
    _compare(A, grid=A.grid, pr=pr)


@pytest.mark.parametrize("idx,scale", [(2, 0.25), (2, 0.5), (3, 0.2), (3, 0.5), (5, 0.125)])
def test_workloads_scaled(idx, scale):
    A, _ = inputs.workload(idx, scale)
    _compare(A, grid=A.grid, pr=True)


@pytest.mark.parametrize("merge", [0.0, 0.125])
def test_workload2_full(merge):
    A, _ = inputs.workload(2)
    v = _compare(A, grid=A.grid, pr=True, merge=merge)
    assert v["nsuper"] > 1000


@pytest.mark.parametrize("idx,scale", [(1, 1.0), (2, 0.5), (3, 0.3), (5, 0.15)])
@pytest.mark.parametrize("merge", [0.05, 0.125, 0.5])
def test_merged_supernodes_bit_exact(idx, scale, merge):
    A, _ = inputs.workload(idx, scale)
    _compare(A, grid=A.grid, pr=True, merge=merge)


@pytest.mark.parametrize("seed", range(4))
def test_merged_random_bit_exact(seed):
    n = 80 + 50 * seed
    A = inputs.random_spd(n, 0.04, seed)
    perm = np.random.default_rng(7 + seed).permutation(n).astype(np.int32)
    _compare(A, user_perm=perm, pr=True, merge=0.125)
    _compare(A, pr=False, merge=0.3)


def test_workload4_members():
    mats, _ = inputs.workload(4, 0.1)
    for A in mats[:4]:
        _compare(A, grid=A.grid, pr=True)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("pr", [False, True])
def test_random_user_perm(seed, pr):
    n = 50 + 40 * seed
    A = inputs.random_spd(n, 0.05, seed)
    perm = np.random.default_rng(100 + seed).permutation(n).astype(np.int32)
    _compare(A, user_perm=perm, pr=pr)
    _compare(A, pr=pr)


def test_closed_form_special_cases():
    n = 40
    tri = inputs.from_lower_pattern(n, [(i + 1, i) for i in range(n - 1)])
    _compare(tri, pr=True)
    dense = inputs.from_lower_pattern(20, [(i, j) for j in range(20) for i in range(j + 1, 20)])
    v = _compare(dense, pr=True)
    assert v["nsuper"] == 1
    arrow = inputs.from_lower_pattern(n, [(n - 1, j) for j in range(n - 1)])
    _compare(arrow, pr=True)


def test_invalid_input_codes():
    A = inputs.laplacian_2d(4, 4)
    bad = A.rowind.copy()
    bad[1], bad[2] = bad[2], bad[1]  # unsorted rows in column 0
    o = sc.sc_options_default()
    rc, _ = sc.sc_analyze(A.n, np.ascontiguousarray(A.colptr), bad, o)
    assert rc == -3
    rc, _ = sc.sc_analyze(0, np.ascontiguousarray(A.colptr), np.ascontiguousarray(A.rowind), o)
    assert rc == -1
    o.ordering = 1
    o.grid[0], o.grid[1], o.grid[2] = 5, 4, 1  # wrong grid size
    rc, _ = sc.sc_analyze(A.n, np.ascontiguousarray(A.colptr), np.ascontiguousarray(A.rowind), o)
    assert rc == -4


def test_batch_concatenates_structures():
    mats = [inputs.laplacian_2d(5, 6, 0.1), inputs.laplacian_2d(7, 4, 0.2), inputs.laplacian_2d(3, 3, 0.3)]
    syms = [sc.Symbolic(A, ordering="grid_nd", grid=A.grid) for A in mats]
    b = sc.Symbolic.batch(syms).view()
    vs = [s.view() for s in syms]
    assert b["n"] == sum(v["n"] for v in vs) and b["nsuper"] == sum(v["nsuper"] for v in vs)
    assert b["nnzL"] == sum(v["nnzL"] for v in vs)
    off = 0
    parts = []
    for v in vs:
        parts.append(v["perm"] + off)
        off += v["n"]
    assert np.array_equal(b["perm"], np.concatenate(parts))


def test_library_exports_every_declared_symbol():
    """The C ABI library loads on a machine without a GPU and exports every function of include/sc.h."""
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "sc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(sc_\w+)\s*\(", hdr, flags=re.M))
    assert {"sc_analyze", "sc_factor", "sc_solve", "sc_refactor", "sc_analyze_batch", "sc_symbolic_export",
            "sc_numeric_free", "sc_symbolic_free", "sc_strerror", "sc_options_default"} <= names
    L = ctypes.CDLL(sc.build())
    for nm in sorted(names):
        assert hasattr(L, nm), nm


@pytest.mark.parametrize("ordering", ["graph_nd", "graph_ml"])
@pytest.mark.parametrize("case", ["rand", "grid2d", "grid3d", "st27", "disconnected", "path"])
@pytest.mark.parametrize("leaf", [1, 8, 32])
def test_graph_nd_ordering_bit_exact(case, leaf, ordering):
    """The general-graph nested dissection (no grid coordinates) gives the same
    permutation as the oracle's set-based restatement, and every symbolic array
    that follows from it agrees bit for bit."""
    if case == "rand":
        A = inputs.random_spd(300, 0.02, 5)
    elif case == "grid2d":
        A = inputs.laplacian_2d(23, 17)
    elif case == "grid3d":
        A = inputs.diffusion_3d_7pt(9, 8, 7, seed=1)
    elif case == "st27":
        A = inputs.stencil_3d_27pt(7, 7, 7, seed=2)
    elif case == "path":
        A = inputs.from_lower_pattern(200, [(i + 1, i) for i in range(199)])
    else:
        # three components: a 2D grid, a path and isolated vertices, interleaved labels
        rng = np.random.default_rng(9)
        lab = rng.permutation(150)
        ents = []
        for y in range(8):
            for x in range(8):
                v = x + 8 * y
                if x + 1 < 8:
                    ents.append((v, v + 1))
                if y + 1 < 8:
                    ents.append((v, v + 8))
        ents += [(64 + i, 65 + i) for i in range(70)]
        ents = [(max(lab[a], lab[b]), min(lab[a], lab[b])) for a, b in ents]
        A = inputs.from_lower_pattern(150, ents, seed=3)
    A.grid = None
    v = _compare(A, graph_nd=ordering == "graph_nd", graph_ml=ordering == "graph_ml", leaf=leaf, pr=True)
    assert np.array_equal(v["perm"][np.argsort(v["perm"])], np.arange(A.n))


@pytest.mark.parametrize("ordering", ["graph_nd", "graph_ml"])
@pytest.mark.parametrize("case", ["grid2d", "two_components"])
def test_graph_orderings_with_threads(case, ordering):
    """Graphs large enough that the top nested-dissection splits order their
    halves on separate threads (halves of at least 2048 vertices): the default
    thread count gives the oracle's permutation and symbolic arrays, and 1, 2,
    3 and 8 threads give the same permutation."""
    if case == "grid2d":
        A = inputs.laplacian_2d(100, 90)
    else:
        # a 2D grid and a 3D grid, labels interleaved: the components are ordered one by one
        rng = np.random.default_rng(4)
        n2, n3 = 80 * 64, 16 * 15 * 14
        lab = rng.permutation(n2 + n3)
        ents = []
        for y in range(64):
            for x in range(80):
                v = x + 80 * y
                if x + 1 < 80:
                    ents.append((v, v + 1))
                if y + 1 < 64:
                    ents.append((v, v + 80))
        for z in range(14):
            for y in range(15):
                for x in range(16):
                    v = n2 + x + 16 * (y + 15 * z)
                    if x + 1 < 16:
                        ents.append((v, v + 1))
                    if y + 1 < 15:
                        ents.append((v, v + 16))
                    if z + 1 < 14:
                        ents.append((v, v + 240))
        ents = [(max(lab[a], lab[b]), min(lab[a], lab[b])) for a, b in ents]
        A = inputs.from_lower_pattern(n2 + n3, ents, seed=5)
    A.grid = None
    v = _compare(A, graph_nd=ordering == "graph_nd", graph_ml=ordering == "graph_ml", leaf=8, pr=False)
    for th in (1, 2, 3, 8):
        w = sc.Symbolic(A, ordering=ordering, nd_leaf=8, pr=False, threads=th).view()
        assert np.array_equal(w["perm"], v["perm"]), th
    with pytest.raises(sc.SCError):
        sc.Symbolic(A, ordering=ordering, threads=-1)


@pytest.mark.parametrize("case", ["grid_merge", "graph_ml", "graph_nd_shortcuts"])
def test_analysis_same_for_every_thread_count(tmp_path, case):
    """The saved analysis (every array: structures, relind(B), the map of A's
    entries into Lnz, the residual's CSR, the launch plan inputs) is byte for
    byte the same on 1, 2 and 8 host threads; 30,000 columns, so the value map
    and the glbind sorts run in several blocks."""
    if case == "grid_merge":
        A = inputs.diffusion_3d_7pt(32, 32, 30, seed=7)
        kw = dict(ordering="grid_nd", grid=A.grid, merge=0.125)
    elif case == "graph_ml":
        A = inputs.laplacian_2d(120, 100)
        A.grid = None
        kw = dict(ordering="graph_ml")
    else:
        # a 2D grid with 600 random long-range edges: irregular separators
        rng = np.random.default_rng(8)
        k = 110
        ents = [(v + 1, v) for v in range(k * k) if (v % k) + 1 < k] + [(v + k, v) for v in range(k * k - k)]
        a, b = rng.integers(0, k * k, 600), rng.integers(0, k * k, 600)
        ents += [(int(max(x, y)), int(min(x, y))) for x, y in zip(a, b) if x != y]
        A = inputs.from_lower_pattern(k * k, sorted(set(ents)), seed=9)
        kw = dict(ordering="graph_nd", merge=0.125)
    blobs = []
    for th in (1, 2, 8):
        path = tmp_path / f"a{th}.scs"
        sc.Symbolic(A, threads=th, **kw).save(str(path))
        blobs.append(path.read_bytes())
    assert blobs[0] == blobs[1] == blobs[2]


def test_graph_nd_fill_close_to_geometric_nd():
    """On a 3D grid given without coordinates the graph ordering's fill stays
    within a small factor of the geometric ND and well below the natural order."""
    A = inputs.diffusion_3d_7pt(16, 16, 16, seed=1)
    nnz = {}
    for name, kw in [("graph", dict(ordering="graph_nd")), ("grid", dict(ordering="grid_nd", grid=(16, 16, 16))),
                     ("natural", dict(ordering="natural")), ("ml", dict(ordering="graph_ml"))]:
        nnz[name] = sc.Symbolic(A, pr=False, **kw).view()["nnzL"]
    assert nnz["graph"] < 2.0 * nnz["grid"], nnz
    assert nnz["graph"] < 0.5 * nnz["natural"], nnz
    assert nnz["ml"] <= nnz["graph"] * 1.05, nnz
    # 27-point coupling: the level separators are cube shells, the multilevel ones planes
    A = inputs.stencil_3d_27pt(16, 16, 16, seed=3)
    fl = {o: sc.Symbolic(A, pr=False, ordering=o, **({"grid": (16, 16, 16)} if o == "grid_nd" else {})).view()["flops"]
          for o in ("graph_nd", "graph_ml", "grid_nd")}
    assert fl["graph_ml"] < 1.15 * fl["grid_nd"] and fl["graph_ml"] < 0.4 * fl["graph_nd"], fl


def test_tune_table_changes_only_the_launch_plan():
    """The launch-plan settings move products between tiled tasks, device
    loops, tensor-core tiles and warp blocks (seen in the host-side plan), and
    leave every symbolic array bit-exact with the oracle."""
    A = inputs.diffusion_3d_7pt(14, 14, 14, seed=1)
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True).symbolic()

    def plan(**t):
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, tune=t or None)
        v = sym.view()
        for k in KEYS:
            assert np.array_equal(v[k], getattr(o, k)), (t, k)
        return sym.plan_stats("fp64"), sym.plan_stats("tf32")

    b64, btf = plan()
    assert btf["tc_tiles"] > 0 and b64["loop_items"] > 0
    # smaller tiling thresholds: more tiled tasks, among them thin ones
    f64, _ = plan(tile_min_entries=64, tile_min_k=1)
    assert f64["tiled_tasks"] > b64["tiled_tasks"] and f64["thin_units"] > 0
    n64, _ = plan(tile_min_entries=64, tile_min_k=1, thin_dim=-1)
    assert n64["thin_units"] == 0 and n64["simt_tiles"] > f64["simt_tiles"]
    h64, _ = plan(tile_min_entries=64, tile_min_k=1, thin_dim=4)
    assert 0 < h64["thin_units"] < f64["thin_units"]
    # larger thresholds: the Alg. 5 products stay in the device loops
    l64, _ = plan(tile_min_entries=1 << 20)
    assert l64["tiled_tasks"] < b64["tiled_tasks"]
    s64, _ = plan(loop_budget=256)
    assert s64["loop_items"] > b64["loop_items"] and s64["tiled_tasks"] == b64["tiled_tasks"]
    _, ttf = plan(tc_min_k=1 << 16)
    assert ttf["tc_tiles"] == 0 and ttf["simt_tiles"] > btf["simt_tiles"]
    _, wtf = plan(tc_wide_n=16, lookahead=-1)
    assert 0 < wtf["tc_tiles"] <= btf["tc_tiles"]


def test_256_column_tiles_only_in_tensor_core_plans():
    """The 256-column tensor-core tiles take the products at least tc_wide256
    wide that would take 128-column tiles: the tensor-core plans have them
    (fewer tiles in all), the FP64 / FP32 plans none, and with the setting
    above every width the plan is the 128-column one."""
    A = _dense_spd(1100, 4)
    sym = sc.Symbolic(A, ordering="natural")
    off = sc.Symbolic(A, ordering="natural", tune=dict(tc_wide256=1 << 20))
    for prec in ("tf32", "tf32x3"):
        s, o = sym.plan_stats(prec), off.plan_stats(prec)
        assert s["tc256_tiles"] > 0 and o["tc256_tiles"] == 0
        assert 0 < s["tc_tiles"] < o["tc_tiles"]
        assert s["tasks"] == o["tasks"] and s["simt_tiles"] == o["simt_tiles"]
    for prec in ("fp64", "fp32"):
        assert sym.plan_stats(prec)["tc256_tiles"] == 0 and sym.plan_stats(prec)["tc_tiles"] == 0
    assert sym.check_schedule()["ok"]
    # clusters of two (the default): the 256-column tiles come in pairs, completed
    # where a product has an odd number of row tiles or a lower product's pair
    # straddles the diagonal; one CTA per tile lists only the real ones
    one = sc.Symbolic(A, ordering="natural", tune=dict(tc_multicast=-1)).plan_stats("tf32")
    pairs = sym.plan_stats("tf32")
    assert pairs["tc256_tiles"] % 2 == 0 and pairs["tc256_tiles"] >= one["tc256_tiles"] > 0
    assert pairs["tc256_tiles"] <= 2 * one["tc256_tiles"]


def test_deferral_depth_changes_only_the_in_panel_products():
    """A third level of trailing-update deferral (outer blocks of 1024 or 4096
    columns) regroups the in-supernode products: the same flops in fewer
    read-modify-write passes (each target column takes at most three updates of
    K = chunk width, three of K = 256, and one of K = the outer width per outer
    block), while every symbolic array stays bit-exact and the schedule check
    passes. One dense supernode of 2100 columns shows it."""
    A = _dense_spd(2100, 3)
    o = oracle.Oracle(A, None, pr=True).symbolic()

    def passes(defer):
        """128-row tensor-core target tiles of the TF32 plan: one read-modify-write pass each"""
        sym = sc.Symbolic(A, ordering="natural", tune=None if defer is None else dict(defer_width=defer))
        assert sym.check_schedule()["ok"]
        v = sym.view()
        for k in KEYS:
            assert np.array_equal(v[k], getattr(o, k)), (defer, k)
        return sym.plan_stats("tf32")["tc_tiles"]

    two = passes(256)  # two levels: macro panels only
    assert passes(None) == passes(512)  # the default outer width
    # an outer block boundary replaces the macro panels' updates of all later columns
    assert passes(512) < two and passes(1024) < two
    # an outer block wider than the supernode is the two-level schedule
    assert passes(4096) == two


@pytest.mark.parametrize("bad", [dict(lookahead=2), dict(tc_min_k=16), dict(tc_wide_n=8), dict(tc_wide256=8),
                                 dict(solve_group=2000), dict(tc_multicast=2),
                                 dict(thin_dim=9),
                                 dict(thin_dim=-2), dict(loop_budget=100), dict(tile_min_entries=-1),
                                 dict(defer_width=128), dict(defer_width=1 << 21)])
def test_tune_table_ranges(bad):
    A = inputs.laplacian_2d(8, 8)
    with pytest.raises(sc.SCError) as e:
        sc.Symbolic(A, tune=bad)
    assert e.value.code == -4


def test_tune_argument_checks_before_device_work():
    A = inputs.laplacian_2d(8, 8)
    sym = sc.Symbolic(A)
    for kw, code in [(dict(reps=0), -5), (dict(reps=16), -5), (dict(precision="fp64", reps=0), -5)]:
        with pytest.raises(sc.SCError) as e:
            sym.tune(A.values, **kw)
        assert e.value.code == code


@pytest.mark.parametrize("variant", ["rlb", "rl"])
@pytest.mark.parametrize("chunk", [8, 24, 64])
@pytest.mark.parametrize("merge", [0.0, 0.125])
def test_schedule_check_on_workloads(variant, chunk, merge):
    """Every product task, device-loop item and RL assembly pair of the schedule
    stays inside its panels, lands where glbind says, and respects the level
    order, on each workload (scaled) and a random matrix."""
    cases = [inputs.workload(i, sc_)[0] for i, sc_ in ((1, 1.0), (2, 0.3), (3, 0.2), (5, 0.15))]
    cases.append(inputs.random_spd(500, 0.01, 3))
    for A in cases:
        kw = dict(ordering="grid_nd", grid=A.grid) if A.grid and A.grid[0] else dict(ordering="graph_nd")
        sym = sc.Symbolic(A, variant=variant, chunk=chunk, merge=merge, **kw)
        chk = sym.check_schedule()
        assert chk["ok"], (A.name, chk)
        assert chk["tasks"] + chk["loop_products"] > 0


def test_schedule_check_under_plan_settings_and_batches():
    A = inputs.diffusion_3d_7pt(12, 12, 12, seed=2)
    for t in (dict(tile_min_entries=64, tile_min_k=1), dict(tile_min_entries=1 << 20, loop_budget=256),
              dict(defer_width=1024), dict(defer_width=4096, lookahead=-1)):
        chk = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, tune=t).check_schedule()
        assert chk["ok"], (t, chk)
    mats, _ = inputs.workload(4, 0.06)
    syms = [sc.Symbolic(M, ordering="grid_nd", grid=M.grid, merge=0.125) for M in mats]
    chk = sc.Symbolic.batch(syms).check_schedule()
    assert chk["ok"], chk


@pytest.mark.parametrize("kind,expect", [(1, "entry mapping"), (2, "critical flag"), (3, "level order"),
                                         (4, "source range")])
def test_schedule_check_finds_planted_mistakes(kind, expect):
    """A mistake planted by the test hook is found, and the altered handle
    refuses to factor (before any device work)."""
    A = inputs.workload(2, 0.5)[0]
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=0.125)
    assert sym._perturb_schedule(kind) == 0
    chk = sym.check_schedule()
    assert not chk["ok"] and chk["kind"] == expect, chk
    with pytest.raises(sc.SCError) as e:
        sym.factor(A.values)
    assert e.value.code == sc.SC_ERR_INTERNAL


def test_schedule_check_finds_tensor_core_k_tail():
    """Chunk widths whose in-panel updates have a K that is not a whole number
    of 8-column MMA steps (36: K = 36 and macro panels of 252 columns): the
    library keeps those products off the tensor cores (the check passes), and a
    plan that routes them there anyway (test hook 5) is found."""
    A = _dense_spd(300, 5)
    for chunk in (24, 36, 40, 48, 64):
        chk = sc.Symbolic(A, ordering="natural", chunk=chunk).check_schedule()
        assert chk["ok"], (chunk, chk)
    sym = sc.Symbolic(A, ordering="natural", chunk=36)
    assert sym._perturb_schedule(5) == 0
    chk = sym.check_schedule()
    assert not chk["ok"] and chk["kind"] == "tensor-core K range", chk
    with pytest.raises(sc.SCError) as e:
        sym.factor(A.values)
    assert e.value.code == sc.SC_ERR_INTERNAL
    # no K tail with chunks of 64: nothing to plant
    assert sc.Symbolic(A, ordering="natural", chunk=64)._perturb_schedule(5) == sc.SC_ERR_UNSUPPORTED


@pytest.mark.parametrize("case", ["st27", "aniso", "random", "batch"])
@pytest.mark.parametrize("chunk", [64, 24])
def test_deterministic_plan(case, chunk):
    """A deterministic schedule (RL): the same pairs as without the option, no
    product tile split along the inner dimension, every target row of every
    RL assembly pair owned by a slab of its target with the pairs in source
    order (the schedule check, kind 13, on the FP64 and tensor-core plans); and
    the option needs the RL variant and matches across a batch."""
    if case == "st27":
        A = inputs.workload(3, 0.2)[0]
        kw = dict(ordering="grid_nd", grid=A.grid, merge=0.125)
    elif case == "aniso":
        A = inputs.anisotropic_3d_7pt(20, 14, 11, seed=3, shift=1e-2)
        kw = dict(ordering="grid_nd", grid=A.grid)
    elif case == "random":
        A = inputs.random_spd(500, 0.02, 9)
        kw = dict(ordering="graph_nd", pr=False)
    else:
        mats, _ = inputs.workload(4, 0.05)
        syms = [sc.Symbolic(M, ordering="grid_nd", grid=M.grid, variant="rl", chunk=chunk, deterministic=True)
                for M in mats]
        b = sc.Symbolic.batch(syms)
        assert b.check_schedule()["ok"]
        assert b.plan_stats("fp64")["split_tiles"] == 0 and b.plan_stats("fp64")["rl_slabs"] > 0
        mixed = syms[:1] + [sc.Symbolic(mats[1], ordering="grid_nd", grid=mats[1].grid, variant="rl", chunk=chunk)]
        with pytest.raises(sc.SCError) as e:
            sc.Symbolic.batch(mixed)
        assert e.value.code == -2
        return
    det = sc.Symbolic(A, variant="rl", chunk=chunk, deterministic=True, **kw)
    chk = det.check_schedule()
    assert chk["ok"], chk
    plain = sc.Symbolic(A, variant="rl", chunk=chunk, **kw)
    for prec in ("fp64", "fp32", "tf32"):
        d, p = det.plan_stats(prec), plain.plan_stats(prec)
        assert d["split_tiles"] == 0 and p["rl_slabs"] == 0 and d["rl_slabs"] >= 1
        assert d["rl_pairs"] == p["rl_pairs"] and d["tasks"] == p["tasks"]
    with pytest.raises(sc.SCError) as e:
        sc.Symbolic(A, variant="rlb", deterministic=True, **kw)
    assert e.value.code == -4


def test_deterministic_plan_split_tiles_exist_without_it():
    """The matrices above do split tiles without the option (the critical
    in-panel updates with K = 64), so the zero counts are not vacuous."""
    A = inputs.workload(3, 0.2)[0]
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=0.125, variant="rl")
    assert sym.plan_stats("fp64")["split_tiles"] > 0


def test_schedule_check_finds_unowned_assembly_row():
    """Test hook 6: the first level of assembly slabs misses a target row; the
    deterministic-plan check (kind 13) finds it and the handle refuses to
    factor. Without the option there is nothing to plant."""
    A = inputs.workload(2, 0.3)[0]
    kw = dict(ordering="grid_nd", grid=A.grid, variant="rl")
    sym = sc.Symbolic(A, deterministic=True, **kw)
    assert sym._perturb_schedule(6) == 0
    chk = sym.check_schedule()
    assert not chk["ok"] and chk["kind"] == "deterministic plan", chk
    with pytest.raises(sc.SCError) as e:
        sym.factor(A.values)
    assert e.value.code == sc.SC_ERR_INTERNAL
    assert sc.Symbolic(A, **kw)._perturb_schedule(6) == sc.SC_ERR_UNSUPPORTED


def _dense_spd(n, seed):
    ents = [(i, j) for j in range(n) for i in range(j + 1, n)]
    return inputs.from_lower_pattern(n, ents, seed=seed)


def _same_handles(a, b, precisions=("fp64", "tf32")):
    va, vb = a.view(), b.view()
    for k in KEYS:
        assert np.array_equal(va[k], vb[k]), k
    for k in ("n", "nsuper", "nnzL", "flops"):
        assert va[k] == vb[k], k
    for p in precisions:
        assert a.plan_stats(p) == b.plan_stats(p), p
    assert b.check_schedule()["ok"]


@pytest.mark.parametrize("case", ["grid_merge", "rl", "graph_nd", "tuned", "deterministic", "batch"])
def test_symbolic_save_load_round_trip(tmp_path, case):
    """A saved analysis loads into a handle equal to the original in every
    exported array and in the launch plan it gives."""
    A = inputs.workload(2, 0.3)[0]
    if case == "grid_merge":
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=0.125)
    elif case == "rl":
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, variant="rl", chunk=24)
    elif case == "graph_nd":
        sym = sc.Symbolic(inputs.random_spd(400, 0.02, 4), ordering="graph_nd", pr=False)
    elif case == "tuned":
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, tune=dict(tile_min_entries=64, thin_dim=4))
    elif case == "deterministic":
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, variant="rl", deterministic=True)
    else:
        mats, _ = inputs.workload(4, 0.05)
        sym = sc.Symbolic.batch([sc.Symbolic(M, ordering="grid_nd", grid=M.grid) for M in mats])
    path = tmp_path / "sym.scs"
    sym.save(path)
    _same_handles(sym, sc.Symbolic.load(path))


def test_symbolic_load_rejects_damaged_files(tmp_path):
    A = inputs.laplacian_2d(20, 20)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=(20, 20, 1))
    path = tmp_path / "sym.scs"
    sym.save(path)
    data = path.read_bytes()
    cases = {"truncated": data[:-20], "flipped": data[:100] + bytes([data[100] ^ 1]) + data[101:],
             "empty": b"", "magic": b"X" + data[1:]}
    for name, blob in cases.items():
        bad = tmp_path / f"{name}.scs"
        bad.write_bytes(blob)
        with pytest.raises(sc.SCError) as e:
            sc.Symbolic.load(bad)
        assert e.value.code == sc.SC_ERR_IO, name
    with pytest.raises(sc.SCError) as e:
        sc.Symbolic.load(tmp_path / "missing.scs")
    assert e.value.code == sc.SC_ERR_IO
    # a handle altered by the test hook is not written
    assert sym._perturb_schedule(4) == 0
    with pytest.raises(sc.SCError) as e:
        sym.save(tmp_path / "poisoned.scs")
    assert e.value.code == sc.SC_ERR_INTERNAL


def test_c_abi_from_plain_c(tmp_path):
    """include/sc.h compiles as C99 with warnings as errors, and a C program
    drives the host half of the ABI (analysis with three orderings, the graph
    orderings also on 1 and 5 threads, export, schedule check, plan, save /
    load) against the built library; its numbers match the Python binding's."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(sc._LIB_PATH)
    exe = tmp_path / "abi_check"
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi", "abi_check.c"), "-o", str(exe), "-L", lib_dir,
                           "-lsc", "-Wl,-rpath," + lib_dir])
    out = subprocess.check_output([str(exe), "24", str(tmp_path / "a.scs")], text=True).splitlines()
    assert len(out) == 4
    A = inputs.laplacian_2d(24, 24)
    for line, (ordering, kw) in zip(out, [("grid_nd", dict(grid=(24, 24, 1))), ("graph_nd", {}), ("graph_ml", {})]):
        f = line.split()
        v = sc.Symbolic(A, ordering=ordering, **kw).view()
        assert int(f[5]) == v["nsuper"] and int(f[7]) == v["nnzL"], (line, ordering)
    # the deterministic RL analysis from C: the same pairs and slabs as through the binding
    st = sc.Symbolic(A, ordering="grid_nd", grid=(24, 24, 1), variant="rl", deterministic=True,
                     tune=dict(defer_width=1024, solve_group=3, tc_multicast=-1)).plan_stats("fp64")
    f = out[3].split()
    assert f[:2] == ["deterministic", "rl"] and int(f[3]) == st["rl_pairs"] and int(f[5]) == st["rl_slabs"], out[3]
    # an 80 x 80 grid: the top splits of the graph orderings run on two threads
    out = subprocess.check_output([str(exe), "80", str(tmp_path / "b.scs")], text=True).splitlines()
    assert len(out) == 4


@pytest.mark.parametrize("seed", range(12))
def test_random_patterns_all_options(seed):
    """Random sparse patterns (varied size and density, sometimes disconnected)
    under every ordering, both variants, merging on/off, PR on/off and several
    chunk widths: the library's symbolic arrays bit-exact with the oracle's and
    the device schedule passing the host-side check."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(5, 160))
    density = float(rng.choice([0.01, 0.03, 0.08, 0.2]))
    ents = set()
    for j in range(n):
        for i in range(j + 1, n):
            if rng.random() < density:
                ents.add((i, j))
    A = inputs.from_lower_pattern(n, sorted(ents), seed=seed)
    A.grid = None
    merge = float(rng.choice([0.0, 0.125, 0.5]))
    pr = bool(rng.integers(0, 2))
    variant = str(rng.choice(["rlb", "rl"]))
    chunk = int(rng.choice([4, 16, 64]))
    for ordering in ("natural", "graph_nd", "graph_ml", "user"):
        if ordering == "user":
            perm0 = rng.permutation(n).astype(np.int32)
            sym = sc.Symbolic(A, ordering="user", user_perm=perm0, pr=pr, merge=merge, variant=variant, chunk=chunk)
        elif ordering == "natural":
            perm0 = None
            sym = sc.Symbolic(A, pr=pr, merge=merge, variant=variant, chunk=chunk)
        else:
            perm0 = (oracle.nd_graph_ml if ordering == "graph_ml" else oracle.nd_graph)(A, 8)
            sym = sc.Symbolic(A, ordering=ordering, pr=pr, merge=merge, variant=variant, chunk=chunk)
        o = oracle.Oracle(A, perm0, pr=pr, merge=merge).symbolic()
        v = sym.view()
        for k in KEYS:
            assert np.array_equal(v[k], getattr(o, k)), (ordering, k)
        chk = sym.check_schedule()
        assert chk["ok"], (ordering, chk)
