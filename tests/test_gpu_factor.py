"""GPU factor and solve through the C ABI against the oracle (needs a GB300).

Parity bars (written here, derived from the arithmetic):
- FP64 factor: every supernode block of L agrees with the oracle's L within
  |L_gpu - L_or| <= 1e-10 * max|L_or| elementwise (the two sum the same
  products in different orders; the growth for these SPD inputs stays far below
  1e6 u), and the solve reaches eta <= 1e-14.
- FP32 / TF32 / TF32x3 factor: L within 1e-3 (FP32, TF32x3) or 2e-2 (TF32) relative to max|L|
  on well-conditioned inputs; after FP64 refinement eta <= 1e-14.
- structure: the library's symbolic arrays are bit-exact with the oracle's.
- non-positive-definite input: the reported column equals the oracle's.
"""
import numpy as np
import pytest

import oracle
import paper_2409_13090_gb300 as sc
from paper_2409_13090_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc.build()
    oracle.build()


def _grid_case(name):
    if name == "lap2d_64":
        return inputs.workload(1)[0]
    if name == "diff7_24":
        return inputs.workload(2, 0.5)[0]
    if name == "diff7_13":
        return inputs.diffusion_3d_7pt(13, 11, 9, seed=5, shift=1e-2)
    if name == "st27_14":
        return inputs.workload(3, 14 / 80)[0]
    if name == "aniso_16":
        return inputs.anisotropic_3d_7pt(16, 16, 16, seed=6, shift=1e-2)
    if name == "lap2d_ragged":
        return inputs.laplacian_2d(37, 29, 0.05)
    raise KeyError(name)


def _oracle_L(A, perm0):
    o = oracle.Oracle(A, perm0, pr=True)
    assert o.factor() == 0
    return o, o.L_supernodal()


def _check_L(Lg, Lo, tol):
    scale = np.abs(Lo).max()
    err = np.abs(Lg - Lo).max()
    assert err <= tol * scale, f"max |L_gpu - L_oracle| = {err:.3e} > {tol:.1e} * {scale:.3e}"


@pytest.mark.parametrize("name", ["lap2d_64", "diff7_24", "diff7_13", "st27_14", "aniso_16", "lap2d_ragged"])
@pytest.mark.parametrize("variant", ["rlb", "rl"])
def test_fp64_factor_matches_oracle(name, variant):
    A = _grid_case(name)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, variant=variant)
    o, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
    num = sym.factor(A.values, precision="fp64")
    assert num.rc == 0
    _check_L(num.export_L(), Lo, 1e-10)
    B = inputs.rhs(A.n, 4, 3)
    X, info = num.solve(B)
    eta = oracle.backward_error(A, B, X)
    assert eta.max() <= 1e-14, eta
    Xo = o.solve(B)
    assert np.abs(X - Xo).max() <= 1e-8 * np.abs(Xo).max()


@pytest.mark.parametrize("merge", [0.125, 0.4])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32", 2e-2)])
def test_merged_supernodes_factor(merge, prec, tol):
    A = _grid_case("st27_14")
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=merge)
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True, merge=merge)
    assert o.factor() == 0
    num = sym.factor(A.values, precision=prec)
    _check_L(num.export_L(), o.L_supernodal(), tol)
    B = inputs.rhs(A.n, 2, 8)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("chunk", [8, 24, 64])
def test_chunk_widths(chunk):
    A = _grid_case("diff7_13")
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, chunk=chunk)
    _, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
    num = sym.factor(A.values, precision="fp64")
    _check_L(num.export_L(), Lo, 1e-10)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("tf32", 2e-2), ("tf32x3", 1e-3)])
@pytest.mark.parametrize("name", ["lap2d_64", "st27_14", "lap2d_ragged"])
def test_low_precision_factor_and_refinement(prec, tol, name):
    A = _grid_case(name)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    _, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    _check_L(num.export_L(), Lo, tol)
    B = inputs.rhs(A.n, 3, 4)
    X, info = num.solve(B)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


def test_values_from_device_and_refactor():
    import torch
    A = _grid_case("diff7_13")
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    dv = torch.tensor(A.values, device="cuda", dtype=torch.float64)
    num = sym.factor(dv, precision="fp64")
    L1 = num.export_L()
    v2 = A.values * 2.0
    num.refactor(v2)
    L2 = num.export_L()
    assert np.allclose(L2, L1 * np.sqrt(2.0), rtol=1e-12, atol=1e-14)
    # device right-hand sides: (nrhs, n) contiguous = column-major n x nrhs
    B = inputs.rhs(A.n, 2, 5)
    Bd = torch.tensor(np.ascontiguousarray(B.T), device="cuda")
    Xd, info = num.solve(Bd)
    X = Xd.cpu().numpy().T
    A2 = inputs.SparseSym(A.n, A.colptr, A.rowind, v2)
    assert oracle.backward_error(A2, B, X).max() <= 1e-14


def test_not_positive_definite_column_matches_oracle():
    A = inputs.laplacian_2d(20, 20)
    v = A.values.copy()
    v[A.colptr[137]] = -50.0  # diagonal of column 137
    perm0 = oracle.nd_grid(20, 20, 1, 8)
    o = oracle.Oracle(A, perm0, pr=True)
    info_or = o.factor(v)
    assert info_or > 0
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    num = sym.factor(v, precision="fp64")
    assert num.rc == info_or and num.failed_col == info_or


def test_batch_factor_matches_per_matrix():
    mats, _ = inputs.workload(4, 0.08)
    syms = [sc.Symbolic(A, ordering="grid_nd", grid=A.grid) for A in mats]
    bsym = sc.Symbolic.batch(syms)
    vals = np.concatenate([A.values for A in mats])
    num = bsym.factor(vals, precision="fp64")
    assert num.rc == 0
    Lb = num.export_L()
    off = 0
    for A in mats:
        _, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
        _check_L(Lb[off:off + Lo.size], Lo, 1e-10)
        off += Lo.size
    B = inputs.rhs(bsym.n, 1, 9)
    X, _ = num.solve(B, refine=True)
    r0 = 0
    for A in mats:
        assert oracle.backward_error(A, B[r0:r0 + A.n], X[r0:r0 + A.n]).max() <= 1e-14
        r0 += A.n


@pytest.mark.parametrize("merge", [0.0, 0.125])
def test_full_workload2_fp64_parity(merge):
    """48^3 7-point variable-coefficient matrix, FP64 RLB (the benchmark's launch uses merge 0.125):
    L elementwise vs the oracle's Alg. 1 factor, and the backward error of 4 right-hand sides."""
    A, nrhs = inputs.workload(2)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=merge)
    num = sym.factor(A.values, precision="fp64")
    assert num.rc == 0
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True, merge=merge)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    _check_L(num.export_L(), Lo, 1e-9)
    B = inputs.rhs(A.n, nrhs, 2)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14


def test_anisotropic_near_singular_fp64_parity_and_cg():
    """The anisotropic 7-point matrix with the 1e-8 shift (1:1:100 coupling x
    log-uniform[0.1, 10]; kappa ~ 1e10 at 16^3): FP64 L against the oracle's L,
    PR on and off, and conjugate gradients preconditioned by the TF32x3 factor
    reaching eta <= 1e-14 (classical refinement cannot: kappa x u > 1)."""
    A, nrhs = inputs.workload(5, 0.125)
    perm0 = oracle.nd_grid(*A.grid, 8)
    B = inputs.rhs(A.n, 4, 17)
    for pr in (True, False):
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, pr=pr)
        o = oracle.Oracle(A, perm0, pr=pr)
        assert o.factor() == 0
        num = sym.factor(A.values, precision="fp64")
        assert num.rc == 0
        _check_L(num.export_L(), o.L_supernodal(), 1e-9)
        X, _ = num.solve(B, refine=True)
        assert oracle.backward_error(A, B, X).max() <= 1e-14
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=0.125)
    num = sym.factor(A.values, precision="tf32x3")
    X, info = num.solve(B, method="cg", max_iterations=500)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_low_pivot_blocks_redone_in_fp64(prec):
    """The low-precision pivot rule: a diagonal block whose FP32 pivot d falls to
    tau * |A_jj| or below is refactored in FP64 from the same stored values, and
    the count is reported. With tau = 0.5 many blocks qualify (pivots drop below
    half the input diagonal as elimination proceeds); with the default 2^-10
    none do on this well-conditioned matrix. Either way L matches the oracle to
    FP32 accuracy and refinement reaches eta <= 1e-14; the redone blocks are
    FP64-accurate, so the factor with tau = 0.5 is no further from the oracle
    (within a factor 2 for the FP32 rounding of the rest)."""
    A = _grid_case("diff7_13")
    _, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
    scale = np.abs(Lo).max()
    B = inputs.rhs(A.n, 2, 19)
    errs = {}
    for tau in (2.0 ** -10, 0.5):
        sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, pivot_tau=tau)
        num = sym.factor(A.values, precision=prec)
        assert num.rc == 0
        fb = num.info.pivot_fallbacks
        if tau == 0.5:
            assert fb > 0
        else:
            assert fb == 0
        errs[tau] = np.abs(num.export_L() - Lo).max() / scale
        assert errs[tau] <= 1e-3
        X, info = num.solve(B)
        assert info["converged"], info
        assert oracle.backward_error(A, B, X).max() <= 1e-14
    assert errs[0.5] <= errs[2.0 ** -10] * 2 + 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_factor_batch_entry_point(prec):
    """sc_factor_batch: the values of each matrix gathered into one batched
    factorization; L of every member matches its oracle factor (FP64 bound, or
    the FP32 bound), and the batch solve reaches eta <= 1e-14 per matrix."""
    import torch
    mats, _ = inputs.workload(4, 0.06)
    syms = [sc.Symbolic(A, ordering="grid_nd", grid=A.grid) for A in mats]
    vals = [torch.tensor(A.values, device="cuda", dtype=torch.float64) for A in mats]
    bsym, num = sc.Symbolic.factor_batch(syms, vals, precision=prec)
    assert num.rc == 0
    Lb = num.export_L()
    off = 0
    for A in mats:
        _, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
        _check_L(Lb[off:off + Lo.size], Lo, 1e-10 if prec == "fp64" else 1e-3)
        off += Lo.size
    B = inputs.rhs(bsym.n, 1, 23)
    X, info = num.solve(B)
    r0 = 0
    for A in mats:
        assert oracle.backward_error(A, B[r0:r0 + A.n], X[r0:r0 + A.n]).max() <= 1e-14
        r0 += A.n


@pytest.mark.parametrize("ordering", ["graph_nd", "graph_ml"])
@pytest.mark.parametrize("case", ["rand", "diff7_14_no_grid", "st27_10_no_grid"])
@pytest.mark.parametrize("variant", ["rlb", "rl"])
def test_graph_nd_ordering_factor(case, variant, ordering):
    """Inputs without grid coordinates ordered by the general-graph nested
    dissections: the FP64 factor matches the oracle's under the oracle's own
    restatement of that ordering, and the solve reaches eta <= 1e-14."""
    if case == "rand":
        A = inputs.random_spd(2000, 0.003, 21)
    elif case == "diff7_14_no_grid":
        A = inputs.diffusion_3d_7pt(14, 14, 14, seed=2)
    else:
        A = inputs.stencil_3d_27pt(10, 10, 10, seed=2)
    A.grid = None
    sym = sc.Symbolic(A, ordering=ordering, variant=variant)
    o, Lo = _oracle_L(A, (oracle.nd_graph_ml if ordering == "graph_ml" else oracle.nd_graph)(A, 8))
    num = sym.factor(A.values, precision="fp64")
    assert num.rc == 0
    _check_L(num.export_L(), Lo, 1e-10)
    B = inputs.rhs(A.n, 3, 5)
    X, info = num.solve(B)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


PLAN_TABLES = [
    dict(tile_min_entries=64, tile_min_k=1),
    dict(tile_min_entries=64, tile_min_k=1, thin_dim=-1, loop_budget=256),
    dict(tile_min_entries=1 << 20, loop_budget=1 << 17),
    dict(lookahead=-1, thin_dim=4),
    dict(tc_min_k=128, tc_wide_n=16),
    dict(tc_wide_n=128, tile_min_entries=512, tile_min_k=32),
]


@pytest.mark.parametrize("table", range(len(PLAN_TABLES)))
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32", 2e-2)])
def test_launch_plan_settings_keep_parity(table, prec, tol):
    """Every launch-plan setting the tuner may pick (and extreme ones) gives
    the same factor: products only move between kernels."""
    A = _grid_case("st27_14")
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, tune=PLAN_TABLES[table])
    o, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    _check_L(num.export_L(), Lo, tol)
    B = inputs.rhs(A.n, 2, 3)
    X, info = num.solve(B)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("name,prec,tol", [("diff7_24", "fp64", 1e-10), ("st27_14", "tf32", 2e-2)])
def test_tuner_keeps_the_fastest_setting(name, prec, tol):
    A = _grid_case(name)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    t = sym.tune(A.values, precision=prec, reps=1)
    assert t["tried"] >= 5 and t["factor_ms"] > 0, t
    # the table is a valid option set; the tuned handle factors correctly
    sc.Symbolic(A, ordering="grid_nd", grid=A.grid, tune={k: t[k] for k in sc.TUNE_FIELDS})
    o, Lo = _oracle_L(A, oracle.nd_grid(*A.grid, 8))
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    _check_L(num.export_L(), Lo, tol)
    # a live numeric handle blocks retuning
    with pytest.raises(sc.SCError) as e:
        sym.tune(A.values, precision=prec, reps=1)
    assert e.value.code == sc.SC_ERR_IN_USE


def test_loaded_symbolic_factors_like_the_original(tmp_path):
    """Analyse, save, load in place of a new analysis: the loaded handle's FP64
    factor matches the oracle's, and its TF32 factor the original handle's."""
    A = _grid_case("diff7_24")
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=0.125)
    sym.save(tmp_path / "a.scs")
    loaded = sc.Symbolic.load(tmp_path / "a.scs")
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True, merge=0.125)
    assert o.factor() == 0
    num = loaded.factor(A.values, precision="fp64")
    assert num.rc == 0
    _check_L(num.export_L(), o.L_supernodal(), 1e-10)
    Lt = sym.factor(A.values, precision="tf32").export_L()
    Ltl = loaded.factor(A.values, precision="tf32").export_L()
    assert np.abs(Lt - Ltl).max() <= 1e-5 * np.abs(Lt).max()
    B = inputs.rhs(A.n, 2, 4)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14


def _degenerate(name):
    rng = np.random.default_rng(11)
    if name == "n1":
        A = inputs.from_lower_pattern(1, [])
        A.values[:] = 4.0
    elif name == "diagonal":
        A = inputs.from_lower_pattern(50, [])
        A.values[:] = rng.uniform(0.5, 2.0, 50)
    elif name == "tridiagonal":
        A = inputs.from_lower_pattern(100, [(i + 1, i) for i in range(99)], seed=2)
    elif name == "dense":
        A = inputs.from_lower_pattern(40, [(i, j) for j in range(40) for i in range(j + 1, 40)], seed=3)
    elif name == "arrowhead":
        A = inputs.from_lower_pattern(60, [(59, j) for j in range(59)], seed=4)
    else:  # two independent dense blocks: a forest of two supernodes
        ents = [(i, j) for j in range(15) for i in range(j + 1, 15)]
        A = inputs.from_lower_pattern(30, ents + [(i + 15, j + 15) for i, j in ents], seed=5)
    return A


@pytest.mark.parametrize("name", ["n1", "diagonal", "tridiagonal", "dense", "arrowhead", "forest"])
@pytest.mark.parametrize("variant", ["rlb", "rl"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("tf32x3", 1e-5)])
def test_degenerate_structures(name, variant, prec, tol):
    """The structures at the method's extremes: one unknown, no off-diagonal
    entries (every supernode a root, no updates), a chain (one level per
    column), one dense supernode, a star, and a forest. L against the oracle's,
    then the solve to eta <= 1e-14."""
    A = _degenerate(name)
    sym = sc.Symbolic(A, variant=variant)
    assert sym.check_schedule()["ok"]
    o, Lo = _oracle_L(A, None)
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    _check_L(num.export_L(), Lo, tol)
    B = inputs.rhs(A.n, 3, 6)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14, info


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-3)])
@pytest.mark.parametrize("name", ["diff7_24s", "st27_14", "lap2d_ragged", "aniso_16"])
@pytest.mark.parametrize("lookahead", [1, -1])
def test_one_persistent_launch_per_level(name, lookahead, prec, tol):
    """The per-level persistent kernel (fused plan, a launch-plan setting for
    FP64 / FP32 RLB): POTRF, TRSM, products, small tasks and device loops of a level, and
    the previous level's lookahead products, in one launch ordered by device
    counters. L against the oracle's, the same as the per-class launches
    (fused = -1), and at most one launch per level plus the value load, the
    tail launch and (FP32) the inverses."""
    # diff7_24s: the 7-point 24^3 matrix with a diagonal shift of 1e-2, so that an
    # FP32 factor is comparable with the FP64 oracle's at the FP32 bound
    A = inputs.diffusion_3d_7pt(24, 24, 24, seed=7, shift=1e-2) if name == "diff7_24s" else _grid_case(name)
    kw = dict(ordering="grid_nd", grid=A.grid, merge=0.125)
    sym = sc.Symbolic(A, tune=dict(lookahead=lookahead, fused=1), **kw)
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True, merge=0.125)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    _check_L(num.export_L(), Lo, tol)
    levels = sym.plan_stats(prec)["levels"]
    assert num.info.kernel_launches <= levels + 4, (num.info.kernel_launches, levels)
    sym2 = sc.Symbolic(A, tune=dict(lookahead=lookahead, fused=-1), **kw)
    num2 = sym2.factor(A.values, precision=prec)
    assert num2.rc == 0
    assert num2.info.kernel_launches > num.info.kernel_launches
    _check_L(num2.export_L(), Lo, tol)
    B = inputs.rhs(A.n, 2, 5)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14, info


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_per_level_kernel_wait_times_out_and_handle_recovers(prec):
    """A chunk whose POTRF / TRSM count target is raised by one (test hook):
    the units that read it give up after spin_limit polls, the factorization
    returns SC_ERR_TIMEOUT, and the same handle then factors correctly."""
    A = _grid_case("diff7_13")
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, spin_limit=1 << 16, tune=dict(fused=1))
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    L0 = num.export_L()
    nchunks = sym.plan_stats(prec)["chunks"]
    for chunk in (0, nchunks // 2, nchunks - 2):
        num.stall_next_factor(chunk)
        with pytest.raises(sc.SCError) as e:
            num.refactor(A.values)
        assert e.value.code == sc.SC_ERR_TIMEOUT
        num.refactor(A.values)
        assert np.abs(num.export_L() - L0).max() <= 1e-5 * np.abs(L0).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-3), ("tf32x3", 1e-3)])
@pytest.mark.parametrize("name,chunk", [("diff7_24s", 64), ("st27_14", 64), ("lap2d_ragged", 64),
                                        ("st27_14", 40)])
def test_deterministic_factor_is_bitwise_reproducible(name, chunk, prec, tol):
    """Deterministic plans (RL, no inner-dimension splitting, target-owned
    assembly in source order): three factorizations of the same values give
    the same bits, and L agrees with the oracle's at the usual bound. The same
    matrix has split tiles and unordered assembly without the option."""
    A = inputs.diffusion_3d_7pt(24, 24, 24, seed=7, shift=1e-2) if name == "diff7_24s" else _grid_case(name)
    kw = dict(ordering="grid_nd", grid=A.grid, merge=0.125, variant="rl", chunk=chunk)
    sym = sc.Symbolic(A, deterministic=True, **kw)
    st = sym.plan_stats(prec)
    assert st["split_tiles"] == 0 and st["rl_slabs"] > 0
    base = sc.Symbolic(A, **kw).plan_stats(prec)
    assert base["rl_slabs"] == 0 and base["rl_pairs"] == st["rl_pairs"]
    Ls = []
    for _ in range(3):
        num = sym.factor(A.values, precision=prec)
        assert num.rc == 0
        Ls.append(num.export_L())
        last = num
    for L in Ls[1:]:
        assert np.array_equal(L.view(np.uint64), Ls[0].view(np.uint64))
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True, merge=0.125)
    assert o.factor() == 0
    _check_L(Ls[0], o.L_supernodal(), tol)
    B = inputs.rhs(A.n, 2, 21)
    X, info = last.solve(B)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14
