"""TF32 tensor-core (tcgen05) product tiles against the oracle (needs a GB300).

Cases are chosen so that the launch plan routes products to the tensor-core
kernel (asserted through sc_plan_stats): a dense matrix (one wide supernode,
trailing updates with K = 64 across many chunks) and 3D stencils whose
separators are wide (cross-supernode updates with K = |J| >= 32). The factor
is compared with the oracle's FP64 L within the TF32 bound used for the other
low-precision tests, and refinement must reach eta <= 1e-14.
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


def _dense(n, seed):
    rng = np.random.default_rng(seed)
    ents = [(i, j) for j in range(n) for i in range(j + 1, n)]
    A = inputs.from_lower_pattern(n, ents, seed=seed)
    A.values[:] = np.where(A.rowind == np.repeat(np.arange(n), np.diff(A.colptr)), A.values, rng.uniform(-1, 1, A.nnz))
    # diagonal dominance for a well-conditioned SPD matrix
    rows = np.repeat(np.arange(n), np.diff(A.colptr))
    off = A.rowind != rows
    s = np.zeros(n)
    np.add.at(s, A.rowind[off], np.abs(A.values[off]))
    np.add.at(s, rows[off], np.abs(A.values[off]))
    A.values[~off] = s + 1.0
    return A


@pytest.mark.parametrize("case", ["dense_700", "st27_16", "diff7_20"])
def test_tf32_tensor_core_tiles_match_oracle(case):
    if case == "dense_700":
        A, perm0, kw = _dense(700, 1), None, dict(ordering="natural")
    elif case == "st27_16":
        A = inputs.stencil_3d_27pt(16, 16, 16, seed=3)
        perm0, kw = oracle.nd_grid(16, 16, 16, 8), dict(ordering="grid_nd", grid=A.grid)
    else:
        A = inputs.diffusion_3d_7pt(20, 20, 20, seed=4, shift=1e-1)
        perm0, kw = oracle.nd_grid(20, 20, 20, 8), dict(ordering="grid_nd", grid=A.grid)
    sym = sc.Symbolic(A, **kw)
    assert sym.plan_stats("tf32")["tc_tiles"] > 0
    o = oracle.Oracle(A, perm0, pr=True)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    num = sym.factor(A.values, precision="tf32")
    assert num.rc == 0
    Lg = num.export_L()
    err = np.abs(Lg - Lo).max() / np.abs(Lo).max()
    assert err <= 2e-2, err
    # the same handle in FP32 SIMT agrees with TF32 to TF32 accuracy
    num32 = sym.factor(A.values, precision="fp32")
    assert np.abs(num32.export_L() - Lg).max() / np.abs(Lo).max() <= 2e-2
    B = inputs.rhs(A.n, 2, 7)
    X, info = num.solve(B)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("case", ["dense_700", "st27_16"])
def test_tf32x3_split_products_reach_fp32_accuracy(case):
    """The three-product split form (x = hi + lo, hi*hi' + hi*lo' + lo*hi') on the
    tensor cores: L within the FP32 bound of the oracle's FP64 L and as close
    to it as the FP32 SIMT factor (within 2x), or 16x closer than the plain
    TF32 factor where TF32 rounding of the products dominates; refinement to
    eta <= 1e-14 in no more steps than the plain TF32 factor."""
    if case == "dense_700":
        A, perm0, kw = _dense(700, 1), None, dict(ordering="natural")
    else:
        A = inputs.stencil_3d_27pt(16, 16, 16, seed=3)
        perm0, kw = oracle.nd_grid(16, 16, 16, 8), dict(ordering="grid_nd", grid=A.grid)
    sym = sc.Symbolic(A, **kw)
    assert sym.plan_stats("tf32x3")["tc_tiles"] > 0
    o = oracle.Oracle(A, perm0, pr=True)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    scale = np.abs(Lo).max()
    errs = {}
    nums = {}
    for prec in ("tf32", "tf32x3", "fp32"):
        nums[prec] = sym.factor(A.values, precision=prec)
        assert nums[prec].rc == 0
        errs[prec] = np.abs(nums[prec].export_L() - Lo).max() / scale
    assert errs["tf32x3"] <= 1e-3, errs
    assert errs["tf32x3"] <= max(2 * errs["fp32"], errs["tf32"] / 16), errs
    B = inputs.rhs(A.n, 2, 7)
    its = {}
    for prec in ("tf32", "tf32x3"):
        X, info = nums[prec].solve(B)
        assert info["converged"], info
        assert oracle.backward_error(A, B, X).max() <= 1e-14
        its[prec] = info["iterations"]
    assert its["tf32x3"] <= its["tf32"], its


@pytest.mark.parametrize("prec,tol", [("tf32", 2e-2), ("tf32x3", 1e-3)])
@pytest.mark.parametrize("chunk", [24, 36, 40, 48])
@pytest.mark.parametrize("case", ["dense_700", "st27_16"])
def test_tensor_core_tiles_at_chunk_widths_with_a_k_tail(case, chunk, prec, tol):
    """Chunk widths other than 32 and 64: the in-panel updates have K = chunk
    (40, 48: whole 8-column MMA steps but not whole 32-column boxes; 36: not a
    whole step, kept on the SIMT units unless the product ends at the panel's
    last column) and macro panels of 240 or 252 columns. The tensor-core tile
    must multiply exactly K columns: L is compared with the oracle's FP64 L
    element by element and refinement must reach eta <= 1e-14."""
    if case == "dense_700":
        A, perm0, kw = _dense(700, 1), None, dict(ordering="natural")
    else:
        A = inputs.stencil_3d_27pt(16, 16, 16, seed=3)
        perm0, kw = oracle.nd_grid(16, 16, 16, 8), dict(ordering="grid_nd", grid=A.grid)
    sym = sc.Symbolic(A, chunk=chunk, **kw)
    assert sym.check_schedule()["ok"]
    # the dense matrix is one supernode: with chunk 36 every in-panel update
    # (K = 36, or 252 for a macro panel) ends before the panel's last column,
    # so none goes to the tensor cores; every other case has tensor-core tiles
    if not (case == "dense_700" and chunk == 36):
        assert sym.plan_stats(prec)["tc_tiles"] > 0
    o = oracle.Oracle(A, perm0, pr=True)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    err = np.abs(num.export_L() - Lo).max() / np.abs(Lo).max()
    assert err <= tol, err
    B = inputs.rhs(A.n, 2, 7)
    X, info = num.solve(B)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32", 2e-2), ("tf32x3", 1e-3)])
@pytest.mark.parametrize("defer", [512, 1024])
def test_deeper_trailing_update_deferral(defer, prec, tol):
    """Outer deferral blocks of 512 and 1024 columns inside a 1300-column
    supernode (a dense matrix): in-panel products with K = 256 and K = the
    outer width, some of them critical (split along K in FP64), against the
    oracle's L element by element and refinement to eta <= 1e-14."""
    A = _dense(1300, 2)
    sym = sc.Symbolic(A, ordering="natural", tune=dict(defer_width=defer))
    assert sym.check_schedule()["ok"]
    o = oracle.Oracle(A, None, pr=True)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    err = np.abs(num.export_L() - Lo).max() / np.abs(Lo).max()
    assert err <= tol, err
    B = inputs.rhs(A.n, 2, 9)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("prec,tol", [("tf32", 2e-2), ("tf32x3", 1e-3)])
@pytest.mark.parametrize("case", ["dense_1300", "dense_700_c40", "st27_24"])
def test_256_column_tensor_core_tiles(case, prec, tol):
    """Products at least 256 columns wide on 128 x 256 tensor-core tiles (the
    B tile loaded as two 128-row boxes, both TMEM accumulators 256 columns):
    L against the oracle's element by element with the 256-column tiles in
    clusters of two sharing B by multicast (the default, pairs completed by
    tiles that write nothing), one CTA per tile, and off (every such product
    on 128-column tiles); ragged widths and lower products that cross the
    diagonal included; refinement reaches eta <= 1e-14."""
    if case.startswith("dense"):
        n = 1300 if case == "dense_1300" else 700
        A, perm0, kw = _dense(n, 3), None, dict(ordering="natural", chunk=40 if case.endswith("c40") else 64)
    else:
        A = inputs.stencil_3d_27pt(24, 24, 24, seed=4, dominance=1.05)
        perm0, kw = oracle.nd_grid(24, 24, 24, 8), dict(ordering="grid_nd", grid=A.grid)
    o = oracle.Oracle(A, perm0, pr=True)
    assert o.factor() == 0
    Lo = o.L_supernodal()
    for wide, mc in ((0, 0), (0, -1), (1 << 20, 0)):
        # the two-level deferral (outer width 256): the macro panels' last chunks update
        # every later column at once, so the 700-column case has products >= 256 wide too
        tune = {k: v for k, v in (("tc_wide256", wide), ("tc_multicast", mc), ("defer_width", 256)) if v}
        sym = sc.Symbolic(A, tune=tune, **kw)
        st = sym.plan_stats(prec)
        assert (st["tc256_tiles"] > 0) == (wide == 0), st
        num = sym.factor(A.values, precision=prec)
        assert num.rc == 0
        err = np.abs(num.export_L() - Lo).max() / np.abs(Lo).max()
        assert err <= tol, (wide, mc, err)
        B = inputs.rhs(A.n, 2, 13)
        X, info = num.solve(B)
        assert info["converged"], info
        assert oracle.backward_error(A, B, X).max() <= 1e-14
