"""Solve sweeps on the GPU (needs a GB300): the bounded waits of the persistent
forward / backward sweeps.

Each sweep is one launch whose CTAs wait on per-chunk counters. Every wait is
bounded: after spin_limit polls it sets an error word, every other wait sees
the word and stops, and sc_solve returns SC_ERR_TIMEOUT. The test makes one
chunk expect an arrival that never comes (sc_test_stall_solve), checks the
status, and then checks that the same handle solves correctly again, i.e. the
CUDA context survived and the expected count was restored.
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("where", ["root", "leaf"])
def test_stalled_chunk_times_out_and_handle_recovers(prec, where):
    A = inputs.diffusion_3d_7pt(13, 11, 9, seed=5, shift=1e-2)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, spin_limit=1 << 16)
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    B = inputs.rhs(A.n, 3, 11)
    X0, info0 = num.solve(B)
    assert oracle.backward_error(A, B, X0).max() <= 1e-14
    nchunks = sym.plan_stats(prec)["chunks"]
    num.stall_next_solve(nchunks - 1 if where == "root" else 0)
    with pytest.raises(sc.SCError) as e:
        num.solve(B)
    assert e.value.code == sc.SC_ERR_TIMEOUT
    X1, info1 = num.solve(B)
    assert oracle.backward_error(A, B, X1).max() <= 1e-14
    assert np.abs(X1 - X0).max() <= 1e-10 * np.abs(X0).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nrhs", [1, 5, 12, 33, 64, 70, 130])
def test_many_right_hand_sides(prec, nrhs):
    """Blocks of up to 64 right-hand sides, one sweep unit covering a whole
    block: 1..4, 5..8, 9..16, 17..32 and 33..64 right-hand sides per block take
    the five register-blocking variants; 70 and 130 make two and three blocks
    (the last one ragged: 6 and 2), each with freshly zeroed counters; counts
    that are not multiples of 4 take the scalar atomic adds. X is compared
    with the oracle's solve and eta <= 1e-14 (FP32: after refinement; the
    7-point matrix with a diagonal shift of 1e-2, whose condition number lets
    classical refinement of an FP32 factor converge)."""
    A = inputs.diffusion_3d_7pt(12, 12, 12, seed=12, shift=1e-2)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    B = inputs.rhs(A.n, nrhs, 12)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14, info
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True)
    assert o.factor() == 0
    Xo = o.solve(B)
    assert np.abs(X - Xo).max() <= 1e-8 * np.abs(Xo).max()


@pytest.mark.parametrize("prec", ["fp32", "tf32", "tf32x3"])
def test_cg_with_low_precision_factor_reaches_fp64_backward_error(prec):
    """The 7-point variable-coefficient matrix (diagonal = row sum + 1e-6, so
    kappa is large) at 24^3: conjugate gradients preconditioned by the
    low-precision factor reaches eta <= 1e-14 (checked with the oracle's eta)."""
    A = inputs.workload(2, 0.5)[0]
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=0.125)
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    B = inputs.rhs(A.n, 4, 13)
    X, info = num.solve(B, method="cg", max_iterations=400)
    assert info["converged"], info
    assert oracle.backward_error(A, B, X).max() <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("group", [1, 3, 7, 16])
def test_solve_group_sizes(prec, group):
    """Runs of 1, 3, 7 and 16 row tiles per sweep unit (the solve_group
    setting; 4 by default): the same solution as the oracle's, ragged last
    runs included, for 5 right-hand sides."""
    A = inputs.diffusion_3d_7pt(14, 12, 10, seed=21, shift=1e-2)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, tune=dict(solve_group=group))
    num = sym.factor(A.values, precision=prec)
    assert num.rc == 0
    B = inputs.rhs(A.n, 5, 22)
    X, info = num.solve(B)
    assert oracle.backward_error(A, B, X).max() <= 1e-14, info
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True)
    assert o.factor() == 0
    Xo = o.solve(B)
    assert np.abs(X - Xo).max() <= 1e-8 * np.abs(Xo).max()


@pytest.mark.parametrize("where", ["pinned", "cuda"])
@pytest.mark.parametrize("pad", [0, 7])
def test_padded_and_contiguous_buffers(where, pad):
    """B and X as (nrhs, n + pad) torch tensors in pinned host memory or on the
    device: contiguous columns (pad 0) move in one copy each way, padded ones
    column by column. Same solution as the numpy path, padding left untouched,
    and the reported copy times are parts of the solve time."""
    torch = pytest.importorskip("torch")
    A = inputs.diffusion_3d_7pt(11, 10, 9, seed=31, shift=1e-2)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    num = sym.factor(A.values, precision="fp64")
    assert num.rc == 0
    nrhs = 6
    B = inputs.rhs(A.n, nrhs, 32)
    Xref, _ = num.solve(B)
    Bt = torch.full((nrhs, A.n + pad), 7.0, dtype=torch.float64)
    Bt[:, :A.n] = torch.from_numpy(np.ascontiguousarray(B.T))
    Xt = torch.full_like(Bt, -3.0)
    if where == "pinned":
        Bt, Xt = Bt.pin_memory(), Xt.pin_memory()
    else:
        Bt, Xt = Bt.cuda(), Xt.cuda()
    _, info = num.solve(Bt, Xt)
    torch.cuda.synchronize()
    X = Xt.cpu().numpy()
    # the sweeps add updates atomically, so the order of additions may differ
    assert np.abs(X[:, :A.n].T - Xref).max() <= 1e-12 * np.abs(Xref).max()
    assert (X[:, A.n:] == -3.0).all()
    assert 0.0 <= info["copy_in_ms"] <= info["solve_ms"]
    assert 0.0 <= info["copy_out_ms"] <= info["solve_ms"]
