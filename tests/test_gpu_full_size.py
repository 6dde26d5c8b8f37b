"""Full-size benchmark matrices through the C ABI, checked by properties that
hold at any size (needs a GB300).

The oracle cannot factor these in seconds, so the factor is checked by what
defines it, L L^T = P A P^T, on random probe vectors (tests/factor_props.py,
pinned on the oracle's factor in test_oracle.py), and the solve by the
backward error the oracle computes in FP64 on the CPU (for the anisotropic
128^3 matrix, whose factor holds 3.2e9 entries, the probe reads the factor in
place on the GPU with torch; no kernel of the library is involved in the
check). Launch configuration
as the benchmark times it: grid ND (leaf 8), PR, supernode merging 0.125, RLB,
CUDA graph replay.

Bars: probe residual <= 1e-12 (FP64), 1e-4 (FP32, TF32x3: unit roundoff 2^-24
products), 1e-2 (TF32: 2^-11 rounding of every product operand); eta <= 1e-14
after the solve (refined for the low-precision factors).
"""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import paper_2409_13090_gb300 as sc
from paper_2409_13090_gb300 import inputs
from tests.factor_props import llt_probe, llt_probe_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc.build()
    oracle.build()


def test_full_stencil27_80_factor_and_solve():
    """80^3 27-point stencil (n = 512,000), 16 right-hand sides: TF32 and
    TF32x3 factors with FP64 refinement, and the FP64 factor."""
    A, nrhs = inputs.workload(3)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb", merge=0.125)
    view = sym.view()
    B = inputs.rhs(A.n, nrhs, inputs.SEED_BASE + 3)
    for prec, bound in (("tf32", 1e-2), ("tf32x3", 1e-4), ("fp64", 1e-12)):
        num = sym.factor(A.values, precision=prec)
        assert num.rc == 0, prec
        L = num.export_L()
        r = llt_probe(A, view, L, nprobe=1)
        del L
        assert r <= bound, (prec, r)
        X, info = num.solve(B)
        eta = oracle.backward_error(A, B, X).max()
        assert eta <= 1e-14, (prec, eta, info)
        num.free()


def test_full_batch_of_256_laplacians():
    """The 256 2D Laplacians of uneven size (n = 6.0 M in total), one batched
    FP32 factorization and refined solve: the probe on the block-diagonal
    matrix and the backward error of every matrix."""
    mats, nrhs = inputs.workload(4)
    syms = [sc.Symbolic(M, ordering="grid_nd", grid=M.grid, merge=0.125) for M in mats]
    bsym = sc.Symbolic.batch(syms)
    vals = np.concatenate([M.values for M in mats])
    num = bsym.factor(vals, precision="fp32")
    assert num.rc == 0
    colptr, rowind, off, nnz = [np.zeros(1, np.int64)], [], 0, 0
    for M in mats:
        colptr.append(np.asarray(M.colptr[1:], np.int64) + nnz)
        rowind.append(np.asarray(M.rowind, np.int64) + off)
        off += M.n
        nnz += M.nnz
    Ab = SimpleNamespace(n=off, colptr=np.concatenate(colptr), rowind=np.concatenate(rowind), values=vals)
    r = llt_probe(Ab, bsym.view(), num.export_L(), nprobe=1)
    assert r <= 1e-4, r
    B = inputs.rhs(off, nrhs, inputs.SEED_BASE + 4)
    X, info = num.solve(B)
    assert info["converged"], info
    row = 0
    worst = 0.0
    for M in mats:
        worst = max(worst, float(oracle.backward_error(M, B[row:row + M.n], X[row:row + M.n]).max()))
        row += M.n
    assert worst <= 1e-14, worst


def test_full_anisotropic_128_factor_and_solve():
    """The anisotropic 7-point matrix on the full 128^3 grid (n = 2,097,152,
    shift 1e-8, condition number near 1e11), 64 right-hand sides, in the
    benchmark's launch configuration: the TF32x3 factor with conjugate
    gradients preconditioned by it, and the FP64 factor with a plain solve.
    The factor is probed in place on the GPU (L L^T = P A P^T), the solution
    by the oracle's FP64 backward error of every right-hand side."""
    A, nrhs = inputs.workload(5)
    assert A.n == 128 ** 3 and nrhs == 64
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb", merge=0.125)
    view = sym.view()
    B = inputs.rhs(A.n, nrhs, inputs.SEED_BASE + 5)
    for prec, bound in (("tf32x3", 1e-4), ("fp64", 1e-12)):
        num = sym.factor(A.values, precision=prec)
        assert num.rc == 0, prec
        r = llt_probe_device(A, view, num.device_view(), nprobe=1)
        assert r <= bound, (prec, r)
        if prec == "fp64":
            X, info = num.solve(B)
        else:
            X, info = num.solve(B, method="cg", max_iterations=1000)
            assert info["converged"], info
        eta = oracle.backward_error(A, B, X).max()
        assert eta <= 1e-14, (prec, eta, info)
        num.free()
