"""The allocation-free residual / backward-error entry point (needs a GB300).

sc_residual_eta_noalloc is for callers that cannot let a library allocate
device memory during a call (applications that give all device memory to their
own pool up front, or latency-critical loops where a cudaMalloc, which can
synchronise the whole device, is not acceptable). Its only working memory is a
fixed array built into the library.

The test calls it through the C ABI and checks it against the backward error
that sc_solve reports for the same solution, on consecutive calls: the first
two calls on the solution, then a call on a perturbed iterate (larger residual,
checked against numpy), then the solution again -- which must not see anything
left over in the shared array from the previous call. Further calls must leave
the device's free memory and torch's allocations unchanged; a NaN in X gives a
NaN eta for its column; R may be B itself.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2409_13090_gb300 as sc
from paper_2409_13090_gb300 import inputs

pytestmark = pytest.mark.gpu


def _full_csr(A):
    """Full symmetric CSR of the lower-triangle CSC input, columns ascending in each row."""
    rows = np.repeat(np.arange(A.n), np.diff(A.colptr))  # column index of each stored entry
    i, j, v = A.rowind.astype(np.int64), rows.astype(np.int64), A.values
    off = i != j
    r = np.concatenate([i, j[off]])
    c = np.concatenate([j, i[off]])
    vv = np.concatenate([v, v[off]])
    order = np.lexsort((c, r))
    r, c, vv = r[order], c[order], vv[order]
    ptr = np.zeros(A.n + 1, np.int64)
    np.add.at(ptr, r + 1, 1)
    return np.cumsum(ptr), c.astype(np.int32), vv


def _fn():
    f = sc.lib().sc_residual_eta_noalloc
    P = C.c_void_p
    f.argtypes = [C.c_int64, P, P, P, C.c_int64, P, C.c_int64, P, C.c_int64, P, C.c_int64, P, P]
    f.restype = C.c_int
    return f


def test_noalloc_residual_eta_matches_solve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc.build()
    A = inputs.diffusion_3d_7pt(11, 10, 9, seed=21, shift=1e-2)
    nrhs = 3
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid)
    num = sym.factor(A.values, precision="fp64")
    B = inputs.rhs(A.n, nrhs, 5)
    X, info = num.solve(B)
    eta_solve = info["eta"]

    ptr, col, val = _full_csr(A)
    dev = torch.device("cuda")
    d_ptr = torch.tensor(ptr, device=dev)
    d_col = torch.tensor(col, device=dev)
    d_val = torch.tensor(val, device=dev)
    d_B = torch.tensor(np.ascontiguousarray(B.T), device=dev)  # (nrhs, n) = column-major n x nrhs
    d_R = torch.empty_like(d_B)
    d_eta = torch.empty(nrhs, dtype=torch.float64, device=dev)
    f = _fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = A.n

    def call(Xh):
        d_X = torch.tensor(np.ascontiguousarray(Xh.T), device=dev)
        rc = f(n, d_ptr.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), nrhs, d_B.data_ptr(), n,
               d_X.data_ptr(), n, d_R.data_ptr(), n, d_eta.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        return d_eta.cpu().numpy().copy(), d_R.cpu().numpy().T.copy()

    def reference(Xh):
        Ad = inputs.dense_from_lower(A)
        R = B - Ad @ Xh
        an = np.abs(Ad).sum(axis=1).max()
        eta = np.abs(R).max(axis=0) / (an * np.abs(Xh).max(axis=0) + np.abs(B).max(axis=0))
        return eta, R, an

    for _ in range(2):  # two calls in a row on the solution
        eta, R = call(X)
        assert np.allclose(eta, eta_solve, rtol=1e-12, atol=0.0), (eta, eta_solve)
        _, Rref, an = reference(X)
        assert np.abs(R - Rref).max() <= 1e-13 * (an * np.abs(X).max() + np.abs(B).max())

    X2 = X + 0.01  # a perturbed iterate: large residual
    eta2, R2 = call(X2)
    eta2_ref, R2_ref, an = reference(X2)
    assert np.allclose(eta2, eta2_ref, rtol=1e-12), (eta2, eta2_ref)
    assert np.abs(R2 - R2_ref).max() <= 1e-13 * (an * np.abs(X2).max() + np.abs(B).max())

    eta3, _ = call(X)  # nothing left over from the previous call
    assert np.allclose(eta3, eta_solve, rtol=1e-12, atol=0.0)

    # the property the entry point exists for: after the calls above, further
    # calls change neither the device's free memory nor torch's allocations
    d_X = torch.tensor(np.ascontiguousarray(X.T), device=dev)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        rc = f(n, d_ptr.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), nrhs, d_B.data_ptr(), n, d_X.data_ptr(), n,
               d_R.data_ptr(), n, d_eta.data_ptr(), stream)
        assert rc == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0

    # a NaN in one column of X: that column's eta is NaN (never "converged"),
    # the other columns keep their values
    Xn = X.copy()
    Xn[n // 2, 1] = np.nan
    eta_n, _ = call(Xn)
    assert np.isnan(eta_n[1]), eta_n
    assert np.allclose(eta_n[[0, 2]], eta_solve[[0, 2]], rtol=1e-12, atol=0.0)
    eta4, _ = call(X)  # and the next call is clean again
    assert np.allclose(eta4, eta_solve, rtol=1e-12, atol=0.0)

    # R may be B itself
    d_B2 = d_B.clone()
    rc = f(n, d_ptr.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), nrhs, d_B2.data_ptr(), n, d_X.data_ptr(), n,
           d_B2.data_ptr(), n, d_eta.data_ptr(), stream)
    assert rc == 0
    torch.cuda.synchronize()
    _, Rref, an = reference(X)
    assert np.abs(d_B2.cpu().numpy().T - Rref).max() <= 1e-13 * (an * np.abs(X).max() + np.abs(B).max())
    assert np.allclose(d_eta.cpu().numpy(), eta_solve, rtol=1e-12, atol=0.0)


def test_noalloc_rejects_too_many_right_hand_sides():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc.build()
    f = _fn()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    for bad in (0, 1025):
        rc = f(4, p, p, p, bad, p, 4, p, 4, p, 4, p, None)
        assert rc == -5
