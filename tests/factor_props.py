"""Properties of a computed factor that hold at any size (test helper).

For sizes where the oracle cannot factor in seconds, the tests check the GPU
factor by what defines it: L L^T = P A P^T. `llt_probe` measures that on random
probe vectors without forming either product: with x in the final ordering,
||P A P^T x - L (L^T x)||_inf / (||A||_inf ||x||_inf).
"""
import numpy as np
import scipy.sparse as sp


def llt_probe(A, view, L, nprobe=2, seed=0) -> float:
    """L is in the canonical supernodal layout (sc_numeric_export_L, the
    oracle's L_supernodal): per supernode J an m_J x |J| row-major block whose
    row r is glbind(J)[r]; view is the symbolic view that gave the layout."""
    n = A.n
    perm, sup, gl, glb = view["perm"], view["sup_ptr"], view["gl_ptr"], view["glbind"]
    lower = sp.csc_matrix((A.values, A.rowind, A.colptr), shape=(n, n))
    full = (lower + lower.T - sp.diags(lower.diagonal())).tocsr()
    anorm = float(abs(full).sum(axis=1).max())
    ns = len(sup) - 1
    offs = np.zeros(ns + 1, np.int64)
    offs[1:] = np.cumsum((gl[1:] - gl[:-1]) * (sup[1:] - sup[:-1]))
    assert offs[-1] == L.size
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(nprobe):
        xh = rng.uniform(-1.0, 1.0, n)
        xo = np.empty(n)
        xo[perm] = xh
        ah = (full @ xo)[perm]
        y = np.empty(n)
        for J in range(ns):
            w = sup[J + 1] - sup[J]
            blk = L[offs[J]:offs[J + 1]].reshape(-1, w)
            y[sup[J]:sup[J + 1]] = blk.T @ xh[glb[gl[J]:gl[J + 1]]]
        z = np.zeros(n)
        for J in range(ns):
            w = sup[J + 1] - sup[J]
            blk = L[offs[J]:offs[J + 1]].reshape(-1, w)
            z[glb[gl[J]:gl[J + 1]]] += blk @ y[sup[J]:sup[J + 1]]
        worst = max(worst, float(np.abs(ah - z).max()) / (anorm * float(np.abs(xh).max())))
    return worst
