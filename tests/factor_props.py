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


def llt_probe_device(A, view, dview, nprobe=1, seed=0, group_entries=1 << 27) -> float:
    """llt_probe on the GPU, for factors too large to copy to the host: the
    factor is read in place through the library's device view (dview =
    Numeric.device_view(); panel J is row-major m_J x ld_J at panel_off[J],
    row r = glbind(J)[r], column f_J + c, entries with c > r not part of L)
    with torch gather / index_add in FP64 -- no kernel of the library runs.
    P A P^T x is formed on the host (scipy, FP64)."""
    import torch
    n = A.n
    dev = dview["lnz"].device
    perm, sup, gl, glb = view["perm"], view["sup_ptr"], view["gl_ptr"], view["glbind"]
    lower = sp.csc_matrix((A.values, A.rowind, A.colptr), shape=(n, n))
    full = (lower + lower.T - sp.diags(lower.diagonal())).tocsr()
    anorm = float(abs(full).sum(axis=1).max())
    ns = len(sup) - 1
    w = (sup[1:] - sup[:-1]).astype(np.int64)
    m = (gl[1:] - gl[:-1]).astype(np.int64)
    cnt = m * w
    # groups of consecutive supernodes with at most group_entries entries (one supernode may exceed it)
    bounds = [0]
    acc = 0
    for J in range(ns):
        if acc and acc + cnt[J] > group_entries:
            bounds.append(J)
            acc = 0
        acc += cnt[J]
    bounds.append(ns)
    glb_d = torch.as_tensor(glb.astype(np.int64), device=dev)
    lnz = dview["lnz"]

    def entries(J0, J1):
        """(storage offset, global row, global column) of every L entry of supernodes J0..J1-1."""
        cj = torch.as_tensor(cnt[J0:J1], device=dev)
        sn = torch.repeat_interleave(torch.arange(J0, J1, device=dev), cj)
        start = torch.cumsum(cj, 0) - cj
        e = torch.arange(int(cj.sum()), device=dev) - torch.repeat_interleave(start, cj)
        wj = torch.as_tensor(w, device=dev)[sn]
        r, c = e // wj, e % wj
        keep = c <= r
        sn, r, c = sn[keep], r[keep], c[keep]
        off = torch.as_tensor(dview["panel_off"], device=dev)[sn] + r * torch.as_tensor(
            dview["panel_ld"].astype(np.int64), device=dev)[sn] + c
        grow = glb_d[torch.as_tensor(gl[:-1], device=dev)[sn] + r]
        gcol = torch.as_tensor(sup[:-1].astype(np.int64), device=dev)[sn] + c
        return off, grow, gcol

    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(nprobe):
        xh = rng.uniform(-1.0, 1.0, n)
        xo = np.empty(n)
        xo[perm] = xh
        ah = (full @ xo)[perm]
        x = torch.as_tensor(xh, device=dev)
        y = torch.zeros(n, dtype=torch.float64, device=dev)
        for g in range(len(bounds) - 1):  # y = L^T x
            off, grow, gcol = entries(bounds[g], bounds[g + 1])
            y.index_add_(0, gcol, lnz[off].double() * x[grow])
        z = torch.zeros(n, dtype=torch.float64, device=dev)
        for g in range(len(bounds) - 1):  # z = L y
            off, grow, gcol = entries(bounds[g], bounds[g + 1])
            z.index_add_(0, grow, lnz[off].double() * y[gcol])
        zh = z.cpu().numpy()
        worst = max(worst, float(np.abs(ah - zh).max()) / (anorm * float(np.abs(xh).max())))
    return worst
