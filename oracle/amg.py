"""Aggregation AMG V-cycle and flexible CG for inverse iteration (paper §7).

TEST INFRASTRUCTURE (as the rest of ``oracle/``).

§7, Algorithm 3 and the text after it:
  * the hierarchy aggregates pairs of consecutive rows (the paper bootstraps the
    pairs from an RCB ordering of the elements; here the pairs follow the row
    order of the graph given, which is RCB order when the elements were
    reordered by RCB): J_i^{i+1} is the Boolean restriction that sums rows 2I
    and 2I + 1 into coarse row I (a last odd row stands alone), and
    L_{i+1} = J_i^{i+1} L_i J_{i+1}^i, which is again a Laplacian;
  * the V-cycle with damping sigma and n_smooth smoothing steps, D = 1 / diag(L):
    u = sigma D r, r = r - L u; n_smooth steps u += sigma D r, r -= L sigma D r;
    coarse correction u += J^T V-cycle(J r) with r updated by it; n_smooth more
    smoothing steps.
  * flexible CG whose first search direction is not preconditioned (§7), so
    that a right-hand side that is already an eigenvector returns after one
    iteration.
Readings (the text is garbled or silent): the printed recursion passes level i
instead of i + 1 and has no coarsest level: the recursion goes to level i + 1
and stops at a 1 x 1 level, whose Laplacian is 0 on a connected graph (the
correction there is 0); the post-smoothing's "r = r - L u" is read as keeping r
the residual of the current u (u += sigma D r, r -= L sigma D r, as in the
pre-smoothing); sigma = 2/3 and n_smooth = 2 (not given); the flexible CG
takes the Polak-Ribiere beta = z_{k+1}.(r_{k+1} - r_k) / z_k.r_k; every
residual and preconditioned residual is projected against the fixed basis
(1 and the deflation vectors), as in the unpreconditioned CG.
"""
from __future__ import annotations

import numpy as np


def laplacian_csr(g):
    """L = D - A as a scipy CSR matrix (§4)."""
    import scipy.sparse as sp

    from .rsb_oracle import adjacency_csr, degree

    return (sp.diags(degree(g)) - adjacency_csr(g)).tocsr()


def amg_hierarchy(L):
    """[(L_0, None), (L_1, J_0), ...]: J_i is the n_i x n_{i+1} Boolean matrix of
    the pair aggregation (row a of level i belongs to coarse row a // 2)."""
    import scipy.sparse as sp

    levels = [(L.tocsr(), None)]
    while levels[-1][0].shape[0] > 1:
        Li = levels[-1][0]
        n = Li.shape[0]
        nc = (n + 1) // 2
        J = sp.csr_matrix((np.ones(n), (np.arange(n), np.arange(n) // 2)), shape=(n, nc))
        levels.append(((J.T @ Li @ J).tocsr(), J))
    return levels


def vcycle(levels, i: int, r: np.ndarray, sigma: float = 2.0 / 3.0, nsmooth: int = 2):
    """Algorithm 3 at level i (readings in the module docstring)."""
    L = levels[i][0]
    if L.shape[0] == 1:
        return np.zeros(1)
    d = L.diagonal()
    D = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    r = np.array(r, dtype=np.float64, copy=True)
    u = sigma * D * r
    r = r - L @ u
    for _ in range(nsmooth):
        du = sigma * D * r
        u = u + du
        r = r - L @ du
    J = levels[i + 1][1]
    ec = vcycle(levels, i + 1, J.T @ r, sigma, nsmooth)
    du = J @ ec
    u = u + du
    r = r - L @ du
    for _ in range(nsmooth):
        du = sigma * D * r
        u = u + du
        r = r - L @ du
    return u


def fcg_solve(g, b: np.ndarray, B: np.ndarray, opts, levels=None):
    """Flexible CG on L x = b from x0 = 0, first direction unpreconditioned,
    later ones preconditioned by one V-cycle; r and z projected against B."""
    from .rsb_oracle import _cgs, laplacian_apply

    if levels is None:
        levels = amg_hierarchy(laplacian_csr(g))
    x = np.zeros_like(b)
    r = b.copy()
    z = r.copy()
    p = z.copy()
    rz = float(r @ z)
    bnorm = float(np.linalg.norm(b))
    it = 0
    for it in range(1, opts.cg_maxit + 1):
        ap = laplacian_apply(g, p)
        a = rz / float(p @ ap)
        x = x + a * p
        rn = r - a * ap
        rn, _ = _cgs(B, rn)
        if np.linalg.norm(rn) <= opts.cg_tol * bnorm:
            break
        zn, _ = _cgs(B, vcycle(levels, 0, rn))
        beta = float(zn @ (rn - r)) / rz
        rz = float(rn @ zn)
        p = zn + beta * p
        r = rn
    return x, it


def amg_inverse_fiedler(g, opts, deflate=(), start=None):
    """Inverse iteration (§7, Algorithm 2) with the AMG-preconditioned flexible
    CG as the inner solver; stops as the unpreconditioned form does (residual,
    a solve that returned after one iteration, or max_outer)."""
    from .rsb_oracle import FiedlerResult, _fixed_basis, _project_start, degree, \
        laplacian_apply, start_vector

    n = g.n
    if n - 1 - len(deflate) <= 0:
        return None
    B = _fixed_basis(n, deflate)
    dmax = float(degree(g).max())
    levels = amg_hierarchy(laplacian_csr(g))
    b = start_vector(g.gid, opts.seed, len(deflate)) if start is None \
        else np.array(start, dtype=np.float64)
    lam, y, res, inner = 0.0, b, np.inf, 0
    for it in range(1, opts.max_outer + 1):
        b = _project_start(B, b)
        x, inner = fcg_solve(g, b, B, opts, levels)
        y = x / np.linalg.norm(x)
        ly = laplacian_apply(g, y)
        lam = float(y @ ly)
        res = float(np.linalg.norm(ly - lam * y))
        if res <= opts.tol * dmax or inner == 1:
            return FiedlerResult(lam, y, res, it, True, inner)
        b = y
    return FiedlerResult(lam, y, res, opts.max_outer, False, inner)
