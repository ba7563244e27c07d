"""Plain FP64 CPU oracle for Recursive Spectral Bisection (RSB).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or run this module.
The CUDA library never calls it and shares no code with it; the two meet only
in the seeded input generators of ``meshgen``.

What it computes (paper: Ratnayaka & Fischer, "parRSB: Exascale Spectral
Element Mesh Partitioning"):

* the weighted Laplacian L = D - A of the element dual graph (§4, Eq. for the
  weighted Laplacian; the diagonal is the row's weight sum over j != i — the
  printed index "i != j" under the sum is read as a typo) and its action on a
  vector (§5, assembled form);
* the Fiedler vector: the eigenvector of the smallest eigenvalue of L on the
  complement of the constant vector (§4, Eqs. eigen0/eigen1), by restarted
  Lanczos (§6) and by inverse iteration with CG (§7, Algorithm 2);
* Recursive Spectral Bisection (§4, Algorithm 1) with the floor/ceil split of
  the processor count and proportional element counts (§4, after Algorithm 1);
* the paper's partition-quality metrics (§8): neighbour counts per part, plus
  the edge cut of the spectral relaxation (§3).

Where the paper is silent the following readings are used (they bind the CUDA
path too):

R1  balance: part sizes differ by at most one (§2 prints "= 1").
R2  recursion acts on the induced subgraph of each half; degrees are
    recomputed from the surviving edges.
R3  Lanczos: Krylov length m = min(krylov_dim, n - 1 - #deflation vectors);
    each step takes w = L q_j and re-orthogonalises it fully by two classical
    Gram-Schmidt passes against [1/sqrt(n), deflation vectors, q_0..q_j]; the
    two passes' coefficients on q_0..q_j form column j of the projected matrix
    S = Q^T L Q (tridiagonal in the first cycle, arrow-plus-tridiagonal after
    a restart), beta_{j+1} = ||w||, q_{j+1} = w / beta_{j+1}.  At the end of a
    cycle the Ritz pairs of S give theta (smallest) and y = Q s_1; the cycle is
    thick-restarted (Wu & Simon, cited in §6): the `keep` smallest Ritz
    vectors and the last residual direction w / beta_m are the first keep + 1
    basis vectors of the next cycle, S restarts as diag(theta_1..theta_keep)
    and the next m - keep steps add its new columns.  Stop when
    ||L y - theta y|| <= tol * d_max (d_max = largest weighted degree, a lower
    bound of ||L||_2), at most max_restarts cycles; a cycle ends early when
    beta <= 1e-14 * d_max (invariant subspace; a cycle that ends that way and
    has not converged restarts from y alone).  Start vector:
    s_i = 2 * (SplitMix64(s_d XOR gid_i) >> 11) * 2^-53 - 1 with
    s_d = SplitMix64(seed + d) for a solve deflated against d vectors, then
    projected and normalised (two classical Gram-Schmidt passes against the
    fixed basis).  Each deflated solve needs a fresh start: deflating v_a from
    the very vector that produced it removes the whole cluster component, so
    the solve would never see the partner eigenvector (the effect §9 describes
    for single-vector iterations); and s_d must be fully mixed, because
    (seed + d) XOR gid for small d only permutes gids within a mesh row and
    keeps the other axes' mode components of the start vector.
    Inverse iteration: CG from x0 = 0 on L x = b with one classical projection
    of r against the fixed basis per step; CG stops at ||r|| <= cg_tol * ||b||;
    the outer loop stops when ||L y - lambda y|| <= tol * d_max, when CG
    returned after a single iteration (§7), or after max_outer iterations.
R4  orientation: g* = smallest gid with |v| >= max|v| / 2; v is negated if
    v[g*] > 0, so g* lands in the left (lower-numbered) half.
R5  repeated lambda_2 (§9): with the "resolve" policy the solver is rerun
    deflated against the vectors found so far while the new eigenvalue lies
    within cluster_tol * lambda_a of the first (cluster dimension <= 3); the
    cluster basis U is rotated by the orthogonal R minimising sum (U R)^4
    (closed form for two columns, cyclic pairwise sweeps for three); every
    rotated column is oriented and split, and the split with the least weighted
    cut wins; equal cuts go to the split whose left set holds the smallest gid
    of the two left sets' symmetric difference.
R6  split sizes: a segment [p0, p1) of a mesh with N elements and P parts holds
    floor(p1 N / P) - floor(p0 N / P) elements; its left child [p0, pm),
    pm = p0 + floor((p1 - p0) / 2), receives floor(pm N/P) - floor(p0 N/P).
R7  median split with ties: with k elements going left, v_k the k-th smallest
    value and tau = tie_rel * (max v - min v): every element with
    v < v_k - tau goes left, every element with |v - v_k| <= tau is a tie and
    the ties go left in ascending gid until k elements are left.
R8  disconnected halves: components are ordered by their smallest gid and
    placed left whole while they fit; the component that straddles the left
    count is split by its own Fiedler vector (R4-R7) with the remaining count;
    every later component goes right.
R9  tiny segments need no special case (n = 2 gives the lower gid left).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------
# options
# ----------------------------------------------------------------------------


@dataclass
class Options:
    method: str = "lanczos"          # "lanczos" | "inverse"
    krylov_dim: int = 40
    keep: int = 8                    # Ritz vectors kept by a thick restart
    max_restarts: int = 50           # §8: the paper's cap of 50 restarts
    tol: float = 1e-10
    cg_tol: float = 1e-12
    cg_maxit: int = 2000
    max_outer: int = 50
    seed: int = 0x5EED
    degenerate: str = "resolve"      # "none" | "resolve"
    cluster_tol: float = 0.05
    tie_rel: float = 1e-5
    breakdown: float = 1e-14
    block: int = 1                   # Lanczos block width (1: single-vector Lanczos)
    amg: bool = False                # inverse iteration: AMG-preconditioned flexible CG (§7)


@dataclass
class FiedlerResult:
    lam: float
    v: np.ndarray
    resid: float
    iters: int
    converged: bool
    inner: int = 0


# ----------------------------------------------------------------------------
# graph and Laplacian (§4, §5)
# ----------------------------------------------------------------------------


def rows_of(g) -> np.ndarray:
    """Row index of every stored entry (cached on the graph object)."""
    r = getattr(g, "_oracle_rows", None)
    if r is None or len(r) != len(g.col):
        r = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
        g._oracle_rows = r
    return r


def degree(g) -> np.ndarray:
    """d_i = sum_{j != i} w_ij (diagonal of the weighted Laplacian, §4)."""
    return np.bincount(rows_of(g), weights=g.w.astype(np.float64), minlength=g.n)


def adjacency_csr(g):
    """The weighted adjacency A as a scipy CSR matrix (cached on the graph)."""
    import scipy.sparse as sp

    a = getattr(g, "_oracle_A", None)
    if a is None or a.shape[0] != g.n or a.nnz != len(g.col):
        a = sp.csr_matrix((g.w.astype(np.float64), np.asarray(g.col, dtype=np.int64),
                           np.asarray(g.row_ptr, dtype=np.int64)), shape=(g.n, g.n))
        g._oracle_A = a
    return a


def laplacian_apply(g, x: np.ndarray) -> np.ndarray:
    """y = (D - A) x with the assembled (CSR) Laplacian (§5, first option); the
    product A x is the library's sparse matrix-vector product."""
    x = np.asarray(x, dtype=np.float64)
    d = getattr(g, "_oracle_deg", None)
    if d is None or len(d) != g.n:
        d = degree(g)
        g._oracle_deg = d
    return d * x - adjacency_csr(g) @ x


def laplacian_dense(g) -> np.ndarray:
    """Dense L = D - A (small graphs only)."""
    L = np.zeros((g.n, g.n))
    r = rows_of(g)
    np.add.at(L, (r, g.col.astype(np.int64)), -g.w.astype(np.float64))
    L[np.arange(g.n), np.arange(g.n)] += degree(g)
    return L


def induced(g, members: np.ndarray):
    """Induced subgraph on the boolean mask `members` (reading R2)."""
    from meshgen import DualGraph

    members = np.asarray(members, dtype=bool)
    newid = np.cumsum(members) - 1
    r = rows_of(g)
    keep = members[r] & members[g.col]
    cnt = np.bincount(r[keep], minlength=g.n)[members]
    row_ptr = np.zeros(int(members.sum()) + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    return DualGraph(int(members.sum()), row_ptr, newid[g.col[keep]].astype(np.int32),
                     g.w[keep].astype(np.int32), g.gid[members].copy())


def components(g) -> np.ndarray:
    """Per-vertex component label = smallest gid in the component.

    Plain min-label propagation until nothing changes.
    """
    lab = g.gid.astype(np.int64).copy()
    has = np.diff(g.row_ptr) > 0
    starts = g.row_ptr[:-1][has]
    while True:
        nb = lab.copy()
        if len(g.col):
            nb[has] = np.minimum(lab[has], np.minimum.reduceat(lab[g.col], starts))
        if np.array_equal(nb, lab):
            return lab
        lab = nb


# ----------------------------------------------------------------------------
# dense symmetric eigensolver: cyclic Jacobi (Golub & Van Loan, §8.5)
# ----------------------------------------------------------------------------


def jacobi_eigh(M: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """All eigenpairs of a symmetric matrix by cyclic-by-row Jacobi rotations.

    Returns (eigenvalues ascending, eigenvectors as columns).
    """
    A = np.array(M, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    scale = np.linalg.norm(A) or 1.0
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                if tau >= 0:
                    t = 1.0 / (tau + np.sqrt(1.0 + tau * tau))
                else:
                    t = -1.0 / (-tau + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap, aq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    lam = np.diag(A).copy()
    order = np.argsort(lam, kind="stable")
    return lam[order], V[:, order]


# ----------------------------------------------------------------------------
# start vector (counter-based generator, SplitMix64)
# ----------------------------------------------------------------------------

_GOLD = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(state) -> np.ndarray:
    """SplitMix64 output for state(s) `state` (Steele, Lea & Flood 2014)."""
    z = np.asarray(state, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLD
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def start_vector(gid: np.ndarray, seed: int, d: int = 0) -> np.ndarray:
    """s_i = 2 u_i - 1, u_i = top 53 bits of SplitMix64(s_d XOR gid_i) / 2^53,
    s_d = SplitMix64(seed + d)."""
    sd = splitmix64(np.uint64((seed + d) % (1 << 64)))
    h = splitmix64(sd ^ np.asarray(gid).astype(np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


# ----------------------------------------------------------------------------
# Fiedler solvers (§6 Lanczos, §7 inverse iteration)
# ----------------------------------------------------------------------------


def _fixed_basis(n: int, deflate) -> np.ndarray:
    cols = [np.full(n, 1.0 / np.sqrt(n))]
    cols += [np.asarray(d, dtype=np.float64) for d in deflate]
    return np.stack(cols, axis=1)


def _cgs(B: np.ndarray, x: np.ndarray):
    """One classical Gram-Schmidt pass: all coefficients from the same x."""
    c = B.T @ x
    return x - B @ c, c


def _project_start(B, x):
    x, _ = _cgs(B, x)
    x, _ = _cgs(B, x)
    return x / np.linalg.norm(x)


def lanczos_fiedler(g, opts: Options, deflate=(), start=None):
    """Fiedler pair of a connected graph by thick-restarted Lanczos (§6, reading R3).

    Returns None when the space orthogonal to 1 and `deflate` is empty.
    """
    n = g.n
    nd = len(deflate)
    dim = n - 1 - nd
    if dim <= 0:
        return None
    m = min(opts.krylov_dim, dim)
    B = _fixed_basis(n, deflate)
    nb = B.shape[1]
    dmax = float(degree(g).max())
    q = start_vector(g.gid, opts.seed, nd) if start is None else np.array(start, dtype=np.float64)
    # columns: the fixed basis [1/sqrt(n), deflation vectors], then q_0..q_{m-1}
    BV = np.zeros((n, nb + m))
    BV[:, :nb] = B
    V = BV[:, nb:]
    S = np.zeros((m, m))
    V[:, 0] = _project_start(B, q)
    j0 = 0
    theta, y, res = 0.0, V[:, 0], np.inf
    for cycle in range(1, opts.max_restarts + 1):
        meff, w_last = m, None
        for j in range(j0, m):
            w = laplacian_apply(g, V[:, j])
            basis = BV[:, :nb + j + 1]
            w, c1 = _cgs(basis, w)
            w, c2 = _cgs(basis, w)
            col = (c1 + c2)[nb:]
            S[:j + 1, j] = col
            S[j, :j + 1] = col
            b = float(np.linalg.norm(w))
            if b <= opts.breakdown * dmax:
                meff, w_last = j + 1, None
                break
            if j + 1 < m:
                V[:, j + 1] = w / b
            else:
                w_last = w / b
        thetas, Y = np.linalg.eigh(S[:meff, :meff])
        theta = float(thetas[0])
        y = V[:, :meff] @ Y[:, 0]
        y = y / np.linalg.norm(y)
        res = float(np.linalg.norm(laplacian_apply(g, y) - theta * y))
        if res <= opts.tol * dmax:
            return FiedlerResult(theta, y, res, cycle, True)
        k = min(opts.keep, meff - 1) if w_last is not None else 0
        S[:] = 0.0
        if k <= 0:
            V[:, 0] = _project_start(B, y)
            j0 = 0
            continue
        V[:, :k] = V[:, :meff] @ Y[:, :k]
        V[:, k] = w_last
        S[np.arange(k), np.arange(k)] = thetas[:k]
        j0 = k
    return FiedlerResult(theta, y, res, opts.max_restarts, False)


def cg_solve(g, b: np.ndarray, B: np.ndarray, opts: Options):
    """CG on L x = b from x0 = 0, r projected against B each step (§7)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.linalg.norm(b))
    it = 0
    for it in range(1, opts.cg_maxit + 1):
        ap = laplacian_apply(g, p)
        a = rr / float(p @ ap)
        x = x + a * p
        r = r - a * ap
        r, _ = _cgs(B, r)
        rr_new = float(r @ r)
        if np.sqrt(rr_new) <= opts.cg_tol * bnorm:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, it


def inverse_fiedler(g, opts: Options, deflate=(), start=None):
    """Fiedler pair by inverse iteration with CG (§7, Algorithm 2)."""
    n = g.n
    if n - 1 - len(deflate) <= 0:
        return None
    B = _fixed_basis(n, deflate)
    dmax = float(degree(g).max())
    b = start_vector(g.gid, opts.seed, len(deflate)) if start is None \
        else np.array(start, dtype=np.float64)
    lam, y, res, inner = 0.0, b, np.inf, 0
    for it in range(1, opts.max_outer + 1):
        b = _project_start(B, b)
        x, inner = cg_solve(g, b, B, opts)
        y = x / np.linalg.norm(x)
        ly = laplacian_apply(g, y)
        lam = float(y @ ly)
        res = float(np.linalg.norm(ly - lam * y))
        if res <= opts.tol * dmax or inner == 1:
            return FiedlerResult(lam, y, res, it, True, inner)
        b = y
    return FiedlerResult(lam, y, res, opts.max_outer, False, inner)


def _block_start(gid, seed, nd, b, cycle=0):
    """Start block: column c is the start vector of seed + (c + b * cycle) * 2^32
    (column 0 of the first cycle is the single-vector start)."""
    return np.stack([start_vector(gid, (seed + ((c + b * cycle) << 32)) % (1 << 64), nd)
                     for c in range(b)], axis=1)


def _chol_scaled(G: np.ndarray, tiny: float, pivot_min: float):
    """Upper R with G = R^T R, from the Cholesky factor of the correlation matrix
    D^-1 G D^-1 (D = sqrt diag G); None when a column is tiny (norm <= tiny) or
    the columns are nearly dependent (a scaled pivot^2 below pivot_min)."""
    d = np.sqrt(np.maximum(np.diag(G), 0.0))
    if (d <= tiny).any():
        return None
    Gs = G / np.outer(d, d)
    try:
        Rs = np.linalg.cholesky(Gs).T
    except np.linalg.LinAlgError:
        return None
    if (np.diag(Rs) ** 2 < pivot_min).any():
        return None
    return Rs * d[None, :]


def block_lanczos_fiedler(g, opts: Options, deflate=(), start=None):
    """Fiedler pair by thick-restarted block Lanczos of width b = opts.block.

    The single-vector method of §6 (reading R3) with a block of b vectors per
    step, the extension §9 names for nearly repeated lambda_2: each block step
    normalises the residual block W by a Cholesky QR (Q_new = W R^-1, G = W^T W
    = R^T R, factored on the correlation matrix), applies L to it, and
    re-orthogonalises Z = L Q_new by two classical Gram-Schmidt passes against
    [1/sqrt(n), deflation vectors, q_0 .. q_{j+b-1}]; the passes' coefficients
    on the basis are the b new columns of S = Q^T L Q.  A cycle adds blocks
    while the basis has room for one (m = krylov_dim columns), then takes the
    Ritz pairs of S, y = Q s_1 and its residual; the thick restart keeps the
    kk smallest Ritz vectors, kk = keep + ((m - keep) mod b) so that whole
    blocks fill the basis, and continues from the residual block.  A block whose
    columns are (nearly) dependent ends the cycle early; the next cycle then
    restarts from y and fresh start columns.  Graphs with fewer than
    krylov_dim + b dimensions orthogonal to the fixed basis use the
    single-vector method.
    """
    n = g.n
    nd = len(deflate)
    dim = n - 1 - nd
    if dim <= 0:
        return None
    b = max(1, int(opts.block))
    m = min(opts.krylov_dim, dim)
    if b == 1 or dim < opts.krylov_dim + b:
        return lanczos_fiedler(g, opts, deflate, start)
    B = _fixed_basis(n, deflate)
    nb = B.shape[1]
    dmax = float(degree(g).max())
    tiny = opts.breakdown * dmax
    W = _block_start(g.gid, opts.seed, nd, b)
    if start is not None:
        W[:, 0] = np.asarray(start, dtype=np.float64)
    W, _ = _cgs(B, W)
    W, _ = _cgs(B, W)
    BV = np.zeros((n, nb + m))
    BV[:, :nb] = B
    V = BV[:, nb:]
    S = np.zeros((m, m))
    kk_restart = opts.keep + (m - opts.keep) % b
    j0 = 0
    theta, y, res = 0.0, None, np.inf
    for cycle in range(1, opts.max_restarts + 1):
        j, broke = j0, False
        while j + b <= m:
            R = _chol_scaled(W.T @ W, tiny, 1e-12)
            if R is None:
                broke = True
                break
            V[:, j:j + b] = W @ np.linalg.inv(R)
            Z = np.stack([laplacian_apply(g, V[:, j + c]) for c in range(b)], axis=1)
            basis = BV[:, :nb + j + b]
            Z, C1 = _cgs(basis, Z)
            Z, C2 = _cgs(basis, Z)
            col = (C1 + C2)[nb:, :]                  # (j + b) x b
            S[:j, j:j + b] = col[:j]
            S[j:j + b, :j] = col[:j].T
            S[j:j + b, j:j + b] = 0.5 * (col[j:] + col[j:].T)
            W = Z
            j += b
        meff = j
        if meff == 0:
            break
        thetas, Y = np.linalg.eigh(S[:meff, :meff])
        theta = float(thetas[0])
        y = V[:, :meff] @ Y[:, 0]
        y = y / np.linalg.norm(y)
        res = float(np.linalg.norm(laplacian_apply(g, y) - theta * y))
        if res <= opts.tol * dmax:
            return FiedlerResult(theta, y, res, cycle, True)
        S[:] = 0.0
        kk = min(kk_restart, meff - 1)
        if broke or kk <= 0:
            W = _block_start(g.gid, opts.seed, nd, b, cycle)
            W[:, 0] = y
            W, _ = _cgs(B, W)
            W, _ = _cgs(B, W)
            j0 = 0
            continue
        V[:, :kk] = V[:, :meff] @ Y[:, :kk]
        S[np.arange(kk), np.arange(kk)] = thetas[:kk]
        j0 = kk
    if y is None:
        return lanczos_fiedler(g, opts, deflate, start)
    return FiedlerResult(theta, y, res, opts.max_restarts, False)


def fiedler(g, opts: Options, deflate=(), start=None):
    if opts.method == "lanczos" and opts.block > 1:
        return block_lanczos_fiedler(g, opts, deflate, start)
    if opts.method == "lanczos":
        return lanczos_fiedler(g, opts, deflate, start)
    if opts.method == "inverse" and opts.amg:
        from .amg import amg_inverse_fiedler

        return amg_inverse_fiedler(g, opts, deflate, start)
    if opts.method == "inverse":
        return inverse_fiedler(g, opts, deflate, start)
    raise ValueError(opts.method)


# ----------------------------------------------------------------------------
# orientation, degeneracy, median split (R4, R5, R7)
# ----------------------------------------------------------------------------


def orient(v: np.ndarray, gid: np.ndarray) -> np.ndarray:
    """R4: negate v unless the smallest gid among |v| >= max|v|/2 is negative."""
    a = np.abs(v)
    cand = a >= 0.5 * a.max()
    gstar = gid[cand].min()
    i = int(np.nonzero(gid == gstar)[0][0])
    return -v if v[i] > 0 else v


def split_k(v: np.ndarray, gid: np.ndarray, k: int, tie_rel: float) -> np.ndarray:
    """R7: boolean mask of the k elements that go left."""
    n = len(v)
    if k <= 0:
        return np.zeros(n, dtype=bool)
    if k >= n:
        return np.ones(n, dtype=bool)
    vk = np.sort(v)[k - 1]
    tau = tie_rel * (v.max() - v.min())
    left = v < vk - tau
    tie = np.abs(v - vk) <= tau
    need = k - int(left.sum())
    ti = np.nonzero(tie)[0]
    ti = ti[np.argsort(gid[ti], kind="stable")]
    left[ti[:need]] = True
    return left


def weighted_cut(g, left: np.ndarray) -> int:
    r = rows_of(g)
    diff = left[r] != left[g.col]
    return int(g.w[diff].astype(np.int64).sum()) // 2


def _quartic_pair_angle(x, y):
    """Angle of the 2-D rotation that minimises sum(a^4 + b^4),
    a = x cos t - y sin t, b = x sin t + y cos t (equivalently maximises sum (ab)^2)."""
    u = x * x - y * y
    w = 2.0 * x * y
    A = 0.5 * (np.sum(w * w) - np.sum(u * u))
    B = np.sum(u * w)
    return 0.25 * np.arctan2(B, A)


def quartic_rotate(U: np.ndarray) -> np.ndarray:
    """R5: columns of U R with R orthogonal minimising sum((U R)^4)."""
    U = np.array(U, dtype=np.float64, copy=True)
    m = U.shape[1]
    if m == 1:
        return U
    for _ in range(50 if m > 2 else 1):
        dmax = 0.0
        for p in range(m - 1):
            for q in range(p + 1, m):
                t = _quartic_pair_angle(U[:, p], U[:, q])
                c, s = np.cos(t), np.sin(t)
                a = U[:, p] * c - U[:, q] * s
                b = U[:, p] * s + U[:, q] * c
                U[:, p], U[:, q] = a, b
                dmax = max(dmax, abs(t))
        if dmax < 1e-12:
            break
    return U


def _lex_prefers(left_a: np.ndarray, left_b: np.ndarray, gid: np.ndarray) -> bool:
    """True when split a wins the gid rule of R5 against split b."""
    diff = left_a != left_b
    if not diff.any():
        return False
    i = np.nonzero(diff)[0][np.argmin(gid[diff])]
    return bool(left_a[i])


def fiedler_candidates(g, opts: Options):
    """Candidate vectors for the split of one connected graph (R5)."""
    ra = fiedler(g, opts)
    vecs, lams, info = [ra.v], [ra.lam], [ra]
    if opts.degenerate == "resolve":
        while len(vecs) < 3:
            rb = fiedler(g, opts, deflate=vecs)
            if rb is None or abs(rb.lam - lams[0]) > opts.cluster_tol * lams[0]:
                break
            vecs.append(rb.v)
            lams.append(rb.lam)
            info.append(rb)
    if len(vecs) == 1:
        return [vecs[0]], info
    U = quartic_rotate(np.stack(vecs, axis=1))
    return [U[:, c] for c in range(U.shape[1])], info


def split_connected(g, k: int, opts: Options, record=None) -> np.ndarray:
    """Left mask of size k for a connected graph (Algorithm 1 steps 1-4)."""
    cands, info = fiedler_candidates(g, opts)
    best, best_cut = None, None
    for v in cands:
        vo = orient(v, g.gid)
        left = split_k(vo, g.gid, k, opts.tie_rel)
        cut = weighted_cut(g, left)
        if best is None or cut < best_cut or (cut == best_cut and _lex_prefers(left, best, g.gid)):
            best, best_cut = left, cut
    if record is not None:
        record.append({"n": g.n, "k": k, "lam": info[0].lam, "resid": info[0].resid,
                       "iters": info[0].iters, "cluster": len(cands), "cut": best_cut})
    return best


def bisect(g, k: int, opts: Options, record=None) -> np.ndarray:
    """Left mask of size k for any graph: components first (R8)."""
    lab = components(g)
    left = np.zeros(g.n, dtype=bool)
    filled = 0
    for c in np.unique(lab):          # ascending smallest gid
        mem = lab == c
        s = int(mem.sum())
        if filled + s <= k:
            left |= mem
            filled += s
        elif filled < k:
            sub = induced(g, mem)
            left[mem] = split_connected(sub, k - filled, opts, record)
            filled = k
    return left


# ----------------------------------------------------------------------------
# recursion (Algorithm 1, R6) and metrics (§8)
# ----------------------------------------------------------------------------


def seg_size(p0: int, p1: int, N: int, P: int) -> int:
    return (p1 * N) // P - (p0 * N) // P


def rsb_partition(g, P: int, opts: Options | None = None, record=None) -> np.ndarray:
    """Part id in [0, P) for every vertex of g (Algorithm 1 with R1-R9)."""
    opts = opts or Options()
    N = g.n
    if P < 1 or P > max(N, 1):
        raise ValueError("need 1 <= P <= n")
    part = np.full(N, -1, dtype=np.int32)
    stack = [(np.arange(N, dtype=np.int64), 0, P)]
    while stack:
        idx, p0, p1 = stack.pop()
        if p1 - p0 == 1:
            part[idx] = p0
            continue
        pm = p0 + (p1 - p0) // 2
        k = (pm * N) // P - (p0 * N) // P
        mem = np.zeros(N, dtype=bool)
        mem[idx] = True
        sub = induced(g, mem)
        left = bisect(sub, k, opts, record)
        stack.append((idx[~left], pm, p1))
        stack.append((idx[left], p0, pm))
    return part


def rcb_partition(coords: np.ndarray, gid: np.ndarray, P: int, tie_rel: float = 1e-5) -> np.ndarray:
    """Recursive coordinate bisection into P parts (the geometric pre-partitioner
    §5 and §8 run before RSB): a segment is split along the axis of its largest
    coordinate extent (the lowest axis on equal extents) at the proportional
    count of R6, lower coordinates left, equal coordinates (within tie_rel of the
    extent) left in ascending gid (R7)."""
    coords = np.asarray(coords, dtype=np.float64)
    N = len(coords)
    part = np.full(N, -1, dtype=np.int32)
    stack = [(np.arange(N, dtype=np.int64), 0, P)]
    while stack:
        idx, p0, p1 = stack.pop()
        if p1 - p0 == 1:
            part[idx] = p0
            continue
        pm = p0 + (p1 - p0) // 2
        k = (pm * N) // P - (p0 * N) // P
        c = coords[idx]
        ext = c.max(axis=0) - c.min(axis=0)
        axis = int(np.argmax(ext))
        left = split_k(c[:, axis], gid[idx], k, tie_rel)
        stack.append((idx[~left], pm, p1))
        stack.append((idx[left], p0, pm))
    return part


def fiedler_of_graph(g, opts: Options | None = None):
    """(lambda_2, oriented Fiedler vector, residual) of a connected graph."""
    opts = opts or Options()
    r = fiedler(g, opts)
    return r.lam, orient(r.v, g.gid), r


def partition_metrics(g, part: np.ndarray, P: int) -> dict:
    """Edge cut, part sizes and neighbour counts per part (§8 quality metrics)."""
    r = rows_of(g)
    diff = part[r] != part[g.col]
    sizes = np.bincount(part, minlength=P)
    pairs = np.unique(np.stack([part[r][diff], part[g.col][diff]], axis=1), axis=0) \
        if diff.any() else np.zeros((0, 2), dtype=np.int64)
    nbr = np.bincount(pairs[:, 0], minlength=P) if len(pairs) else np.zeros(P, dtype=np.int64)
    return {
        "weighted_cut": int(g.w[diff].astype(np.int64).sum()) // 2,
        "edge_cut": int(diff.sum()) // 2,
        "sizes": sizes,
        "max_neighbours": int(nbr.max()) if P else 0,
        "avg_neighbours": float(nbr.mean()) if P else 0.0,
    }
