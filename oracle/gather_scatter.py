"""Matrix-free Laplacian by gather-scatter, and the dual graph of an element list.

TEST INFRASTRUCTURE (as the rest of ``oracle/``): only the tests, smoke() and
bench.py's CPU legs may use it; the CUDA library never does.

Paper §5 ("Evaluating the Laplacian"): with P the local copy matrix that maps
an element's value to its v local vertices and Q the Boolean matrix that maps
every global vertex to its local copies, the weighted adjacency of the dual
graph is A_w = P^T Q Q^T P (Q^T sums the local copies of a global vertex; Q
copies the sum back), the weighted degree matrix is D_w = diag(A_w 1), and
L = D_w - A_w.  The diagonal of A_w (an element meets itself at all v of its
vertices) cancels in L.  Off the diagonal, (A_w)_ef is the number of global
vertices elements e and f share: the weight omega of §2.  Sparse products are
the library's (scipy), the matrices are built as the text defines them.
"""
from __future__ import annotations

import numpy as np


def gs_operators(ev: np.ndarray):
    """(P, Q) of §5 for the element -> global vertex table ev (m x v)."""
    import scipy.sparse as sp

    ev = np.asarray(ev, dtype=np.int64)
    m, v = ev.shape
    ids, local = np.unique(ev.reshape(-1), return_inverse=True)
    rows = np.arange(m * v)
    P = sp.csr_matrix((np.ones(m * v), (rows, np.repeat(np.arange(m), v))), shape=(m * v, m))
    Q = sp.csr_matrix((np.ones(m * v), (rows, local)), shape=(m * v, len(ids)))
    return P, Q


def gs_adjacency_apply(ev: np.ndarray, x: np.ndarray) -> np.ndarray:
    """A_w x = P^T Q Q^T P x: copy to local vertices, sum per global vertex,
    copy back, sum per element."""
    P, Q = gs_operators(ev)
    return P.T @ (Q @ (Q.T @ (P @ np.asarray(x, dtype=np.float64))))


def gs_laplacian_apply(ev: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L x = D_w x - A_w x with D_w = diag(A_w 1)."""
    x = np.asarray(x, dtype=np.float64)
    d = gs_adjacency_apply(ev, np.ones(len(x)))
    return d * x - gs_adjacency_apply(ev, x)


def dual_graph_from_vertices(ev: np.ndarray, gid=None):
    """The weighted dual graph (A_w without its diagonal) as CSR with ascending
    columns: elements that share vertices, weighted by how many (§2)."""
    import scipy.sparse as sp

    from meshgen import DualGraph

    P, Q = gs_operators(ev)
    M = Q.T @ P                     # global vertex x element incidence
    A = (M.T @ M).tocsr()           # P^T Q Q^T P
    A.setdiag(0)
    A.eliminate_zeros()
    A.sort_indices()
    m = A.shape[0]
    return DualGraph(m, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                     np.rint(A.data).astype(np.int32),
                     np.arange(m, dtype=np.int64) if gid is None else np.asarray(gid, np.int64),
                     None, {"kind": "vertex_lists"})
