"""Box hex meshes and their element dual graphs (paper §2).

A vertex of the dual graph is a hex element of an nx x ny x nz structured box
mesh; element (i, j, k) has global id  gid = i + nx * (j + ny * k).  Two
elements are adjacent when they share a face ("face" adjacency, unit weight,
6 neighbours in the interior) or any vertex ("vertex" adjacency, 26
neighbours), and in the vertex form the edge weight is the number of mesh
vertices the two elements share: 4 across a face, 2 across an edge, 1 across a
corner (paper §2, weight function omega).  For a neighbour offset
(di, dj, dk) that count is (2-|di|)(2-|dj|)(2-|dk|).

Rows are emitted in gid order and the columns of each row ascend, so the CSR is
canonical.  Deletion draws and batch dimensions come from SplitMix64 (Steele,
Lea & Flood, OOPSLA 2014), a counter-based generator whose output for state s is
mix(s + 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state) -> np.ndarray:
    """SplitMix64 output for the given 64-bit state(s) (one generator step)."""
    z = np.asarray(state, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


@dataclass
class DualGraph:
    """Symmetric weighted graph in CSR form.

    row_ptr: int64[n+1]; col: int32[nnz]; w: int32[nnz] (positive integers);
    gid: int64[n], the element id used for tie-breaks and start vectors.
    """

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    gid: np.ndarray
    dims: tuple | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self) -> np.ndarray:
        """Row index of every stored entry (int64[nnz])."""
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))

    def box_index(self) -> np.ndarray:
        """Box element index i + nx (j + ny k) of every row (box meshes only)."""
        if "box_index" in self.meta:
            return self.meta["box_index"]
        if self.meta.get("kind") == "box_deleted":
            return self.meta["orig_gid"]
        if self.meta.get("kind") == "box":
            return self.gid
        raise ValueError("not a box mesh")

    def centroids(self) -> np.ndarray:
        """Element centroids (n x 3, float64): element (i, j, k) of a box with unit
        spacing has its centre at (i + 1/2, j + 1/2, k + 1/2)."""
        nx, ny, _ = self.dims
        idx = self.box_index()
        return np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], axis=1) + 0.5

    def hex_vertices(self) -> np.ndarray:
        """Global vertex ids of every element's 8 corners (n x 8, int64): corner
        (a, b, c) in {0,1}^3 of element (i, j, k) is mesh vertex
        (i + a) + (nx + 1) ((j + b) + (ny + 1) (k + c)), listed with a fastest."""
        nx, ny, _ = self.dims
        idx = self.box_index()
        i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
        out = np.empty((len(idx), 8), dtype=np.int64)
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    out[:, a + 2 * b + 4 * c] = (i + a) + (nx + 1) * ((j + b) + (ny + 1) * (k + c))
        return out


def _offsets(adjacency: str):
    if adjacency == "face":
        offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
        # ordered so that the column offset di + nx*(dj + ny*dk) ascends
        offs = sorted(offs, key=lambda o: (o[2], o[1], o[0]))
        return [(di, dj, dk, 1) for (di, dj, dk) in offs]
    if adjacency == "vertex":
        offs = []
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    if di == dj == dk == 0:
                        continue
                    w = (2 - abs(di)) * (2 - abs(dj)) * (2 - abs(dk))
                    offs.append((di, dj, dk, w))
        return offs
    raise ValueError(f"unknown adjacency {adjacency!r}")


def _neighbour_table(nx: int, ny: int, nz: int, adjacency: str):
    """Dense (n, K) table of neighbour gids (-1 where outside the box)."""
    offs = _offsets(adjacency)
    n = nx * ny * nz
    g = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    cols = np.full((n, len(offs)), -1, dtype=np.int64)
    wts = np.array([o[3] for o in offs], dtype=np.int32)
    view = cols.reshape(nz, ny, nx, len(offs))
    for t, (di, dj, dk, _) in enumerate(offs):
        zs = slice(max(0, -dk), nz - max(0, dk))
        ys = slice(max(0, -dj), ny - max(0, dj))
        xs = slice(max(0, -di), nx - max(0, di))
        zd = slice(zs.start + dk, zs.stop + dk)
        yd = slice(ys.start + dj, ys.stop + dj)
        xd = slice(xs.start + di, xs.stop + di)
        view[zs, ys, xs, t] = g[zd, yd, xd]
    return cols, wts


def _csr_from_table(cols: np.ndarray, wts: np.ndarray, valid: np.ndarray):
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[valid].astype(np.int32)
    w = np.broadcast_to(wts, cols.shape)[valid].astype(np.int32)
    return row_ptr, col, w


def box_graph(nx: int, ny: int, nz: int, adjacency: str = "face") -> DualGraph:
    """Dual graph of an nx x ny x nz hex box (rows in gid order)."""
    cols, wts = _neighbour_table(nx, ny, nz, adjacency)
    valid = cols >= 0
    row_ptr, col, w = _csr_from_table(cols, wts, valid)
    n = nx * ny * nz
    return DualGraph(n, row_ptr, col, w, np.arange(n, dtype=np.int64), (nx, ny, nz),
                     {"kind": "box", "adjacency": adjacency})


def _components_min_label(n, row_ptr, col):
    """Component label = smallest vertex index in the component (scipy BFS)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    a = sp.csr_matrix((np.ones(len(col), dtype=np.int8), col, row_ptr), shape=(n, n))
    ncomp, lab = connected_components(a, directed=False)
    first = np.full(ncomp, n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(n, dtype=np.int64))
    return ncomp, lab, first


def box_graph_deleted(nx: int, ny: int, nz: int, frac: float, seed: int,
                      adjacency: str = "vertex") -> DualGraph:
    """Box dual graph with a seeded element deletion, largest component kept.

    Exactly floor(frac * n) elements are deleted: those with the smallest
    SplitMix64(seed XOR gid), ties broken by gid.  The largest connected
    component of what remains is kept (ties: the one holding the smallest gid)
    and renumbered compactly in original gid order; the new row index is the
    element's gid.
    """
    n = nx * ny * nz
    ndel = int(np.floor(frac * n))
    gid0 = np.arange(n, dtype=np.int64)
    h = splitmix64(np.uint64(seed) ^ gid0.astype(np.uint64))
    order = np.lexsort((gid0, h))
    keep = np.ones(n, dtype=bool)
    keep[order[:ndel]] = False

    cols, wts = _neighbour_table(nx, ny, nz, adjacency)
    valid = cols >= 0
    valid &= keep[np.where(valid, cols, 0)]
    valid &= keep[:, None]
    row_ptr, col, w = _csr_from_table(cols, wts, valid)
    del cols, valid

    ncomp, lab, first = _components_min_label(n, row_ptr, col)
    size = np.bincount(lab, minlength=ncomp)
    size[lab[~keep]] -= 1  # deleted elements are isolated singletons
    # largest component; ties go to the one with the smallest first index
    best = np.lexsort((first, -size))[0]
    member = (lab == best) & keep
    newid = np.cumsum(member) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    ent = member[rows]
    counts = np.bincount(rows[ent], minlength=n)[member]
    row_ptr2 = np.zeros(int(member.sum()) + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr2[1:])
    col2 = newid[col[ent]].astype(np.int32)
    w2 = w[ent]
    m = int(member.sum())
    return DualGraph(m, row_ptr2, col2, w2, np.arange(m, dtype=np.int64), (nx, ny, nz),
                     {"kind": "box_deleted", "adjacency": adjacency, "frac": frac,
                      "seed": seed, "orig_gid": np.nonzero(member)[0]})


def batch_box_dims(count: int, lo: int, hi: int, seed: int) -> list[tuple[int, int, int]]:
    """Box dimensions drawn uniformly from the integers [lo, hi] per axis.

    Axis a of mesh m uses u = (SplitMix64(seed + 3m + a) >> 11) * 2^-53 and
    side = lo + floor(u * (hi - lo + 1)).
    """
    s = np.uint64(seed) + np.arange(3 * count, dtype=np.uint64)
    u = (splitmix64(s) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    sides = lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
    return [tuple(int(x) for x in sides[3 * m:3 * m + 3]) for m in range(count)]


def random_graph(n: int, extra_edges: int, seed: int, weights=(1, 2, 4),
                 connected: bool = True) -> DualGraph:
    """Random weighted graph for property tests.

    A random spanning tree (when connected) plus `extra_edges` random chords,
    weights drawn from `weights`.  Uses numpy's PCG64 generator.
    """
    rng = np.random.default_rng(seed)
    edges = {}
    if connected and n > 1:
        perm = rng.permutation(n)
        for t in range(1, n):
            a = int(perm[t])
            b = int(perm[rng.integers(0, t)])
            edges[(min(a, b), max(a, b))] = int(rng.choice(weights))
    tries = 0
    while extra_edges > 0 and tries < 100 * (extra_edges + 1) and n > 1:
        tries += 1
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b or (min(a, b), max(a, b)) in edges:
            continue
        edges[(min(a, b), max(a, b))] = int(rng.choice(weights))
        extra_edges -= 1
    return _graph_from_edges(n, edges, np.arange(n, dtype=np.int64), {"kind": "random"})


def _graph_from_edges(n, edges: dict, gid, meta) -> DualGraph:
    if edges:
        e = np.array([(a, b, w) for (a, b), w in edges.items()], dtype=np.int64)
        src = np.concatenate([e[:, 0], e[:, 1]])
        dst = np.concatenate([e[:, 1], e[:, 0]])
        ww = np.concatenate([e[:, 2], e[:, 2]])
    else:
        src = dst = ww = np.zeros(0, dtype=np.int64)
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return DualGraph(n, row_ptr, dst.astype(np.int32), ww.astype(np.int32),
                     np.asarray(gid, dtype=np.int64), None, meta)


def disjoint_union(graphs: list[DualGraph], gid_stride: int | None = None) -> DualGraph:
    """Block-diagonal union of graphs; gids are offset so that they stay distinct."""
    n = sum(g.n for g in graphs)
    row_ptr = [np.zeros(1, dtype=np.int64)]
    cols, ws, gids = [], [], []
    off = 0
    nnz = 0
    goff = 0
    for g in graphs:
        row_ptr.append(g.row_ptr[1:] + nnz)
        cols.append(g.col.astype(np.int64) + off)
        ws.append(g.w)
        gids.append(g.gid + goff)
        off += g.n
        nnz += g.nnz
        goff += gid_stride if gid_stride is not None else (int(g.gid.max()) + 1 if g.n else 0)
    return DualGraph(n, np.concatenate(row_ptr), np.concatenate(cols).astype(np.int32),
                     np.concatenate(ws).astype(np.int32), np.concatenate(gids), None,
                     {"kind": "union"})


def quad_vertex_lists_dual(vertex_lists: list[list[int]]) -> DualGraph:
    """Dual graph of elements given by their global vertex ids (paper §5, Fig. 2).

    Elements e != f are adjacent when they share at least one global vertex id;
    the weight is the number of shared ids.
    """
    m = len(vertex_lists)
    sets = [set(v) for v in vertex_lists]
    edges = {}
    for a in range(m):
        for b in range(a + 1, m):
            s = len(sets[a] & sets[b])
            if s:
                edges[(a, b)] = s
    return _graph_from_edges(m, edges, np.arange(m, dtype=np.int64), {"kind": "vertex_lists"})


def permute_graph(g: DualGraph, seed: int) -> DualGraph:
    """The same graph with its rows in a seeded random order (numpy PCG64);
    every element keeps its gid (and its box position), so any method that
    depends only on gids and the graph gives the same answer."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)          # new row r holds old row perm[r]
    inv = np.empty(g.n, dtype=np.int64)
    inv[perm] = np.arange(g.n)
    lens = np.diff(g.row_ptr)[perm]
    row_ptr = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    starts = g.row_ptr[perm]
    take = np.repeat(starts - row_ptr[:-1], lens) + np.arange(row_ptr[-1])
    col = inv[g.col[take]].astype(np.int32)
    w = g.w[take]
    meta = dict(g.meta)
    try:
        meta["box_index"] = g.box_index()[perm]
    except ValueError:
        pass
    meta["perm"] = perm
    # columns of each row ascending again
    rows = np.repeat(np.arange(g.n, dtype=np.int64), lens)
    order = np.lexsort((col, rows))
    return DualGraph(g.n, row_ptr, col[order], w[order], g.gid[perm].copy(), g.dims, meta)
