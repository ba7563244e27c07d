"""Closed-form RSB partitions of face-adjacency box meshes.

TEST INFRASTRUCTURE (same import rule as the rest of ``oracle``).

For an a x b x c box with face adjacency and unit weights the Laplacian is the
Kronecker sum of path Laplacians, so its spectrum is
    lambda(k1, k2, k3) = sum_axes 2 (1 - cos(pi k_a / n_a))
with eigenvectors prod_a cos(pi k_a (i_a + 1/2) / n_a).  lambda_2 belongs to the
longest axis and its Fiedler vector is constant on the slabs normal to that
axis, so a bisection whose left count is a whole number of slabs cuts the box
into two boxes.  When several axes share the longest length the cluster rule
(R5) applies: every axis candidate cuts the same number of faces, and the gid
rule prefers the axis with the largest gid stride (z, then y, then x).  The
orientation rule (R4) puts the low-coordinate end, which holds the box's
smallest gid, on the left.

``box_partition_closed_form`` follows that derivation and raises NotClean when
some split would cut through a slab (the children are then no longer boxes and
no closed form is claimed).
"""
from __future__ import annotations

import numpy as np


class NotClean(Exception):
    """A split falls inside a slab; the recursion leaves the closed form."""


def box_lambda2(nx: int, ny: int, nz: int) -> float:
    """2 (1 - cos(pi / n_max)) for the face-adjacency unit-weight box."""
    return 2.0 * (1.0 - np.cos(np.pi / max(nx, ny, nz)))


def box_spectrum(nx: int, ny: int, nz: int) -> np.ndarray:
    """All eigenvalues of the face-adjacency box Laplacian, ascending."""
    ev = [2.0 * (1.0 - np.cos(np.pi * np.arange(n) / n)) for n in (nx, ny, nz)]
    s = ev[0][None, None, :] + ev[1][None, :, None] + ev[2][:, None, None]
    return np.sort(s.ravel())


def box_fiedler_x(nx: int, ny: int, nz: int) -> np.ndarray:
    """Unit Fiedler vector cos(pi (i + 1/2) / nx) for a box whose x side is longest."""
    i = np.arange(nx)
    v = np.broadcast_to(np.cos(np.pi * (i + 0.5) / nx)[None, None, :], (nz, ny, nx)).ravel()
    return v / np.linalg.norm(v)


def box_partition_closed_form(nx: int, ny: int, nz: int, P: int) -> np.ndarray:
    """Part id per gid (gid = i + nx (j + ny k)) for RSB of a box into P parts."""
    N = nx * ny * nz
    part = np.full(N, -1, dtype=np.int32)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = (ii.ravel(), jj.ravel(), kk.ravel())
    gid = np.arange(N)

    def rec(lo, hi, p0, p1):
        sel = ((coords[0] >= lo[0]) & (coords[0] < hi[0]) & (coords[1] >= lo[1]) &
               (coords[1] < hi[1]) & (coords[2] >= lo[2]) & (coords[2] < hi[2]))
        if p1 - p0 == 1:
            part[gid[sel]] = p0
            return
        pm = p0 + (p1 - p0) // 2
        k = (pm * N) // P - (p0 * N) // P
        ext = [hi[a] - lo[a] for a in range(3)]
        longest = max(ext)
        axis = max(a for a in range(3) if ext[a] == longest)   # z > y > x on ties
        slab = int(np.prod([ext[a] for a in range(3) if a != axis]))
        if k % slab:
            raise NotClean(f"split of {ext} at {k} cuts a slab")
        cut = lo[axis] + k // slab
        hl, lh = list(hi), list(lo)
        hl[axis] = cut
        lh[axis] = cut
        rec(lo, hl, p0, pm)
        rec(lh, hi, pm, p1)

    rec([0, 0, 0], [nx, ny, nz], 0, P)
    return part
