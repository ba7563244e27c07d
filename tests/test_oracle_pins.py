"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every oracle function is checked against something other than itself: the
paper's worked example (§5, Fig. 2), closed-form spectra of path and box
Laplacians, the cut identity of the spectral relaxation (§3), the component
count = multiplicity of the zero eigenvalue (§4), brute force on tiny inputs,
and the balance rule (§2, §4).  A few tests plant a mistake in a copy of an
oracle routine and check that the pin catches it.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from meshgen import (box_graph, box_graph_deleted, disjoint_union, quad_vertex_lists_dual,
                     random_graph, splitmix64)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig2():
    lines = [ln.split("#")[0].strip() for ln in open(os.path.join(GOLDEN, "fig2_gather_scatter.txt"))]
    lines = [ln for ln in lines if ln]
    i = lines.index("vertex_lists")
    vl = [[int(t) for t in lines[i + 1 + r].split()] for r in range(3)]
    i = lines.index("laplacian")
    L = np.array([[float(t) for t in lines[i + 1 + r].split()] for r in range(3)])
    kv = {ln.split()[0]: [float(t) for t in ln.split()[1:]] for ln in lines if ln.split()[0] in
          ("z2_for_x1", "spectrum", "fiedler_unnormalised")}
    return vl, L, kv


# ---------------------------------------------------------------- generators


def test_splitmix64_published_first_output():
    # first output of SplitMix64 from state 0 (Steele, Lea & Flood 2014 reference code)
    assert int(O.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    assert int(splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF


def test_box_graph_counts():
    g = box_graph(16, 8, 4)
    assert (g.n, g.nnz) == (512, 2624)
    g = box_graph(64, 64, 32)
    assert (g.n, g.nnz) == (131072, 770048)
    gv = box_graph(5, 4, 3, "vertex")
    # interior element of a 3x3x3 neighbourhood: 6 faces (w 4), 12 edges (w 2), 8 corners (w 1)
    assert sorted(np.bincount(gv.w)[1:].tolist()) == sorted(np.bincount(gv.w)[1:].tolist())
    d = O.degree(box_graph(3, 3, 3, "vertex"))
    assert d[13] == 6 * 4 + 12 * 2 + 8 * 1


# ---------------------------------------------------------------- Laplacian


def _apply_checks(apply, g):
    """The pins a correct Laplacian action must satisfy."""
    n = g.n
    one = np.ones(n)
    if np.abs(apply(g, one)).max() != 0.0:                      # L 1 = 0 (§4)
        return False
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    if abs(x @ apply(g, y) - y @ apply(g, x)) > 1e-9 * (1 + abs(x @ apply(g, y))):
        return False                                            # symmetry
    s = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    cut = 0
    for i in range(n):                                          # brute-force cut
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            j = g.col[e]
            if j > i and s[i] != s[j]:
                cut += int(g.w[e])
    return float(s @ apply(g, s)) == 4.0 * cut                  # x^T L x = 4 cut (§3)


@pytest.mark.parametrize("g", [box_graph(6, 5, 4), box_graph(5, 4, 3, "vertex"),
                               random_graph(40, 60, 3)])
def test_laplacian_pins(g):
    assert _apply_checks(O.laplacian_apply, g)


def test_planted_laplacian_mistakes_are_caught():
    g = random_graph(30, 40, 5)

    def no_diag(g, x):          # dropped degree term
        return O.laplacian_apply(g, x) - O.degree(g) * x

    def wrong_sign(g, x):       # sign flip on the adjacency term
        return O.degree(g) * x + (O.degree(g) * x - O.laplacian_apply(g, x))

    def unit_weights(g, x):     # weights ignored
        r = O.rows_of(g)
        return np.bincount(r, minlength=g.n) * x - np.bincount(r, weights=x[g.col], minlength=g.n)

    for bad in (no_diag, wrong_sign, unit_weights):
        assert not _apply_checks(bad, g)


def test_fig2_worked_example():
    vl, L, kv = _read_fig2()
    g = quad_vertex_lists_dual(vl)
    assert np.array_equal(O.laplacian_dense(g), L)
    x = np.array([1.0, 0.0, 0.0])
    z = O.degree(g) * x - O.laplacian_apply(g, x)              # A_w x
    assert z[1] == kv["z2_for_x1"][0]
    lam, V = O.jacobi_eigh(L)
    assert np.allclose(lam, kv["spectrum"], atol=1e-13)
    lam2, v, _ = O.fiedler_of_graph(g)
    assert abs(lam2 - 4.0) < 1e-12
    f = np.array(kv["fiedler_unnormalised"]) / np.sqrt(2)
    assert min(np.abs(v - f).max(), np.abs(v + f).max()) < 1e-12
    # orientation R4: both nonzero entries have |v| = max, the smaller gid (1) goes left
    assert v[1] < 0 < v[2]
    li, _, _ = O.fiedler_of_graph(g, O.Options(method="inverse"))
    assert abs(li - 4.0) < 1e-10


def test_gather_scatter_fig2():
    """§5 with the paper's Fig. 2 vertex lists: A_w = P^T Q Q^T P gives the
    printed Laplacian, and x = e_1 reaches element 2 along two paths."""
    vl, L, kv = _read_fig2()
    ev = np.array(vl)
    z = O.gs_adjacency_apply(ev, np.array([1.0, 0.0, 0.0]))
    assert z[1] == kv["z2_for_x1"][0]
    assert z[0] == 4.0                      # an element meets itself at its 4 vertices
    Lgs = np.stack([O.gs_laplacian_apply(ev, e) for e in np.eye(3)], axis=1)
    assert np.array_equal(Lgs, L)
    assert np.array_equal(O.laplacian_dense(O.dual_graph_from_vertices(ev)), L)


@pytest.mark.parametrize("g", [box_graph(5, 4, 3, "vertex"),
                               box_graph_deleted(9, 7, 6, 0.1, 4, "vertex")])
def test_gather_scatter_equals_assembled_dual_graph(g):
    """The dual graph built from the hexes' vertex ids is the vertex-adjacency
    graph of the generator, entry for entry, and the matrix-free action equals
    the assembled one (exactly, for integer vectors)."""
    ev = g.hex_vertices()
    h = O.dual_graph_from_vertices(ev)
    assert np.array_equal(h.row_ptr, g.row_ptr)
    assert np.array_equal(h.col, g.col) and np.array_equal(h.w, g.w)
    x = np.random.default_rng(1).integers(-5, 6, g.n).astype(np.float64)
    assert np.array_equal(O.gs_laplacian_apply(ev, x), O.laplacian_apply(g, x))


def test_planted_gather_scatter_mistake_is_caught():
    """Forgetting the diagonal correction (L = A_w instead of D_w - A_w) fails L 1 = 0."""
    vl, L, kv = _read_fig2()
    ev = np.array(vl)
    assert np.abs(O.gs_laplacian_apply(ev, np.ones(3))).max() == 0.0
    assert np.abs(O.gs_adjacency_apply(ev, np.ones(3))).max() > 0.0


# ---------------------------------------------------------------- dense eigensolver


def test_jacobi_path_graph_closed_form():
    for n in (2, 5, 17):
        edges = np.zeros((n, n))
        for i in range(n - 1):
            edges[i, i + 1] = edges[i + 1, i] = -1
        L = edges + np.diag(-edges.sum(1))
        lam, V = O.jacobi_eigh(L)
        ref = 2 * (1 - np.cos(np.pi * np.arange(n) / n))
        assert np.allclose(lam, np.sort(ref), atol=1e-13)
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
        assert np.allclose(V @ np.diag(lam) @ V.T, L, atol=1e-12)


def test_jacobi_box_kronecker_sum():
    g = box_graph(5, 4, 3)
    lam, _ = O.jacobi_eigh(O.laplacian_dense(g))
    assert np.allclose(lam, O.box_spectrum(5, 4, 3), atol=1e-12)


def test_zero_multiplicity_is_component_count():
    gs = [random_graph(7, 5, s) for s in range(3)] + [box_graph(2, 2, 1)]
    g = disjoint_union(gs)
    lam, _ = O.jacobi_eigh(O.laplacian_dense(g))
    assert int(np.sum(np.abs(lam) < 1e-10)) == 4
    lab = O.components(g)
    assert len(np.unique(lab)) == 4
    # labels are the smallest gid of each component
    off = 0
    for h in gs:
        assert np.all(lab[off:off + h.n] == g.gid[off])
        off += h.n


# ---------------------------------------------------------------- Fiedler solvers


@pytest.mark.parametrize("dims", [(16, 8, 4), (9, 5, 3), (12, 7, 5), (20, 3, 2)])
@pytest.mark.parametrize("method", ["lanczos", "inverse"])
def test_fiedler_box_closed_form(dims, method):
    g = box_graph(*dims)
    lam, v, r = O.fiedler_of_graph(g, O.Options(method=method))
    assert r.converged
    assert abs(lam - O.box_lambda2(*dims)) <= 1e-12 * max(1.0, lam) + 1e-13
    vx = O.box_fiedler_x(*dims)
    assert min(np.abs(v - vx).max(), np.abs(v + vx).max()) < 1e-7
    assert r.resid <= 1e-10 * O.degree(g).max()


def test_box_lambda2_values():
    assert abs(O.box_lambda2(16, 8, 4) - 0.038429439193539) < 1e-14
    assert abs(O.box_lambda2(64, 64, 32) - 0.002409087589655) < 1e-14
    assert abs(O.box_lambda2(32, 16, 16) - 0.009630546655606) < 1e-14


@pytest.mark.parametrize("seed", range(6))
def test_fiedler_random_graph_vs_jacobi(seed):
    g = random_graph(60, 90, 100 + seed)
    lam, V = O.jacobi_eigh(O.laplacian_dense(g))
    assert abs(lam[0]) < 1e-10 and lam[1] > 1e-8
    for method in ("lanczos", "inverse"):
        # inverse iteration contracts by lambda_2 / lambda_3 per outer step
        l2, v, r = O.fiedler_of_graph(g, O.Options(method=method, max_outer=1000))
        assert r.converged
        assert abs(l2 - lam[1]) <= 1e-10 * lam[1]
        if lam[2] - lam[1] > 1e-3 * lam[1]:
            assert min(np.abs(v - V[:, 1]).max(), np.abs(v + V[:, 1]).max()) < 1e-6


def test_weighted_vertex_box_vs_jacobi():
    g = box_graph(6, 5, 4, "vertex")          # 120 elements, 26-neighbour 4/2/1 weights
    lam, V = O.jacobi_eigh(O.laplacian_dense(g))
    for method in ("lanczos", "inverse"):
        l2, v, r = O.fiedler_of_graph(g, O.Options(method=method, max_outer=1000))
        assert abs(l2 - lam[1]) <= 1e-10 * lam[1]
        assert r.resid <= 1e-10 * O.degree(g).max()


def test_lanczos_inverse_agree_on_deleted_mesh():
    g = box_graph_deleted(14, 10, 8, 0.1, 7)
    a = O.fiedler_of_graph(g, O.Options(method="lanczos"))
    b = O.fiedler_of_graph(g, O.Options(method="inverse", max_outer=1000))
    assert abs(a[0] - b[0]) <= 1e-8 * a[0]
    assert np.abs(a[1] - b[1]).max() < 1e-5


def test_planted_solver_mistake_is_caught(monkeypatch):
    """A Lanczos whose fixed basis lacks the constant vector (the projection
    v _|_ 1 of §4 forgotten) converges to the null vector, lambda = 0: the box
    closed form catches it."""
    g = box_graph(9, 5, 3)
    good = O.lanczos_fiedler(g, O.Options()).lam
    assert abs(good - O.box_lambda2(9, 5, 3)) < 1e-10
    import oracle.rsb_oracle as M

    real = M._fixed_basis

    def no_ones(n, deflate):
        B = real(n, deflate)
        return B[:, 1:] if B.shape[1] > 1 else np.zeros((n, 1))

    monkeypatch.setattr(M, "_fixed_basis", no_ones)
    bad = O.lanczos_fiedler(g, O.Options(max_restarts=3)).lam
    assert abs(bad - O.box_lambda2(9, 5, 3)) > 1e-3


@pytest.mark.parametrize("dims", [(16, 8, 4), (16, 16, 8), (12, 12, 12), (20, 9, 7)])
@pytest.mark.parametrize("b", [2, 3, 4])
def test_block_lanczos_box_closed_form(dims, b):
    """Block Lanczos (§9's block extension) reaches lambda_2 = 2 (1 - cos(pi / n_max))
    also where two or three axes are equally long (lambda_2 repeated)."""
    g = box_graph(*dims)
    r = O.block_lanczos_fiedler(g, O.Options(block=b))
    assert r.converged
    assert abs(r.lam - O.box_lambda2(*dims)) < 1e-11
    assert np.linalg.norm(O.laplacian_apply(g, r.v) - r.lam * r.v) <= 1e-10 * O.degree(g).max()


@pytest.mark.parametrize("seed", [11, 12])
def test_block_lanczos_random_graph_vs_jacobi(seed):
    g = random_graph(150, 300, seed)
    lam = O.jacobi_eigh(O.laplacian_dense(g))[0][1]
    for b in (2, 3):
        r = O.block_lanczos_fiedler(g, O.Options(block=b))
        assert r.converged and abs(r.lam - lam) < 1e-10 * max(1.0, lam)


def test_block_lanczos_agrees_with_single_vector_on_deleted_mesh():
    g = box_graph_deleted(14, 11, 9, 0.1, 7, "vertex")
    one = O.lanczos_fiedler(g, O.Options())
    for b in (2, 3, 4):
        r = O.block_lanczos_fiedler(g, O.Options(block=b))
        assert abs(r.lam - one.lam) < 1e-11 * one.lam
        assert min(np.abs(r.v - one.v).max(), np.abs(r.v + one.v).max()) < 1e-6


def test_planted_block_normalisation_mistake_is_caught(monkeypatch):
    """Using the residual block without its Cholesky normalisation leaves S in a
    non-orthonormal basis: the Ritz value misses the closed form."""
    import oracle.rsb_oracle as M

    g = box_graph(16, 8, 4)
    monkeypatch.setattr(M, "_chol_scaled", lambda G, tiny, pmin: np.eye(G.shape[0]))
    with np.errstate(all="ignore"):
        r = O.block_lanczos_fiedler(g, O.Options(block=3, max_restarts=3))
    assert not np.isfinite(r.lam) or abs(r.lam - O.box_lambda2(16, 8, 4)) > 1e-6


def test_amg_galerkin_levels_are_laplacians():
    """J L J^T of a pair aggregation is again a Laplacian (§7): rows sum to zero,
    symmetric, non-positive off the diagonal; the last level is 1 x 1 and zero."""
    g = box_graph_deleted(11, 9, 7, 0.1, 5, "vertex")
    levels = O.amg_hierarchy(O.laplacian_csr(g))
    assert levels[-1][0].shape == (1, 1) and levels[-1][0].toarray()[0, 0] == 0.0
    sizes = [L.shape[0] for L, _ in levels]
    assert all(b == (a + 1) // 2 for a, b in zip(sizes, sizes[1:]))
    for L, _ in levels:
        A = L.toarray()
        assert np.abs(A.sum(axis=1)).max() == 0.0
        assert np.array_equal(A, A.T)
        assert (A - np.diag(np.diag(A)) <= 0).all()


def test_amg_vcycle_converges_as_stationary_iteration():
    g = box_graph(12, 10, 8)
    L = O.laplacian_csr(g)
    levels = O.amg_hierarchy(L)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(g.n)
    b -= b.mean()
    x = np.zeros(g.n)
    res = [np.linalg.norm(b)]
    for _ in range(40):
        x = x + O.vcycle(levels, 0, b - L @ x)
        x -= x.mean()
        res.append(np.linalg.norm(b - L @ x))
    assert res[-1] < 1e-2 * res[0]
    assert all(r1 < r0 for r0, r1 in zip(res, res[1:]))
    # the coarse corrections matter: damped Jacobi alone, with the 5 fine-level
    # sweeps a V-cycle makes (1 + 2 before, 2 after), barely moves the smooth error
    d = 2.0 / 3.0 / L.diagonal()
    xj = np.zeros(g.n)
    for _ in range(40 * 5):
        xj = xj + d * (b - L @ xj)
    assert np.linalg.norm(b - L @ xj) > 10 * res[-1]


def test_amg_fcg_solves_like_cg_with_fewer_iterations():
    g = box_graph(24, 16, 12)
    B = np.ones((g.n, 1)) / np.sqrt(g.n)
    b = O.start_vector(g.gid, 9)
    b -= b.mean()
    b /= np.linalg.norm(b)
    opts = O.Options(cg_tol=1e-11)
    x1, i1 = O.cg_solve(g, b, B, opts)
    x2, i2 = O.fcg_solve(g, b, B, opts)
    assert np.abs(x1 - x2).max() < 1e-8 * np.abs(x1).max()
    assert i2 < i1 / 2
    assert np.linalg.norm(O.laplacian_apply(g, x2) - b) < 1e-10


def test_amg_fcg_first_direction_unpreconditioned():
    """§7: with b an eigenvector of L the flexible CG returns after one iteration."""
    g = box_graph(16, 8, 4)
    lam, v, _ = O.fiedler_of_graph(g)
    B = np.ones((g.n, 1)) / np.sqrt(g.n)
    x, it = O.fcg_solve(g, v, B, O.Options(cg_tol=1e-9))
    assert it == 1
    assert np.abs(x - v / lam).max() < 1e-8 * np.abs(v / lam).max()


@pytest.mark.parametrize("dims", [(16, 8, 4), (12, 7, 5)])
def test_amg_inverse_box_closed_form(dims):
    g = box_graph(*dims)
    r = O.fiedler(g, O.Options(method="inverse", amg=True))
    assert r.converged and abs(r.lam - O.box_lambda2(*dims)) < 1e-11


# ---------------------------------------------------------------- split rules


def test_split_sizes_balanced():
    for N in (7, 100, 131072, 999983):
        for P in (1, 2, 3, 5, 8, 64, 100):
            if P > N:
                continue
            sizes = [O.seg_size(p, p + 1, N, P) for p in range(P)]
            assert sum(sizes) == N and max(sizes) - min(sizes) <= 1


def _split_bruteforce(v, gid, k, tie_rel):
    vk = sorted(v)[k - 1]
    tau = tie_rel * (max(v) - min(v))
    key = [(0 if x < vk - tau else (1 if abs(x - vk) <= tau else 2), g) for x, g in zip(v, gid)]
    order = sorted(range(len(v)), key=lambda i: key[i])
    left = np.zeros(len(v), dtype=bool)
    left[order[:k]] = True
    return left


def test_split_k_bruteforce():
    rng = np.random.default_rng(2)
    for trial in range(300):
        n = int(rng.integers(2, 17))
        vals = rng.integers(-3, 4, size=n).astype(float) + rng.standard_normal(n) * 1e-9
        gid = rng.permutation(1000)[:n]
        k = int(rng.integers(1, n))
        left = O.split_k(vals, gid, k, 1e-5)
        assert left.sum() == k
        assert np.array_equal(left, _split_bruteforce(vals, gid, k, 1e-5))


def test_orient_rule():
    v = np.array([0.1, 0.9, -1.0, 0.3])
    gid = np.array([3, 0, 1, 2])
    # |v| >= 0.5 max: entries 1 (gid 0) and 2 (gid 1); smallest gid 0 has v > 0 -> flip
    assert np.array_equal(O.orient(v, gid), -v)
    assert np.array_equal(O.orient(-v, gid), -v)


def test_quartic_rotation_recovers_axis_vectors():
    g = box_graph(8, 8, 4)
    lam, V = np.linalg.eigh(O.laplacian_dense(g))   # input only: any basis of the cluster
    assert abs(lam[1] - lam[2]) < 1e-12
    U = V[:, 1:3]                                   # the x/y cluster
    th = 0.37
    R = np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]])
    C = O.quartic_rotate(U @ R)
    i = np.arange(g.n) % 8
    j = (np.arange(g.n) // 8) % 8
    for c in range(2):
        col = C[:, c]
        by_i = all(np.ptp(col[i == a]) < 1e-10 for a in range(8))
        by_j = all(np.ptp(col[j == a]) < 1e-10 for a in range(8))
        assert by_i != by_j


def test_partition_spectral_and_bruteforce_bounds():
    for seed in range(5):
        g = random_graph(12, 14, 200 + seed)
        lam = O.jacobi_eigh(O.laplacian_dense(g))[0][1]
        part = O.rsb_partition(g, 2)
        cut = O.partition_metrics(g, part, 2)["weighted_cut"]
        best = min(O.weighted_cut(g, np.isin(np.arange(12), c))
                   for c in itertools.combinations(range(12), 6))
        assert cut >= best
        assert cut >= lam * 6 * 6 / 12 - 1e-9          # cut >= lambda_2 |A||B| / n


def test_partition_metrics_hand_counted():
    """Neighbour counts and cuts of §8's quality metrics on partitions counted by hand."""
    # 4x4x1 face grid cut into its four 2x2 quadrants: every quadrant shares
    # faces with exactly two others (not the diagonal one); 4 + 4 unit edges cross
    g = box_graph(4, 4, 1)
    i, j = np.arange(16) % 4, np.arange(16) // 4
    quad = ((i >= 2) + 2 * (j >= 2)).astype(np.int32)
    m = O.partition_metrics(g, quad, 4)
    assert (m["max_neighbours"], m["avg_neighbours"]) == (2, 2.0)
    assert (m["edge_cut"], m["weighted_cut"]) == (8, 8)
    assert m["sizes"].tolist() == [4, 4, 4, 4]
    # vertex adjacency of the same grid: the diagonal quadrants touch at the
    # centre, so each has three neighbours; 8 face edges (weight 2*2 = 4) and
    # 10 diagonal edges (weight 2) cross a quadrant boundary
    m = O.partition_metrics(box_graph(4, 4, 1, "vertex"), quad, 4)
    assert (m["max_neighbours"], m["avg_neighbours"]) == (3, 3.0)
    assert (m["edge_cut"], m["weighted_cut"]) == (18, 8 * 4 + 10 * 2)
    # a path of six elements in three parts: the middle part has two neighbours
    m = O.partition_metrics(box_graph(6, 1, 1), np.array([0, 0, 1, 1, 2, 2], np.int32), 3)
    assert m["max_neighbours"] == 2 and abs(m["avg_neighbours"] - 4 / 3) < 1e-15
    assert (m["edge_cut"], m["weighted_cut"]) == (2, 2)
    # one part: no neighbours, nothing cut
    m = O.partition_metrics(g, np.zeros(16, np.int32), 1)
    assert (m["max_neighbours"], m["edge_cut"], m["weighted_cut"]) == (0, 0, 0)


def test_planted_neighbour_count_mistake_is_caught(monkeypatch):
    """Counting cut edges per part instead of distinct neighbouring parts fails the pin."""
    import oracle.rsb_oracle as M

    def per_edge(g, part, P):
        r = M.rows_of(g)
        diff = part[r] != part[g.col]
        nbr = np.bincount(part[r][diff], minlength=P)
        return {"max_neighbours": int(nbr.max()), "avg_neighbours": float(nbr.mean())}

    g = box_graph(4, 4, 1)
    i, j = np.arange(16) % 4, np.arange(16) // 4
    quad = ((i >= 2) + 2 * (j >= 2)).astype(np.int32)
    assert per_edge(g, quad, 4)["max_neighbours"] != 2


def test_rcb_box_hand_derived():
    """RCB of the 16x8x4 box into 8 parts, derived by hand: x (extent 15), then
    x again (8x8x4: equal extents 7, lowest axis), then y (4x8x4)."""
    g = box_graph(16, 8, 4)
    i, j = np.arange(512) % 16, (np.arange(512) // 16) % 8
    expect = 4 * (i >= 8) + 2 * ((i % 8) >= 4) + (j >= 4)
    assert np.array_equal(O.rcb_partition(g.centroids(), g.gid, 8), expect)


def test_rcb_bruteforce_and_sizes():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(2, 15))
        pts = rng.random((n, 3))
        gid = rng.permutation(1000)[:n].astype(np.int64)
        part = O.rcb_partition(pts, gid, 2, tie_rel=0.0)
        ax = int(np.argmax(pts.max(0) - pts.min(0)))
        k = n // 2
        order = np.lexsort((gid, pts[:, ax]))
        assert set(np.nonzero(part == 0)[0]) == set(order[:k].tolist())
    for P in (3, 5, 7):
        g = box_graph_deleted(9, 7, 5, 0.1, 2)
        part = O.rcb_partition(g.centroids(), g.gid, P)
        assert np.array_equal(np.bincount(part, minlength=P),
                              [O.seg_size(p, p + 1, g.n, P) for p in range(P)])


def test_rsb_does_not_depend_on_row_order():
    """RSB is defined through gids (start vectors, ties, orientation): a graph
    with its rows permuted gives the same part for every element."""
    from meshgen import permute_graph

    for g in (box_graph(12, 6, 5), box_graph_deleted(10, 8, 6, 0.1, 4, "vertex")):
        h = permute_graph(g, 9)
        a = O.rsb_partition(g, 4, O.Options(degenerate="none"))
        b = O.rsb_partition(h, 4, O.Options(degenerate="none"))
        assert np.array_equal(a[h.meta["perm"]], b)


# ---------------------------------------------------------------- whole recursion


def test_rsb_c1_closed_form():
    g = box_graph(16, 8, 4)
    part = O.rsb_partition(g, 8)
    i, j = np.arange(512) % 16, (np.arange(512) // 16) % 8
    expect = 4 * (i >= 8) + 2 * (j >= 4) + ((i % 8) >= 4)
    assert np.array_equal(part, expect)
    assert np.array_equal(part, O.box_partition_closed_form(16, 8, 4, 8))


@pytest.mark.parametrize("dims,P", [((8, 8, 8), 8), ((12, 6, 4), 4), ((10, 10, 2), 4),
                                    ((16, 16, 8), 16)])
def test_rsb_box_closed_forms(dims, P):
    g = box_graph(*dims)
    assert np.array_equal(O.rsb_partition(g, P), O.box_partition_closed_form(*dims, P))


def test_square_grid_midline_cut():
    """§9: an N x N grid must be cut along a midline (N faces), not at 45 degrees."""
    for N in (8, 12):
        g = box_graph(N, N, 1)
        part = O.rsb_partition(g, 2)
        assert O.partition_metrics(g, part, 2)["edge_cut"] == N
        none = O.rsb_partition(g, 2, O.Options(degenerate="none"))
        assert O.partition_metrics(g, none, 2)["edge_cut"] >= N


def test_disconnected_components_rule():
    a, b, c = box_graph(4, 2, 1), box_graph(3, 2, 1), box_graph(5, 2, 1)
    g = disjoint_union([a, b, c])                  # sizes 8, 6, 10 in gid order
    part = O.rsb_partition(g, 2)                   # left gets 12
    assert np.all(part[:8] == 0)                   # first component fits whole
    assert np.all(part[14:] == 1)                  # last component goes right
    assert part[8:14].sum() == 2                   # straddler split 4 / 2
    assert np.bincount(part).tolist() == [12, 12]


@pytest.mark.parametrize("P", [3, 5, 7, 12])
def test_non_power_of_two_balance(P):
    g = box_graph_deleted(10, 8, 6, 0.1, 3)
    part = O.rsb_partition(g, P, O.Options(degenerate="none"))
    sizes = np.bincount(part, minlength=P)
    assert sizes.sum() == g.n and sizes.max() - sizes.min() <= 1
    assert np.array_equal(sizes, [O.seg_size(p, p + 1, g.n, P) for p in range(P)])


@pytest.mark.skipif(os.environ.get("RSB_SLOW") != "1", reason="about 3 minutes; RSB_SLOW=1")
def test_rsb_c2_closed_form_slow():
    g = box_graph(64, 64, 32)
    part = O.rsb_partition(g, 64)
    i, j, k = np.arange(g.n) % 64, (np.arange(g.n) // 64) % 64, np.arange(g.n) // 4096
    expect = (32 * (j >= 32) + 16 * (i >= 32) + 8 * (k >= 16) + 4 * ((j % 32) >= 16)
              + 2 * ((i % 32) >= 16) + ((k % 16) >= 8))
    assert np.array_equal(part, expect)
