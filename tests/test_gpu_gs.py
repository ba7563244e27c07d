"""Element -> vertex ids through the C ABI: the dual graph built on the GPU and
the matrix-free (gather-scatter) Laplacian of §5, against the oracle.

The dual graph is integer work, so it must equal the oracle's
P^T Q Q^T P (without its diagonal) and the generator's vertex-adjacency graph
entry for entry.  The gather-scatter action in FP64 is exact on integer
vectors; on real vectors it is held to 1e-13 d_max |x| (FP64) and to
2e-6 d_max |x| (FP32: c_v x_e - w_v differs from the sum of differences by
the rounding of the vertex sums w_v, at most about 8 units of FP32 rounding of
|x| per vertex term).
"""
import os

import numpy as np
import pytest

import oracle as O
from meshgen import box_graph, box_graph_deleted

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2606_14659_gb300 as R  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig2_gather_scatter.txt")


def _fig2_lists():
    lines = [ln.split("#")[0].strip() for ln in open(GOLDEN)]
    lines = [ln for ln in lines if ln]
    i = lines.index("vertex_lists")
    return np.array([[int(t) for t in lines[i + 1 + r].split()] for r in range(3)])


@pytest.mark.parametrize("g", [box_graph(7, 5, 4, "vertex"),
                               box_graph_deleted(20, 14, 9, 0.1, 3, "vertex"),
                               box_graph_deleted(64, 48, 40, 0.05, 11, "vertex")])
@pytest.mark.parametrize("where", ["cuda", "host"])
def test_dual_graph_equals_generator_and_oracle(g, where):
    ev = g.hex_vertices()
    n, rp, col, w = R.rsb.rsb_dual_graph(ev, device=where)
    rp, col, w = (a.cpu().numpy() if hasattr(a, "cpu") else a for a in (rp, col, w))
    assert n == g.n
    assert np.array_equal(rp, g.row_ptr)
    assert np.array_equal(col, g.col) and np.array_equal(w, g.w)
    if g.n < 5000:
        h = O.dual_graph_from_vertices(ev)
        assert np.array_equal(h.col, col) and np.array_equal(h.w, w)


def test_dual_graph_fig2():
    """The paper's three quads: weights 2, 2, 1 (shared vertices)."""
    ev = _fig2_lists()
    n, rp, col, w = R.rsb.rsb_dual_graph(ev)
    assert rp.cpu().tolist() == [0, 2, 4, 6]
    assert col.cpu().tolist() == [1, 2, 0, 2, 0, 1]
    assert w.cpu().tolist() == [2, 2, 2, 1, 2, 1]


@pytest.mark.parametrize("g", [box_graph(9, 7, 5, "vertex"),
                               box_graph_deleted(40, 32, 24, 0.1, 20262, "vertex")])
def test_gather_scatter_laplacian_vs_oracle(g):
    ev = torch.from_numpy(g.hex_vertices()).cuda()
    rng = np.random.default_rng(2)
    xi = rng.integers(-7, 8, g.n).astype(np.float64)
    y = R.rsb.rsb_laplacian_apply_gs(ev, torch.from_numpy(xi).cuda()).cpu().numpy()
    assert np.array_equal(y, O.gs_laplacian_apply(g.hex_vertices(), xi))
    assert np.array_equal(y, O.laplacian_apply(g, xi))
    dmax = O.degree(g).max()
    xr = rng.standard_normal(g.n)
    ref = O.laplacian_apply(g, xr)
    y = R.rsb.rsb_laplacian_apply_gs(ev, torch.from_numpy(xr).cuda()).cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-13 * dmax * np.abs(xr).max()
    y32 = R.rsb.rsb_laplacian_apply_gs(ev, torch.from_numpy(xr.astype(np.float32)).cuda())
    assert np.abs(y32.cpu().numpy() - ref).max() <= 2e-6 * dmax * np.abs(xr).max()


def test_partition_from_gpu_built_graph():
    g = box_graph_deleted(24, 20, 16, 0.1, 7, "vertex")
    n, rp, col, w = R.rsb.rsb_dual_graph(g.hex_vertices())
    G = R.Graph(n, rp, col, w, torch.from_numpy(g.gid).cuda(), "cuda")
    a, _, ca = R.rsb_partition(G, 8, R.options(precision="mixed"))
    b, _, cb = R.rsb_partition(R.graph(g), 8, R.options(precision="mixed"))
    assert ca == cb == 0
    assert torch.equal(a, b)


def test_dual_graph_rejects_bad_input():
    lib = R.rsb.load()
    ev = torch.tensor([[0, 1, 2, 3], [2, 3, -1, 5]], dtype=torch.int64, device="cuda")
    with pytest.raises(R.RSBError):
        R.rsb.rsb_dual_graph(ev)
    ev = torch.tensor([[0, 1, 2, 3], [2, 3, 4, 5]], dtype=torch.int64, device="cuda")
    import ctypes as C

    rp = torch.empty(3, dtype=torch.int64, device="cuda")
    col = torch.empty(1, dtype=torch.int32, device="cuda")
    w = torch.empty(1, dtype=torch.int32, device="cuda")
    nnz = C.c_int64(0)
    code = lib.rsb_dual_graph(2, 4, ev.data_ptr(), rp.data_ptr(), col.data_ptr(), w.data_ptr(),
                              1, C.byref(nnz), None)
    assert code == R.rsb.RSB_EINVAL and nnz.value == 2
    assert rp.cpu().tolist() == [0, 1, 2]
