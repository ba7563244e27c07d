"""Recursive coordinate bisection and the RCB reordering through the C ABI.

RCB is the geometric partitioner the paper runs before RSB (§5, §8: it
organises the elements into contiguous subsets; Lanczos ran about twice as
fast after it).  Here it is both a method of its own (method = rcb, compared
with the oracle's rcb_partition bit for bit: its decisions are comparisons of
exact coordinates and gids) and a reordering of the elements before the
spectral recursion (reorder = 1), which must not change the partition: RSB is
defined through gids, so a graph whose rows arrive in a random order, reordered
by RCB or not, must give every element the same part (bit for bit on
closed-form boxes; on irregular meshes the summation order of the Laplacian
changes, so sizes exactly and the cut within 2 %).
"""
import numpy as np
import pytest

import oracle as O
from meshgen import box_graph, box_graph_deleted, permute_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2606_14659_gb300 as R  # noqa: E402


@pytest.mark.parametrize("g,P", [(box_graph(16, 8, 4), 8), (box_graph(9, 24, 13), 16),
                                 (box_graph_deleted(20, 14, 9, 0.1, 3, "vertex"), 7),
                                 (box_graph_deleted(40, 32, 24, 0.1, 20262, "vertex"), 64)])
def test_rcb_matches_oracle(g, P):
    part, st, code = R.rsb_partition(R.graph(g), P, R.options(method="rcb"))
    assert code == 0
    ref = O.rcb_partition(g.centroids(), g.gid, P)
    assert np.array_equal(part.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_reorder_permuted_box_gives_closed_form(prec):
    g = box_graph(32, 16, 8)
    h = permute_graph(g, 17)
    cf = O.box_partition_closed_form(32, 16, 8, 16)
    for reorder in (0, 1):
        part, st, code = R.rsb_partition(R.graph(h), 16, R.options(precision=prec,
                                                                   reorder=reorder))
        assert code == 0
        assert np.array_equal(part.cpu().numpy(), cf[h.meta["perm"]]), reorder


def test_reorder_natural_order_and_batch():
    gs = [box_graph(16, 8, 4), box_graph(24, 12, 6), box_graph(16, 16, 8)]
    P = [8, 8, 16]
    parts, _, code = R.rsb_partition_batch([R.graph(g) for g in gs], P,
                                           R.options(precision="mixed", reorder=1))
    assert code == 0
    for g, p, k in zip(gs, parts, P):
        assert np.array_equal(p.cpu().numpy(), O.box_partition_closed_form(*g.dims, k))


def test_reorder_irregular_permuted_mesh():
    g = box_graph_deleted(40, 32, 24, 0.1, 20262, "vertex")
    h = permute_graph(g, 5)
    P = 16
    base, _, c0 = R.rsb_partition(R.graph(g), P, R.options(precision="mixed"))
    re, _, c1 = R.rsb_partition(R.graph(h), P, R.options(precision="mixed", reorder=1))
    assert c0 == 0 and c1 == 0
    re = re.cpu().numpy()
    sizes = np.bincount(re, minlength=P)
    assert np.array_equal(sizes, [O.seg_size(p, p + 1, g.n, P) for p in range(P)])
    cut_base = O.partition_metrics(g, base.cpu().numpy(), P)["weighted_cut"]
    cut_re = O.partition_metrics(h, re, P)["weighted_cut"]
    assert abs(cut_re - cut_base) <= 0.02 * cut_base


def test_rcb_needs_coords():
    g = box_graph(8, 4, 4)
    G = R.graph(g)
    G.coords = None
    with pytest.raises(R.RSBError) as err:
        R.rsb_partition(G, 4, R.options(method="rcb"))
    assert err.value.code == R.rsb.RSB_EINVAL
    with pytest.raises(R.RSBError):
        R.rsb_partition(G, 4, R.options(reorder=1))
