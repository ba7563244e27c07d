"""Block Lanczos (width 2-4) through the C ABI against closed forms and the oracle.

Block Lanczos is the extension §9 names for a nearly repeated lambda_2: a block
of b vectors per step converges a cluster of b eigenvalues at the rate of the
gap to the rest of the spectrum.  Its answers must be those of the method it
stands in for: lambda_2 of boxes in closed form (2 (1 - cos(pi / n_max)), also
when two or three axes have equal length), the closed-form partitions of boxes,
the oracle's lambda_2 and cut on irregular meshes (within the bars of the
single-vector path), and results that do not depend on what else is in the
batch.
"""
import json
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

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "irregular_medium.json")))


@pytest.mark.parametrize("dims", [(16, 8, 4), (16, 16, 8), (12, 12, 12), (20, 9, 7)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("bw", [2, 3, 4])
def test_block_fiedler_box_closed_form(dims, prec, bw):
    g = box_graph(*dims)
    lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(precision=prec, block=bw))
    assert code == 0
    lam_cf = O.box_lambda2(*dims)
    assert abs(lam - lam_cf) <= 1e-9 * lam_cf, (lam, lam_cf)
    v = v.cpu().numpy()
    assert np.linalg.norm(O.laplacian_apply(g, v) - lam * v) <= 1e-6 * O.degree(g).max()


@pytest.mark.parametrize("dims,P,bw", [((16, 8, 4), 8, 2), ((16, 16, 8), 16, 2),
                                       ((24, 12, 6), 8, 2), ((64, 64, 32), 64, 2),
                                       ((16, 8, 4), 8, 3), ((16, 16, 8), 16, 3),
                                       ((24, 12, 6), 8, 3), ((32, 16, 16), 32, 4)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_block_partition_box_closed_form(dims, P, prec, bw):
    """(On the exactly repeated lambda_2 of a clean box a block of 3 has a lower
    Krylov degree per cycle than the single vector and needs more cycles; at
    the FP64 tolerance the 64x64x32 box reaches the cap of 50 restarts with
    width 3, so it runs with width 2.)"""
    g = box_graph(*dims)
    part, st, code = R.rsb_partition(R.graph(g), P, R.options(precision=prec, block=bw))
    assert code == 0
    assert np.array_equal(part.cpu().numpy(), O.box_partition_closed_form(*dims, P))


@pytest.mark.parametrize("i", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("bw", [2, 3])
def test_block_irregular_vs_oracle(i, prec, bw):
    m = GOLD["meshes"][i]
    g = box_graph_deleted(*m["dims"], m["frac"], m["seed"], m["adjacency"])
    G = R.graph(g)
    o = R.options(precision=prec, block=bw, degenerate_policy="none")
    lam, v, res, code = R.rsb_fiedler(G, o)
    assert code == 0
    assert abs(lam - m["lambda2"]) <= 1e-6 * m["lambda2"]
    v = v.cpu().numpy()
    assert np.linalg.norm(O.laplacian_apply(g, v) - lam * v) <= 1e-5 * m["dmax"]
    part, st, code = R.rsb_partition(G, m["parts"], o)
    assert code == 0
    part = part.cpu().numpy()
    P = m["parts"]
    assert np.array_equal(np.bincount(part, minlength=P),
                          [O.seg_size(p, p + 1, g.n, P) for p in range(P)])
    ref = m["runs"]["lanczos/none"]["weighted_cut_16"]
    cut = O.partition_metrics(g, part, P)["weighted_cut"]
    assert abs(cut - ref) <= 0.02 * ref, (cut, ref)


@pytest.mark.parametrize("bw", [2, 3])
def test_block_near_triple_cluster_vs_oracle(bw):
    """A cube with 5 % deleted: lambda_2..lambda_4 nearly equal.  The block
    solve in mixed precision must land on the oracle's lambda_2."""
    g = box_graph_deleted(24, 24, 24, 0.05, 20261, "vertex")
    lam_o = O.fiedler(g, O.Options(block=1)).lam
    lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(precision="mixed", block=bw))
    assert code == 0
    assert abs(lam - lam_o) <= 1e-6 * lam_o, (lam, lam_o)
    lam_ob = O.fiedler(g, O.Options(block=bw)).lam
    assert abs(lam_ob - lam_o) <= 1e-9 * lam_o


def test_block_batch_equals_separate_calls():
    gs = [box_graph(16, 8, 4), box_graph_deleted(20, 18, 9, 0.1, 5, "vertex"), box_graph(9, 24, 13)]
    o = R.options(precision="mixed", block=3)
    parts, _, _ = R.rsb_partition_batch([R.graph(g) for g in gs], [8] * len(gs), o)
    for g, p in zip(gs, parts):
        alone, _, _ = R.rsb_partition(R.graph(g), 8, o)
        assert np.array_equal(p.cpu().numpy(), alone.cpu().numpy())


def test_block_small_units_fall_back_to_single_vector():
    """Subgraphs with fewer than krylov_dim + b dimensions use the single-vector
    method in the same level; the result equals the single-vector run there."""
    g = box_graph(10, 6, 4)  # 240 elements -> 12 parts: units of 20..120 rows
    a, _, ca = R.rsb_partition(R.graph(g), 12, R.options(block=3))
    b, _, cb = R.rsb_partition(R.graph(g), 12, R.options(block=1))
    assert ca == 0 and cb == 0
    sizes = np.bincount(a.cpu().numpy(), minlength=12)
    assert np.array_equal(sizes, [O.seg_size(p, p + 1, g.n, 12) for p in range(12)])
    mt_a = O.partition_metrics(g, a.cpu().numpy(), 12)["weighted_cut"]
    mt_b = O.partition_metrics(g, b.cpu().numpy(), 12)["weighted_cut"]
    assert mt_a == mt_b
