"""AMG-preconditioned flexible CG for inverse iteration (§7) through the C ABI.

The preconditioner changes how fast the inner solves converge, not what inverse
iteration converges to: lambda_2 and the partitions must be those of plain CG
(closed forms on boxes, the oracle's values on irregular meshes), and the
V-cycle must do its job (the flexible CG needs fewer iterations than plain CG
on a 3-D mesh; the oracle's own AMG-FCG needs 3.5-4x fewer).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from meshgen import box_graph, box_graph_deleted, permute_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2606_14659_gb300 as R  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "irregular_medium.json")))


@pytest.mark.parametrize("dims", [(16, 8, 4), (20, 9, 7), (32, 16, 16)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_amg_fiedler_box_closed_form(dims, prec):
    g = box_graph(*dims)
    lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(method="inverse", amg=1,
                                                            precision=prec))
    assert code == 0
    lam_cf = O.box_lambda2(*dims)
    assert abs(lam - lam_cf) <= 1e-9 * lam_cf, (lam, lam_cf)


@pytest.mark.parametrize("reorder", [0, 1])
def test_amg_partition_box_closed_form(reorder):
    g = box_graph(32, 16, 8)
    h = permute_graph(g, 3)
    part, st, code = R.rsb_partition(R.graph(h), 16, R.options(method="inverse", amg=1,
                                                               precision="mixed",
                                                               reorder=reorder))
    assert code == 0
    assert np.array_equal(part.cpu().numpy(), O.box_partition_closed_form(32, 16, 8, 16)[h.meta["perm"]])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_amg_irregular_vs_oracle(prec):
    m = GOLD["meshes"][0]
    g = box_graph_deleted(*m["dims"], m["frac"], m["seed"], m["adjacency"])
    G = R.graph(g)
    o = R.options(method="inverse", amg=1, precision=prec, degenerate_policy="none")
    lam, v, res, code = R.rsb_fiedler(G, o)
    assert code == 0
    assert abs(lam - m["lambda2"]) <= 1e-6 * m["lambda2"]
    part, st, code = R.rsb_partition(G, 16, o)
    assert code == 0
    part = part.cpu().numpy()
    ref = m["runs"]["inverse/none"]["weighted_cut_16"]
    cut = O.partition_metrics(g, part, 16)["weighted_cut"]
    assert abs(cut - ref) <= 0.02 * ref


def test_amg_reduces_inner_iterations():
    g = box_graph_deleted(48, 40, 32, 0.05, 8, "vertex")
    G = R.graph(g)
    plain = R.rsb_partition(G, 2, R.options(method="inverse", precision="fp64",
                                            degenerate_policy="none"))[1]
    amg = R.rsb_partition(G, 2, R.options(method="inverse", amg=1, precision="fp64",
                                          degenerate_policy="none", reorder=1))[1]
    assert amg["inner"] < plain["inner"] / 2, (amg["inner"], plain["inner"])
    assert abs(amg["lambda_first"] - plain["lambda_first"]) <= 1e-9 * plain["lambda_first"]


def test_amg_c3_first_split_vs_oracle():
    """The 192x128x96 mesh with 10 % deleted, in RCB order, first split by
    AMG-FCG inverse iteration: the oracle's lambda_2 and cut (stored by
    tests/golden/make_golden.py)."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c3_levels01.json")))
    g = box_graph_deleted(192, 128, 96, 0.10, 20260, "vertex")
    o = R.options(method="inverse", amg=1, precision="mixed", degenerate_policy="none",
                  reorder=1, polish_cycles=8)
    part, st, code = R.rsb_partition(R.graph(g), 2, o)
    assert code == 0
    lam0 = gold["splits"][0]["lambda2"]
    assert abs(st["lambda_first"] - lam0) <= 1e-6 * lam0, (st["lambda_first"], lam0)
    cut = O.weighted_cut(g, part.cpu().numpy() == 0)
    assert abs(cut - gold["weighted_cut_2"]) <= 0.02 * gold["weighted_cut_2"]
