"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every comparison runs the library and the oracle on the same seeded input.
Tolerances: integer work (part ids, sizes, cuts of closed-form boxes) is
bit-exact; the FP64 Laplacian action is exact on integer vectors and within
1e-14 relative otherwise; FP32 within 1e-6; lambda_2 within 1e-6 relative and
residual / ||L|| <= 1e-5 (the stated bar), FP64 solves much tighter.
"""
import numpy as np
import pytest

import oracle as O
from meshgen import box_graph, box_graph_deleted, disjoint_union, random_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2606_14659_gb300 as R  # noqa: E402


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


GRAPHS = {
    "c1_box": lambda: box_graph(16, 8, 4),
    "vertex_13x7x5": lambda: box_graph(13, 7, 5, "vertex"),
    "random_1000": lambda: random_graph(1000, 2500, 11),
    "deleted_18x12x9": lambda: box_graph_deleted(18, 12, 9, 0.1, 5),
    "single_edge": lambda: random_graph(2, 0, 1),
}


# ---------------------------------------------------------------- Laplacian action


@pytest.mark.parametrize("name", list(GRAPHS))
def test_laplacian_f64_integer_exact(name):
    g = GRAPHS[name]()
    x = np.random.default_rng(0).integers(-50, 50, g.n).astype(np.float64)
    y = _np(R.rsb_laplacian_apply(R.graph(g), torch.from_numpy(x).cuda()))
    assert np.array_equal(y, O.laplacian_apply(g, x))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_laplacian_f64_f32_random(name):
    g = GRAPHS[name]()
    x = np.random.default_rng(1).standard_normal(g.n)
    ref = O.laplacian_apply(g, x)
    scale = np.abs(ref).max() + np.abs(x).max() * O.degree(g).max()
    y = _np(R.rsb_laplacian_apply(R.graph(g), torch.from_numpy(x).cuda()))
    assert np.abs(y - ref).max() <= 1e-14 * scale
    x32 = x.astype(np.float32)
    y32 = _np(R.rsb_laplacian_apply(R.graph(g), torch.from_numpy(x32).cuda()))
    assert np.abs(y32 - O.laplacian_apply(g, x32.astype(np.float64))).max() <= 1e-6 * scale


def test_laplacian_host_pointers():
    g = box_graph(9, 7, 5, "vertex")
    x = np.random.default_rng(2).standard_normal(g.n)
    y = R.rsb_laplacian_apply(R.graph(g, device="host"), x)
    assert np.abs(y - O.laplacian_apply(g, x)).max() <= 1e-13


def test_laplacian_ones_and_cut_identity():
    g = box_graph(11, 6, 5, "vertex")
    G = R.graph(g)
    assert np.abs(_np(R.rsb_laplacian_apply(G, torch.ones(g.n, dtype=torch.float64).cuda()))).max() == 0
    s = np.where(np.random.default_rng(3).random(g.n) < 0.5, 1.0, -1.0)
    ls = _np(R.rsb_laplacian_apply(G, torch.from_numpy(s).cuda()))
    assert float(s @ ls) == 4.0 * O.weighted_cut(g, s < 0)


# ---------------------------------------------------------------- Fiedler pair


@pytest.mark.parametrize("method", ["lanczos", "inverse"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dims", [(16, 8, 4), (12, 7, 5)])
def test_fiedler_box(method, precision, dims):
    g = box_graph(*dims)
    lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(method=method, precision=precision))
    assert code == 0
    lam_ref = O.box_lambda2(*dims)
    lo, vo, _ = O.fiedler_of_graph(g, O.Options(method=method))
    dmax = O.degree(g).max()
    if precision == "fp64":
        assert abs(lam - lam_ref) <= 1e-9 * lam_ref
        assert np.abs(_np(v) - vo).max() < 1e-6
        assert res <= 1e-10 * dmax * 1.01
    else:  # FP32 stage + FP64 Rayleigh quotient + short polish: the mixed form's stated bar
        assert abs(lam - lam_ref) <= 1e-6 * lam_ref
        assert np.abs(_np(v) - vo).max() < 1e-4
        assert res <= 1e-5 * dmax


@pytest.mark.parametrize("cycles,dim", [(2, 40), (50, 16)])
def test_fiedler_mixed_polish_reaches_fp64(cycles, dim):
    g = box_graph(12, 7, 5)
    lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(precision="mixed",
                                                             polish_cycles=cycles,
                                                             polish_dim=dim))
    assert abs(lam - O.box_lambda2(12, 7, 5)) <= 1e-10 * O.box_lambda2(12, 7, 5)
    assert res <= 1e-9 * O.degree(g).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dims,tile_rows", [((64, 64, 32), 2), ((64, 64, 32), 4),
                                            ((25, 22, 12), 2), ((128, 128, 96), 2)])
def test_resident_launch_matches_graph_launch_bit_for_bit(precision, dims, tile_rows):
    # launch mode 3 keeps each tile's basis rows in shared memory when the level
    # fits (the 64x64x32 and 25x22x12 boxes), else falls back to graphs (the
    # 128x128x96 box); the steps and their accumulation order are those of the
    # streaming kernels
    G = R.graph(box_graph(*dims))
    ref = R.rsb_fiedler(G, R.options(precision=precision, use_graph=1, tile_rows=tile_rows))
    res = R.rsb_fiedler(G, R.options(precision=precision, use_graph=3, tile_rows=tile_rows))
    assert ref[0] == res[0] and ref[2] == res[2] and ref[3] == res[3]
    assert torch.equal(ref[1], res[1])


def test_mixed_partition_resolves_tied_slab_like_oracle():
    # 9x24x13 -> 16: after the 24-axis split the 13-axis median falls inside the
    # middle slab, whose values tie (cos = 0); the tie must go by gid (R7) as in
    # the oracle.  FP32 vectors alone order that slab by their error instead.
    g = box_graph(9, 24, 13)
    ref = O.rsb_partition(g, 16)
    for prec in ("fp64", "mixed"):
        part, st, code = R.rsb_partition(R.graph(g), 16, R.options(precision=prec))
        assert code == 0
        assert np.array_equal(_np(part), ref), prec


@pytest.mark.parametrize("keep", [0, 4, 8, 16])
def test_thick_restart_sizes_agree_with_oracle(keep):
    g = box_graph(25, 22, 12)
    ref = O.fiedler_of_graph(g, O.Options(keep=keep))
    lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(keep=keep))
    assert abs(lam - ref[0]) <= 1e-9 * ref[0]
    assert np.abs(_np(v) - ref[1]).max() < 1e-6
    if keep:
        assert ref[2].converged and code == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fiedler_random_vs_oracle(seed):
    g = random_graph(300, 700, 40 + seed)
    lam_o, v_o, r_o = O.fiedler_of_graph(g)
    for prec, lt, vt in (("fp64", 1e-9, 1e-5), ("mixed", 1e-6, 1e-3)):
        lam, v, res, code = R.rsb_fiedler(R.graph(g), R.options(precision=prec))
        assert abs(lam - lam_o) <= lt * lam_o
        assert np.abs(_np(v) - v_o).max() < vt
        assert res / O.degree(g).max() <= 1e-5


def test_fiedler_weighted_vs_jacobi():
    g = box_graph(6, 5, 4, "vertex")
    lam, V = O.jacobi_eigh(O.laplacian_dense(g))
    l2, v, res, code = R.rsb_fiedler(R.graph(g))
    assert abs(l2 - lam[1]) <= 1e-10 * lam[1]


def test_fiedler_disconnected():
    g = disjoint_union([box_graph(3, 2, 1), box_graph(4, 2, 1)])
    lam, v, res, code = R.rsb_fiedler(R.graph(g))
    assert code == R.rsb.RSB_EDISCONNECTED and lam == 0.0
    v = _np(v)
    assert abs(v.sum()) < 1e-12 and abs(np.linalg.norm(v) - 1) < 1e-12
    assert v[0] < 0 and np.all(v[:6] == v[0]) and np.all(v[6:] > 0)


# ---------------------------------------------------------------- partitions


def _closed_c1():
    i, j = np.arange(512) % 16, (np.arange(512) // 16) % 8
    return 4 * (i >= 8) + 2 * (j >= 4) + ((i % 8) >= 4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("batched", [1, 0])
@pytest.mark.parametrize("use_graph", [3, 2, 1, 0])
def test_partition_c1_closed_form(precision, batched, use_graph):
    g = box_graph(16, 8, 4)
    part, st, code = R.rsb_partition(R.graph(g), 8, R.options(precision=precision, batched=batched,
                                                               use_graph=use_graph))
    assert code == 0
    assert np.array_equal(_np(part), _closed_c1())
    assert st["levels"] == 3 and st["elements_bisected"] == 3 * 512
    assert abs(st["lambda_first"] - O.box_lambda2(16, 8, 4)) <= 1e-6 * O.box_lambda2(16, 8, 4)


@pytest.mark.parametrize("method", ["lanczos", "inverse"])
def test_partition_c1_methods(method):
    g = box_graph(16, 8, 4)
    part, st, code = R.rsb_partition(R.graph(g), 8, R.options(method=method))
    assert np.array_equal(_np(part), _closed_c1())


@pytest.mark.parametrize("dims,P", [((8, 8, 8), 8), ((12, 6, 4), 4), ((10, 10, 2), 4),
                                    ((16, 16, 8), 16), ((32, 16, 16), 32)])
def test_partition_boxes_closed_form(dims, P):
    g = box_graph(*dims)
    part, st, code = R.rsb_partition(R.graph(g), P)
    assert np.array_equal(_np(part), O.box_partition_closed_form(*dims, P))


def test_partition_host_pointers():
    g = box_graph(16, 8, 4)
    part, st, code = R.rsb_partition(R.graph(g, device="host"), 8)
    assert isinstance(part, np.ndarray) and np.array_equal(part, _closed_c1())


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("P", [2, 3, 5])
def test_partition_random_vs_oracle(seed, P):
    g = random_graph(240, 520, 70 + seed)
    ref = O.rsb_partition(g, P, O.Options(degenerate="none"))
    part, st, code = R.rsb_partition(R.graph(g), P, R.options(degenerate_policy="none"))
    part = _np(part)
    assert np.array_equal(np.bincount(part, minlength=P), np.bincount(ref, minlength=P))
    mr = O.partition_metrics(g, ref, P)["weighted_cut"]
    mg = O.partition_metrics(g, part, P)["weighted_cut"]
    assert mg <= 1.02 * mr
    assert np.mean(part == ref) > 0.95


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_launch_partitions_equal_resident_on_unaligned_units(precision):
    # an irregular mesh split 7 ways and a batch of odd-sized boxes: from the
    # second level on, units start at arbitrary rows, so the bulk copies of the
    # graph launch start inside a 16-byte group and end on ragged chunks; the
    # staged kernels must reproduce the resident kernel bit for bit
    g = box_graph_deleted(23, 17, 11, 0.07, 5, "vertex")
    res = R.rsb_partition(R.graph(g), 7, R.options(precision=precision, use_graph=3))[0]
    gra = R.rsb_partition(R.graph(g), 7, R.options(precision=precision, use_graph=1))[0]
    assert np.array_equal(_np(res), _np(gra))
    gs = [R.graph(box_graph(*d)) for d in [(7, 5, 3), (9, 13, 5), (11, 3, 7), (6, 6, 6)]]
    res = R.rsb_partition_batch(gs, [5, 3, 6, 7], R.options(precision=precision, use_graph=3))[0]
    gra = R.rsb_partition_batch(gs, [5, 3, 6, 7], R.options(precision=precision, use_graph=1))[0]
    for a, b in zip(res, gra):
        assert np.array_equal(_np(a), _np(b))


def test_partition_disconnected_vs_oracle():
    g = disjoint_union([box_graph(4, 2, 1), box_graph(3, 2, 1), box_graph(5, 2, 1),
                        random_graph(9, 6, 3)])
    for P in (2, 3, 4):
        ref = O.rsb_partition(g, P)
        part, st, code = R.rsb_partition(R.graph(g), P)
        assert np.array_equal(_np(part), ref)


def test_partition_deleted_mesh_inverse_vs_oracle():
    g = box_graph_deleted(20, 14, 10, 0.1, 9)
    opts_o = O.Options(method="inverse", degenerate="none")
    ref = O.rsb_partition(g, 8, opts_o)
    mr = O.partition_metrics(g, ref, 8)
    for prec in ("fp64", "mixed"):
        part, st, code = R.rsb_partition(
            R.graph(g), 8, R.options(method="inverse", precision=prec, degenerate_policy="none"))
        m = O.partition_metrics(g, _np(part), 8)
        assert np.array_equal(m["sizes"], mr["sizes"])
        assert m["weighted_cut"] <= 1.02 * mr["weighted_cut"]
        lam_o = O.fiedler_of_graph(g, opts_o)[0]
        assert abs(st["lambda_first"] - lam_o) <= 1e-6 * lam_o


def test_batch_equals_separate_calls_and_closed_form():
    dims = [(16, 8, 4), (8, 8, 8), (12, 6, 4), (10, 10, 2)]
    P = [8, 8, 4, 4]
    gs = [box_graph(*d) for d in dims]
    parts, st, code = R.rsb_partition_batch([R.graph(g) for g in gs], P)
    for g, d, p, out in zip(gs, dims, P, parts):
        alone, _, _ = R.rsb_partition(R.graph(g), p)
        assert np.array_equal(_np(out), _np(alone))
        assert np.array_equal(_np(out), O.box_partition_closed_form(*d, p))


def test_edge_cases():
    g = box_graph(5, 3, 2)
    part, st, code = R.rsb_partition(R.graph(g), 1)
    assert np.all(_np(part) == 0) and st["levels"] == 0
    part, st, code = R.rsb_partition(R.graph(g), g.n)
    assert np.array_equal(np.sort(_np(part)), np.arange(g.n))
    g2 = random_graph(2, 0, 1)
    part, _, _ = R.rsb_partition(R.graph(g2), 2)
    assert _np(part).tolist() == [0, 1]
    with pytest.raises(R.RSBError):
        R.rsb_partition(R.graph(g), 0)
    with pytest.raises(R.RSBError):
        R.rsb_partition(R.graph(g), g.n + 1)


def test_invalid_graphs_rejected():
    g = box_graph(4, 3, 2)
    bad = box_graph(4, 3, 2)
    bad.col = bad.col.copy()
    bad.col[0] = g.n + 5
    with pytest.raises(R.RSBError) as e:
        R.rsb_partition(R.graph(bad), 2)
    assert e.value.code == R.rsb.RSB_EINVAL
    bad = box_graph(4, 3, 2)
    bad.w = bad.w.copy()
    bad.w[3] = 0
    with pytest.raises(R.RSBError):
        R.rsb_partition(R.graph(bad), 2)
    bad = box_graph(4, 3, 2)
    bad.col = bad.col.copy()
    bad.col[0] = 0
    with pytest.raises(R.RSBError):
        R.rsb_partition(R.graph(bad), 2)
    asym = box_graph(4, 3, 2)
    asym.w = asym.w.copy()
    asym.w[0] = 2
    with pytest.raises(R.RSBError):
        R.rsb_partition(R.graph(asym), 2, R.options(validate=1))


# ---------------------------------------------------------------- full-size boxes


def _closed_c2():
    n = np.arange(64 * 64 * 32)
    i, j, k = n % 64, (n // 64) % 64, n // 4096
    return (32 * (j >= 32) + 16 * (i >= 32) + 8 * (k >= 16) + 4 * ((j % 32) >= 16)
            + 2 * ((i % 32) >= 16) + ((k % 16) >= 8))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("use_graph", [3, 2, 1])
def test_partition_c2_closed_form(precision, use_graph):
    g = box_graph(64, 64, 32)
    part, st, code = R.rsb_partition(R.graph(g), 64, R.options(precision=precision,
                                                                use_graph=use_graph))
    assert np.array_equal(_np(part), _closed_c2())
    assert st["levels"] == 6
    assert abs(st["lambda_first"] - O.box_lambda2(64, 64, 32)) <= 1e-6 * O.box_lambda2(64, 64, 32)


def test_autotune_picks_a_candidate_and_keeps_results():
    g = box_graph(64, 64, 32)
    G = R.graph(g)
    base = R.options(precision="mixed")
    tuned, ms = R.rsb_autotune([G], [64], base)
    assert (tuned.tile_rows, tuned.use_graph) in ms
    assert all(np.isfinite(v) and v > 0 for v in ms.values())
    assert ms[(tuned.tile_rows, tuned.use_graph)] == min(ms.values())
    for f, _ in R.rsb.rsb_options._fields_:
        if f not in ("tile_rows", "use_graph"):
            assert getattr(tuned, f) == getattr(base, f), f
    part, st, code = R.rsb_partition(G, 64, tuned)
    assert code == 0 and np.array_equal(_np(part), _closed_c2())
