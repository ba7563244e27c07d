"""rsb_laplacian_apply_noalloc against rsb_laplacian_apply and the oracle.

The no-allocation entry point serves callers that cannot call cudaMalloc (a
framework's caching allocator holds the device, a region where the implicit
synchronisation of cudaMalloc/cudaFree is not allowed, or an embedder that
budgets every device byte).  It must give the same y = L x as the allocating
entry point, call after call, although every call reuses one static device
array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from meshgen import box_graph, box_graph_deleted, random_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_2606_14659_gb300 as R  # noqa: E402


def _apply_both(g, x):
    G = R.graph(g)
    xd = torch.from_numpy(x).cuda()
    ref = R.rsb_laplacian_apply(G, xd).cpu().numpy()
    y = torch.full((g.n,), np.nan, dtype=torch.float64, device="cuda")
    code = R.rsb.rsb_laplacian_apply_noalloc(G, xd, y)
    assert code == 0, R.rsb.load().rsb_last_error_detail()
    return y.cpu().numpy(), ref


def test_noalloc_matches_allocating_entry_two_calls():
    rng = np.random.default_rng(7)
    # two different graphs back to back: the second call must not see the first's scratch
    for g in (box_graph(40, 30, 20, "vertex"), box_graph_deleted(25, 19, 13, 0.1, 3)):
        xi = rng.integers(-9, 9, g.n).astype(np.float64)
        y, ref = _apply_both(g, xi)
        assert np.array_equal(y, ref)                  # integer vectors: exact
        assert np.array_equal(y, O.laplacian_apply(g, xi))
        xr = rng.standard_normal(g.n)
        y, ref = _apply_both(g, xr)
        scale = np.abs(xr).max() * 56.0
        assert np.abs(y - ref).max() <= 1e-14 * scale


def test_noalloc_rejects_oversized_and_host_inputs():
    lib = R.rsb.load()
    g = box_graph(160, 160, 80, "vertex")              # ~2M rows, far above 32 MiB of scratch
    G = R.graph(g)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    assert R.rsb.rsb_laplacian_apply_noalloc(G, x, y) == R.rsb.RSB_EINVAL
    assert b"32 MiB" in lib.rsb_last_error_detail()
    small = random_graph(50, 80, 1)
    Gh = R.graph(small, device="host")
    xh = np.zeros(small.n)
    yh = np.zeros(small.n)
    assert R.rsb.rsb_laplacian_apply_noalloc(Gh, xh, yh) == R.rsb.RSB_EINVAL
    # a valid call still works after the rejections
    y2, ref = _apply_both(small, np.arange(small.n, dtype=np.float64))
    assert np.array_equal(y2, ref)
