"""Failure path of the bounded device waits.

The persistent launch modes synchronise their CTAs with a grid barrier whose
wait is bounded by the GPU's global timer.  The test hook starts the barrier
from an arrival count that never completes (a flag nothing sets): the call
must come back with RSB_ETIMEOUT after the bound, not hang, and the next call
must start from a clean barrier and give the usual result.  No GPU fault is
involved.
"""
import time

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2606_14659_gb300 as R  # noqa: E402
from meshgen import box_graph  # noqa: E402


@pytest.mark.parametrize("use_graph", [3, 2])
def test_grid_barrier_timeout_returns_error_then_recovers(use_graph):
    G = R.graph(box_graph(16, 8, 4))
    opts = R.options(use_graph=use_graph)
    ref = R.rsb_fiedler(G, opts)
    R.rsb.rsb_test_poison_barrier(True)
    try:
        t0 = time.time()
        with pytest.raises(R.RSBError) as err:
            R.rsb_fiedler(G, opts)
        assert err.value.code == R.rsb.RSB_ETIMEOUT
        assert time.time() - t0 < 60
    finally:
        R.rsb.rsb_test_poison_barrier(False)
    again = R.rsb_fiedler(G, opts)
    assert again[0] == ref[0] and again[3] == ref[3]
    assert torch.equal(again[1], ref[1])
