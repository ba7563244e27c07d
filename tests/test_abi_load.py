"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(rsb.h: the method's calls; rsb_test.h: measurement and test hooks).

CPU only: no compute call is made here.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(headers=None):
    inc = os.path.join(ROOT, "include")
    names = set()
    for h in headers or sorted(f for f in os.listdir(inc) if f.endswith(".h")):
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
        names |= set(re.findall(r"\b(rsb_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared(["rsb.h"])
    for n in ("rsb_partition", "rsb_partition_batch", "rsb_fiedler", "rsb_strerror",
              "rsb_options_default", "rsb_release", "rsb_laplacian_apply"):
        assert n in names
    hooks = _declared(["rsb_test.h"])
    assert set(hooks) == {"rsb_profile_begin", "rsb_profile_end", "rsb_profile_read",
                         "rsb_test_poison_barrier"}
    assert not set(hooks) & set(names)


def test_library_exports_every_declared_symbol():
    from paper_2606_14659_gb300 import build as B

    try:
        path = B.build()
    except Exception as e:  # pragma: no cover
        pytest.fail(f"build failed: {e}")
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_struct_layout_and_strerror():
    import paper_2606_14659_gb300.rsb as R

    lib = R.load()
    assert ctypes.sizeof(R.rsb_options) == 120 and R.rsb_options.block.offset == 108
    assert R.rsb_options.amg.offset == 116
    assert R.rsb_options.reorder.offset == 112 and ctypes.sizeof(R.rsb_csr) == 48
    assert R.rsb_options.keep.offset == 96 and R.rsb_options.tile_rows.offset == 100
    assert R.rsb_options.polish_dim.offset == 104
    assert R.rsb_options.polish_cycles.offset == 92 and R.rsb_options.seed.offset == 40
    assert ctypes.sizeof(R.rsb_stats) == 72
    assert lib.rsb_strerror(0) == b"success"
    assert lib.rsb_strerror(R.RSB_EDISCONNECTED) == b"graph is disconnected"
    o = R.options(method="inverse", precision="mixed")
    assert o.method == 1 and o.precision == 1 and o.krylov_dim == 40 and o.max_restarts == 50
    for name in R.EXPORTED:
        assert name in _declared()
