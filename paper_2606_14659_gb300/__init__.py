"""GB300-native Recursive Spectral Bisection (RSB) of element dual graphs.

The compute path is the CUDA library librsb.so (csrc/, C ABI in include/rsb.h);
``rsb`` is its ctypes binding.  Build with ``paper_2606_14659_gb300.build``.
"""
from . import rsb  # noqa: F401
from .rsb import (  # noqa: F401
    Graph, graph, options, rsb_partition, rsb_partition_batch, rsb_fiedler,
    rsb_laplacian_apply, rsb_laplacian_bench, rsb_release, RSBError, rsb_profile_begin,
    rsb_profile_end, rsb_profile_read, rsb_autotune,
)
