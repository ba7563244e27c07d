"""FP64 CPU oracle for recursive spectral bisection — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The CUDA product path never does.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force or the paper's worked example, except the
weighted 26-neighbour Fiedler pair at sizes above a dense solve, which is
"parity unpinned" by any closed form and is held only by the residual, the
Lanczos / inverse-iteration agreement and the spectral cut bound.
"""
from .rsb_oracle import (  # noqa: F401
    Options, FiedlerResult, rows_of, degree, laplacian_apply, laplacian_dense, induced,
    components, jacobi_eigh, splitmix64, start_vector, adjacency_csr,
    lanczos_fiedler, block_lanczos_fiedler, inverse_fiedler, cg_solve, fiedler, orient, split_k,
    weighted_cut, quartic_rotate, fiedler_candidates, split_connected, bisect,
    seg_size, rsb_partition, fiedler_of_graph, partition_metrics, rcb_partition,
)
from .amg import (  # noqa: F401
    laplacian_csr, amg_hierarchy, vcycle, fcg_solve, amg_inverse_fiedler,
)
from .gather_scatter import (  # noqa: F401
    gs_operators, gs_adjacency_apply, gs_laplacian_apply, dual_graph_from_vertices,
)
from .box_closed_form import (  # noqa: F401
    NotClean, box_lambda2, box_spectrum, box_fiedler_x, box_partition_closed_form,
)
