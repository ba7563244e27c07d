"""Seeded synthetic inputs for recursive spectral bisection.

This package builds the element dual graphs that both the CUDA path and the
CPU oracle consume.  It holds no arithmetic of the partitioning method itself:
only mesh geometry (which hex elements touch and how many vertices they share),
seeded element deletion, largest-connected-component extraction and CSR
packing.
"""
from .boxes import (  # noqa: F401
    DualGraph,
    splitmix64,
    box_graph,
    box_graph_deleted,
    batch_box_dims,
    random_graph,
    disjoint_union,
    quad_vertex_lists_dual,
    permute_graph,
)
