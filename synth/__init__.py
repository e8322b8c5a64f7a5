"""Seeded synthetic graph generators shared by the tests, the bench and the oracle checks.

This package holds input recipes only (random graph models, planted blocks, weight
grids).  It contains none of the densest-subgraph method's arithmetic, and neither the
CUDA library nor the CPU oracle imports it: callers generate a graph here and hand the
same arrays to both sides.
"""
from .graphs import (  # noqa: F401
    Graph,
    WEIGHT_GRID_BITS,
    quantise_weights,
    chung_lu,
    rmat,
    erdos_renyi,
    planted_background,
    small_family,
    workload,
    WORKLOADS,
    batch_graph,
    batch,
)
