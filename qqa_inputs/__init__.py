"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and bench.py.

This package holds graph generators and workload recipes only: no step of the
annealing method is computed here. Both sides of every parity test take their
graphs (and nothing else) from here.
"""
from .graphs import (  # noqa: F401
    CSRGraph,
    from_edges,
    erdos_renyi,
    erdos_renyi_avg_degree,
    random_regular,
    barabasi_albert,
    clique_blocks,
    disjoint_union,
)
from . import workloads  # noqa: F401
