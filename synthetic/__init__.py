"""Seeded synthetic directed graphs shared by the CUDA path, the oracle, the tests
and the benchmark.

This package only produces inputs: sorted int32 CSR arrays of directed graphs with
the shapes of the paper's biological and communication networks (Table 2: a few
hundred to a few thousand vertices, sparse, heavy-tailed degrees, some reciprocal
arcs).  It holds none of the motif method's arithmetic.
"""
from .graphs import (  # noqa: F401
    Graph,
    WORKLOADS,
    chung_lu_digraph,
    complete_digraph,
    csr_from_arcs,
    directed_cycle,
    bidirected_path,
    out_star,
    empty_graph,
    disjoint_union,
    relabel,
    reverse,
    uniform_digraph,
    random_small_digraph,
    serving_stream,
    workload_graph,
)
