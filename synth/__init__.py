"""Seeded synthetic inputs for the gather-and-refine scoring path.

This module is the one thing the oracle side and the CUDA side share: it makes
an index (centroids, per-centroid token types, the doc -> centroid-id CSR, PQ
codebooks, PQ codes, residual norms) and query batches from a seed. It holds
none of the query-time scoring arithmetic (no query x centroid products, no
max/sum late interaction, no lookup tables, no selection); the per-type
k-means and the PQ encoding below only *build* the index the scoring path
reads, the way the paper's offline stage does (Sec. 2.1, "Token-Aware
Clustering" and "Residuals Compression").

Shapes follow the paper's workloads (Sec. 3: 128-d unit-norm token vectors,
Zipfian token types, passage-ranking and long-tail-QA document lengths).
"""
from .gen import (  # noqa: F401
    CONFIGS,
    SynthConfig,
    make_index,
    make_queries,
    load_or_make,
    index_bytes,
    random_index,
    random_queries,
)
