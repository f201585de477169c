"""GB300 (sm_103a) hybrid spectral-temporal diffusion: the online query path of
Iscen et al., "Hybrid Diffusion: Spectral-Temporal Graph Filtering for
Manifold Ranking" (Eq. 17-20), behind the C ABI of include/hd.h.

`hd` is the thin ctypes binding; `build` compiles libhd.so in-tree.
"""
from . import hd  # noqa: F401
from .hd import (  # noqa: F401
    Context, Graph, Eig, HDError, build_graph, graph_from_csr, knn, observe, observe_regional, eig_from_host,
    eigendecompose, query_batch, rank, Server, spectrum_min, cg_bound, convergence_table,
    filter_poly, temporal_truncated, rank_shortlists, graph_load, eig_load, selftest_wait,
    COL_CONVERGED, COL_MAX_ITER, COL_BREAKDOWN, COL_EMPTY, COL_CANCELLED, COL_STAGNATED,
)
