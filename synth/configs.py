"""Workload recipes: synthetic stand-ins for the paper's retrieval workloads.

The paper evaluates on ROxford/RParis + R1M with d=2048 GeM descriptors,
k=50 reciprocal neighbours, weights (v^T z)_+^3, alpha=0.99 and y holding the
top-5 neighbours of the query (Sec. 5.1).  Those datasets and descriptor
weights are not available, so each recipe below draws descriptors from a
seeded von Mises-Fisher mixture with the stated sizes.  Seeds are
1807_08692 + config number.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Config:
    name: str
    seed: int
    n: int                 # database items (graph nodes)
    d: int                 # descriptor dimension
    dtype: str             # "f32" or "bf16" storage of the descriptors
    ncl: int               # mixture components
    kappa_lo: float
    kappa_hi: float
    sizes: str = "equal"   # "equal" or "zipf"
    zipf_s: float = 1.1
    k: int = 50            # neighbours per node before symmetrisation
    gamma: float = 3.0     # edge weight max(s, 0)^gamma
    alpha: float = 0.99
    ranks: tuple = (0,)
    batch: int = 16        # queries per batch
    k_y: int = 10          # non-zeros of each observation vector
    tol: float = 1e-6
    topk: int = 100
    regions: int = 1       # rows per image (regional workload)
    extra: dict = field(default_factory=dict)


BASE_SEED = 1807_08692

CONFIGS = {
    # 2,000 fp32 descriptors, d=128, 20 equal vMF components, kappa=50; k=30
    # graph; r in {0, 50}; 16 queries with top-10 observations; tol 1e-6.
    "cfg1": Config("cfg1_n2k_d128", BASE_SEED + 1, 2000, 128, "f32", 20, 50.0, 50.0,
                   k=30, ranks=(0, 50), batch=16, k_y=10, tol=1e-6),
    # 100,000 fp32 descriptors, d=512, 1,000 Zipf(1.1)-sized components,
    # kappa=50 (unstated in the recipe, assumed); k=50; r in {0,100,400}; B=64,
    # top-50 observations.
    "cfg2": Config("cfg2_n100k_d512", BASE_SEED + 2, 100_000, 512, "f32", 1000, 50.0, 50.0,
                   sizes="zipf", k=50, ranks=(0, 100, 400), batch=64, k_y=50, tol=1e-6),
    # 1,000,000 bf16 descriptors, d=2048, 10,000 equal components with kappa
    # uniform in [20, 200]; k=50; r in {0,50,100,200,400}; B in {1,16,64,256};
    # top-10 observations; top-100 ranking.
    "cfg3": Config("cfg3_n1m_d2048", BASE_SEED + 3, 1_000_000, 2048, "bf16", 10_000, 20.0, 200.0,
                   k=50, ranks=(0, 50, 100, 200, 400), batch=64, k_y=10, tol=1e-6,
                   extra={"batches": (1, 16, 64, 256)}),
    # Serving on the cfg3 graph with r=200 and bf16 U; Poisson arrivals.
    "cfg4": Config("cfg4_serve_n1m", BASE_SEED + 3, 1_000_000, 2048, "bf16", 10_000, 20.0, 200.0,
                   k=50, ranks=(200,), batch=64, k_y=10, tol=1e-6,
                   extra={"rates": (100, 300, 1000, 3000, 10000, 20000),
                          "tols": (1e-2, 1e-4, 1e-6), "ks": (10, 100, 1000)}),
    # Regional: 240,000 images x 21 regions (n=5.04M), d=512 bf16; regions
    # share the image's component with p=0.8; r=100 with fp8 U; 128 queries
    # of 21 regions each; per-image score = sum over its regions.
    "cfg5": Config("cfg5_regional_n5m", BASE_SEED + 5, 240_000 * 21, 512, "bf16", 10_000, 20.0, 200.0,
                   k=50, ranks=(100,), batch=128, k_y=10, tol=1e-6, regions=21,
                   extra={"images": 240_000, "p_stay": 0.8}),
}


def get_config(key: str) -> Config:
    return CONFIGS[key]
