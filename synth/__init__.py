"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This package draws random numbers and nothing else: von Mises-Fisher mixture
descriptors (Wood's rejection sampler), query descriptors, cluster-size laws,
Poisson arrival streams and per-request tolerance / K draws.  It holds none of
the diffusion method's arithmetic (no similarities, no k-NN, no graph, no
solve), so the oracle and the CUDA path may both import it without sharing any
method code.

The workloads stand in for the image-retrieval benchmarks of Sec. 5.1
(ROxford/RParis + R1M with d=2048 GeM descriptors), which are not available
here; see `synth.configs` for the recipes.
"""
from .vmf import (  # noqa: F401
    wood_radial,
    sample_vmf_rows,
    mixture_means,
    mixture_labels,
    database,
    queries,
    regional_database,
    round_bf16,
    bf16_bits,
    poisson_arrivals,
    request_draws,
    a_d_kappa,
)
from .configs import CONFIGS, Config, get_config  # noqa: F401
