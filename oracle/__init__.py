"""Plain FP64 CPU oracle for hybrid spectral-temporal diffusion (arXiv 1807.08692).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import or run this
package.  The product path (the CUDA library and its Python binding) never
calls it and shares no code with it; both sides read the same seeded inputs
from `synth`, which holds no method arithmetic.

What it computes (NumPy / SciPy, float64, one column at a time):

* `graph`     - k-NN graph by brute-force dot products, weights (v^T z)_+^gamma,
                symmetrisation and W = D^-1/2 A D^-1/2          (Sec. 3; Sec. 5.1)
* `observe`   - observation vectors y: top-k_y similarities of a query (Sec. 3; Sec. 5.1)
* `diffusion` - the ranking vector x by every route the paper names:
                closed form (1-alpha)(I - alpha W)^-1 y           (Eq. 3)
                temporal filtering by CG on L_alpha(W) x = y        (Eq. 1-2)
                spectral filtering U h(Lambda) U^T y                (Eq. 4)
                hybrid x = x^s + x^t with the black-box operator    (Eq. 17-20)
                plus the projected form (Form N) and the spectrally
                preconditioned CG form (Form S) read from Eq. 15-23
* `spectral`  - dense eigenpairs, condition numbers and the CG bound (Eq. 5, 21-23)
* `rank`      - top-K ranking by decreasing x, ties to the smaller id (Sec. 3)
* `shybrid`   - sparsified U_1 (SHybrid, Sec. 5.3)
* `general`   - Theorem 2 decomposition for a general series h (Appendix A)

Every function is pinned by `tests/test_oracle_*.py` against closed forms,
brute force, the paper's worked numbers and invariants.
"""
from . import graph, observe, diffusion, spectral, rank, shybrid, general  # noqa: F401
