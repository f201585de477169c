"""The convergence analyser of Sec. 4.4 (Eq. 21-23): hd_cg_bound is host
arithmetic in the library, checked here without a GPU against the oracle's
counting loop; hd_spectrum_min (device Lanczos on -W) and the bound against
measured iteration counts are the GPU tests at the end."""
import numpy as np
import pytest

from oracle import spectral as S


@pytest.mark.parametrize("mode", ["paper", "proj", "pcg"])
def test_cg_bound_matches_oracle(mode):
    import paper_1807_08692_gb300 as hd
    rng = np.random.default_rng(3)
    cases = [(0.99, 1.0, -0.5), (0.99, 0.7, -0.5), (0.85, 0.2, -0.9), (0.99, -0.1, -0.3), (0.5, 0.0, 0.0),
             (0.999, 0.95, -1.0)]
    cases += [(rng.uniform(0.5, 0.999), *np.sort(rng.uniform(-1, 1, 2))[::-1]) for _ in range(30)]
    for alpha, lam_next, lam_min in cases:
        for tol in (1e-1, 1e-3, 1e-6, 1e-9):
            kap, ia, ir = hd.cg_bound(mode, alpha, lam_next, lam_min, tol)
            ref = S.kappa_deflated(alpha, lam_next, lam_min)
            assert kap == pytest.approx(ref, rel=1e-13)
            kap_res = S.kappa_deflated(alpha, 1.0, lam_min) if mode == "pcg" else ref
            assert ia == S.cg_iterations_bound(ref, tol)
            assert ir == S.cg_iterations_bound(ref, tol, kap_res)


def test_cg_bound_worked_example():
    # Sec. 4.4: alpha = 0.99, lambda_{r+1} = 0.7 cuts kappa to 0.0326 of r = 0's
    import paper_1807_08692_gb300 as hd
    k0, i0, _ = hd.cg_bound("paper", 0.99, 1.0, -0.5, 1e-6)
    k1, i1, _ = hd.cg_bound("paper", 0.99, 0.7, -0.5, 1e-6)
    assert round(k1 / k0, 4) == 0.0326
    assert i1 < i0


def test_cg_bound_rejects_bad_arguments():
    import paper_1807_08692_gb300 as hd
    for args in [(1.0, 0.5, -0.5, 1e-6), (0.9, 0.5, -0.5, 0.0), (0.9, -0.6, -0.5, 1e-6), (0.9, 1.2, -0.5, 1e-6),
                 (0.9, 0.5, -1.5, 1e-6)]:
        with pytest.raises(hd.HDError):
            hd.cg_bound("paper", *args)


def test_convergence_table_decreases_with_r():
    import paper_1807_08692_gb300 as hd
    lam = np.concatenate([[1.0], np.linspace(0.95, 0.1, 399)])
    rows = hd.convergence_table(lam, -0.6, 0.99, 1e-6, [0, 50, 100, 200, 300])
    its = [r["iters_resid"] for r in rows]
    assert its == sorted(its, reverse=True) and its[0] > its[-1]
    assert rows[0]["kappa"] == pytest.approx((1 + 0.99 * 0.6) / 0.01)


@pytest.mark.gpu
def test_spectrum_min_matches_eigh(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    from _helpers import csr_of
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    lam_min, conv = hd.spectrum_min(gpu_ctx, g, tol=1e-6)
    assert conv
    assert lam_min == pytest.approx(cfg1_data["lam"][-1], abs=1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("mode,r", [("paper", 0), ("paper", 50), ("proj", 50), ("pcg", 50), ("pcg", 20)])
def test_measured_iterations_within_bound(gpu_ctx, cfg1_data, mode, r):
    # fp32 CG on the GPU with exact (f32-stored) eigenpairs: the iteration count
    # never exceeds the Eq. 21 bound for its stopping rule.
    import paper_1807_08692_gb300 as hd
    from _helpers import csr_of, y_arrays
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    lam_all = cfg1_data["lam"]
    eig = hd.eig_from_host(gpu_ctx, g, lam_all[:r], cfg1_data["U"][:, :r], "f32") if r else None
    lam_min, _ = hd.spectrum_min(gpu_ctx, g, tol=1e-6)
    lam_next = lam_all[r] if r else 1.0
    for tol in (1e-2, 1e-4):
        _, _, bound = hd.cg_bound(mode, 0.99, lam_next, lam_min, tol)
        _, it, _, st = hd.query_batch(gpu_ctx, g, eig, mode, *y_arrays(cfg1_data["yp"], cfg1_data["yi"],
                                                                          cfg1_data["yv"]), 0.99, tol, 1000)
        assert np.all(st == 0)
        assert np.max(it) <= bound, (np.max(it), bound)
