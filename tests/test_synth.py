"""Checks of the seeded input generators (they hold no method arithmetic)."""
import numpy as np
import pytest

import synth
from synth import vmf


@pytest.mark.parametrize("d,kappa", [(128, 50.0), (2048, 200.0), (512, 50.0)])
def test_vmf_mean_resultant_length(d, kappa):
    # E[mu^T x] = A_d(kappa) = I_{d/2}(kappa) / I_{d/2-1}(kappa) for vMF on S^{d-1}.
    rng = np.random.default_rng(0)
    w = vmf.wood_radial(np.full(20000, kappa), d, rng)
    assert abs(w.mean() - synth.a_d_kappa(d, kappa)) < 4 * w.std() / np.sqrt(w.size) + 1e-4


def test_samples_unit_norm_and_centered():
    X, lab = synth.database(1, 3000, 64, 3, 400.0, 400.0)
    assert np.allclose(np.linalg.norm(X, axis=1), 1, atol=1e-5)
    mu = vmf.mixture_means(1, 3, 64)
    cos = np.einsum("ij,ij->i", X, mu[lab])
    assert abs(cos.mean() - synth.a_d_kappa(64, 400.0)) < 0.01


def test_thread_count_does_not_change_output(monkeypatch):
    monkeypatch.setattr(vmf, "BLOCK_ROWS", 128)
    monkeypatch.setattr(vmf, "_threads", lambda: 1)
    a, _ = synth.database(9, 1000, 16, 5, 10.0, 90.0)
    monkeypatch.setattr(vmf, "_threads", lambda: 6)
    b, _ = synth.database(9, 1000, 16, 5, 10.0, 90.0)
    assert np.array_equal(a, b)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).standard_normal(10000).astype(np.float32)
    x[:4] = [1.00390625, 1.01171875, -1.00390625, 3.0e-39]  # ties and a subnormal
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(synth.round_bf16(x), want)
    assert np.array_equal(synth.bf16_bits(synth.round_bf16(x)),
                          torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16))


def test_zipf_sizes_and_regions():
    lab = vmf.mixture_labels(3, 200000, 100, "zipf", 1.1)
    counts = np.bincount(lab, minlength=100)
    p = np.arange(1, 101) ** -1.1
    p /= p.sum()
    assert np.allclose(counts / counts.sum(), p, atol=0.005)
    X, img = synth.regional_database(4, 50, 21, 16, 8, 50.0, 50.0)
    assert X.shape == (1050, 16) and img[20] == 0 and img[21] == 1


def test_arrivals_and_draws():
    t = synth.poisson_arrivals(1, 1000.0, 20000)
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() - 1e-3) < 5e-5
    tol, K = synth.request_draws(1, 3000)
    assert set(tol) == {1e-2, 1e-4, 1e-6} and set(K) == {10, 100, 1000}
