"""General transfer functions (Appendix A, Theorem 2) on the device against the
oracle's Horner evaluation of the same series."""
import numpy as np
import pytest

from _helpers import csr_of, rel_l2_cols, y_arrays
from oracle import diffusion as D
from oracle import general

pytestmark = pytest.mark.gpu

COEFFS = [0.3, 0.5, -0.2, 0.0, 0.15, 0.1, -0.05]


def _setup(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    args = y_arrays(cfg1_data["yp"], cfg1_data["yi"], cfg1_data["yv"])
    return g, args


def test_poly_without_eigenpairs(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    g, args = _setup(gpu_ctx, cfg1_data)
    X = hd.filter_poly(gpu_ctx, g, None, *args, COEFFS).cpu().numpy().astype(np.float64)
    ref = general.poly_apply(lambda z: cfg1_data["W"] @ z, COEFFS, cfg1_data["Y"])
    assert rel_l2_cols(X, ref).max() <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_poly_theorem2(gpu_ctx, cfg1_data, storage):
    import paper_1807_08692_gb300 as hd
    g, args = _setup(gpu_ctx, cfg1_data)
    r = 50
    eig = hd.eig_from_host(gpu_ctx, g, cfg1_data["lam"][:r], cfg1_data["U"][:, :r], storage)
    lam, Uq = eig.export()
    X = hd.filter_poly(gpu_ctx, g, eig, *args, COEFFS).cpu().numpy().astype(np.float64)
    W, Y = cfg1_data["W"], cfg1_data["Y"]
    ref = np.stack([general.hybrid_poly(W, Uq.astype(np.float64), lam, COEFFS, Y[:, j]) for j in range(Y.shape[1])], 1)
    assert rel_l2_cols(X, ref).max() <= 1e-5
    if storage == "f32":
        # with (nearly) exact eigenpairs Theorem 2 gives h(W) y itself
        direct = general.poly_apply(lambda z: W @ z, COEFFS, Y)
        assert rel_l2_cols(X, direct).max() <= 1e-5


@pytest.mark.parametrize("r", [0, 50])
def test_truncated_h_alpha_series(gpu_ctx, cfg1_data, r):
    # c_i = (1 - alpha) alpha^i: the first terms of Eq. 3's series (Appendix A)
    import paper_1807_08692_gb300 as hd
    g, args = _setup(gpu_ctx, cfg1_data)
    a, terms = 0.9, 80
    co = [(1 - a) * a ** i for i in range(terms)]
    eig = hd.eig_from_host(gpu_ctx, g, cfg1_data["lam"][:r], cfg1_data["U"][:, :r], "f32") if r else None
    X = hd.filter_poly(gpu_ctx, g, eig, *args, co).cpu().numpy().astype(np.float64)
    assert rel_l2_cols(X, D.neumann(cfg1_data["W"], cfg1_data["Y"], a, terms)).max() <= 1e-5


def test_poly_edge_cases(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    g, args = _setup(gpu_ctx, cfg1_data)
    X = hd.filter_poly(gpu_ctx, g, None, *args, [2.5]).cpu().numpy()
    assert np.array_equal(X, np.float32(2.5) * cfg1_data["Y"].astype(np.float32))
    # host output buffer, sparse eigenpairs
    eig = hd.eig_from_host(gpu_ctx, g, cfg1_data["lam"][:20], cfg1_data["U"][:, :20], "bf16").sparsify(0.9)
    n, B = cfg1_data["Y"].shape
    Xh = np.zeros((n, B), np.float32)
    hd.filter_poly(gpu_ctx, g, eig, *args, COEFFS, X=Xh)
    Xd = hd.filter_poly(gpu_ctx, g, eig, *args, COEFFS).cpu().numpy()
    assert np.array_equal(Xh, Xd)
    with pytest.raises(hd.HDError):
        hd.filter_poly(gpu_ctx, g, None, *args, [])
    with pytest.raises(hd.HDError):
        hd.filter_poly(gpu_ctx, g, None, *args, [1.0, float("nan")])
