"""SHybrid (Sec. 5.3): the sparsified embedding on the device against the
oracle's selection rule, its products, and the hybrid solves that use it."""
import ctypes as C

import numpy as np
import pytest

from _helpers import csr_of, rel_l2_cols, y_arrays
from oracle import diffusion as D
from oracle import shybrid

pytestmark = pytest.mark.gpu


def _cycle(ctx, n):
    import paper_1807_08692_gb300 as hd
    rp = np.arange(n + 1, dtype=np.int32)
    col = ((np.arange(n) + 1) % n).astype(np.int32)
    return hd.graph_from_csr(ctx, rp, col, np.ones(n, np.float32), normalized=True)


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("sparsity", [0.0, 0.5, 0.9, 0.99, 1.0])
def test_sparsify_selects_like_the_oracle(gpu_ctx, storage, sparsity):
    import paper_1807_08692_gb300 as hd
    rng = np.random.default_rng(5)
    n, r = 3001, 37
    U = rng.standard_normal((n, r)).astype(np.float32)
    g = _cycle(gpu_ctx, n)
    eig = hd.eig_from_host(gpu_ctx, g, np.linspace(1, 0.2, r), U, storage)
    lam, Uq = eig.export()
    es = eig.sparsify(sparsity)
    lam_s, Us = es.export()
    ref = shybrid.sparsify(Uq.astype(np.float64), sparsity)
    assert np.array_equal(Us.astype(np.float64), ref)
    assert es.nnz == n * r - int(round(sparsity * n * r))
    assert np.array_equal(lam_s, lam)


def test_sparsify_tie_rule(gpu_ctx):
    # magnitudes on a grid of 1/8: many exact ties at the threshold; the later
    # row-major entry is dropped first (zeros included)
    import paper_1807_08692_gb300 as hd
    rng = np.random.default_rng(6)
    n, r = 1000, 24
    U = (rng.integers(-6, 7, (n, r)) / 8.0).astype(np.float32)
    g = _cycle(gpu_ctx, n)
    eig = hd.eig_from_host(gpu_ctx, g, np.linspace(1, 0.2, r), U, "f32")
    for s in (0.1, 0.37, 0.5, 0.77, 0.999):
        es = eig.sparsify(s)
        _, Us = es.export()
        ref = shybrid.sparsify(U.astype(np.float64), s)
        assert np.array_equal(Us.astype(np.float64), ref)
        assert es.nnz == n * r - int(round(s * n * r))


@pytest.mark.parametrize("n,r,B", [(4099, 200, 64), (777, 130, 4), (2500, 64, 256)])
def test_sparse_products(gpu_ctx, n, r, B):
    import torch
    import paper_1807_08692_gb300 as hd
    from paper_1807_08692_gb300.hd import lib
    rng = np.random.default_rng(n + r)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    g = _cycle(gpu_ctx, n)
    es = hd.eig_from_host(gpu_ctx, g, np.linspace(1, 0.1, r), U.astype(np.float32), "bf16").sparsify(0.95)
    _, Us = es.export()
    Us = Us.astype(np.float64)
    V = rng.standard_normal((n, B)).astype(np.float32)
    Vd = torch.from_numpy(V).cuda()
    Cg = np.zeros((r, B), np.float64)
    gpu_ctx.check(lib().hd_eig_project(gpu_ctx.handle, es.handle, C.c_void_p(Vd.data_ptr()), B,
                                       Cg.ctypes.data_as(C.c_void_p)), "project")
    Cref = Us.T @ V.astype(np.float64)
    assert np.linalg.norm(Cg - Cref) / np.linalg.norm(Cref) <= 1e-6
    H = rng.standard_normal((r, B))
    Xd = torch.empty((n, B), dtype=torch.float32, device="cuda")
    gpu_ctx.check(lib().hd_eig_expand(gpu_ctx.handle, es.handle, H.ctypes.data_as(C.c_void_p), B,
                                      C.c_void_p(Xd.data_ptr())), "expand")
    Xref = Us @ H
    assert np.linalg.norm(Xd.cpu().numpy() - Xref) / np.linalg.norm(Xref) <= 1e-6


@pytest.mark.parametrize("sparsity", [0.5, 0.99])
def test_shybrid_solves(gpu_ctx, cfg1_data, sparsity):
    # Form S stays exact with the sparsified U; Form P with it is the paper's
    # SHybrid approximation, compared with the oracle's Form P on the same U.
    import paper_1807_08692_gb300 as hd
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    r = 50
    lam, U = cfg1_data["lam"][:r], cfg1_data["U"][:, :r]
    es = hd.eig_from_host(gpu_ctx, g, lam, U, "f32").sparsify(sparsity)
    _, Us = es.export()
    args = y_arrays(cfg1_data["yp"], cfg1_data["yi"], cfg1_data["yv"])
    Xs, its, _, sts = hd.query_batch(gpu_ctx, g, es, "pcg", *args, 0.99, 1e-6, 500)
    assert np.all(sts == 0)
    assert rel_l2_cols(Xs.cpu().numpy().astype(np.float64), cfg1_data["xstar"]).max() <= 1e-4
    Xp, _, _, stp = hd.query_batch(gpu_ctx, g, es, "paper", *args, 0.99, 1e-6, 500)
    xref, _, _, _ = D.hybrid(cfg1_data["W"], Us.astype(np.float64), lam, cfg1_data["Y"], 0.99, 1e-10, 2000)
    assert rel_l2_cols(Xp.cpu().numpy().astype(np.float64), xref).max() <= 1e-4
    # repeatable bit for bit
    Xs2, *_ = hd.query_batch(gpu_ctx, g, es, "pcg", *args, 0.99, 1e-6, 500)
    assert np.array_equal(Xs.cpu().numpy(), Xs2.cpu().numpy())
