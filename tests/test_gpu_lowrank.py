"""Spectral products U^T V and U H on the device (tensor cores for every
storage: bf16 directly, fp8 through converter warps, fp32 through its bf16
[hi | lo] split) against numpy on the dequantised U."""
import numpy as np
import pytest

from _helpers import csr_of

pytestmark = pytest.mark.gpu


def _graph(ctx, n):
    import paper_1807_08692_gb300 as hd
    rp = np.arange(n + 1, dtype=np.int32)
    col = ((np.arange(n) + 1) % n).astype(np.int32)
    val = np.ones(n, np.float32)
    return hd.graph_from_csr(ctx, rp, col, val, normalized=True)


@pytest.mark.parametrize("storage", ["bf16", "f32", "fp8"])
@pytest.mark.parametrize("n,r,B", [(1000, 50, 16), (4099, 200, 64), (777, 130, 4), (2500, 400, 64), (1300, 64, 256)])
def test_project_and_expand(gpu_ctx, storage, n, r, B):
    import ctypes as C
    import torch
    import paper_1807_08692_gb300 as hd
    from paper_1807_08692_gb300.hd import lib
    rng = np.random.default_rng(n + r + B)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    lam = np.sort(rng.uniform(-0.5, 1.0, r))[::-1].copy()
    g = _graph(gpu_ctx, n)
    eig = hd.eig_from_host(gpu_ctx, g, lam, U.astype(np.float32), storage)
    _, Uq = eig.export()          # the stored basis, dequantised
    Uq = Uq.astype(np.float64)
    V = rng.standard_normal((n, B)).astype(np.float32)
    Vd = torch.from_numpy(V).cuda()
    Cg = np.zeros((r, B), np.float64)
    gpu_ctx.check(lib().hd_eig_project(gpu_ctx.handle, eig.handle, C.c_void_p(Vd.data_ptr()), B,
                                       Cg.ctypes.data_as(C.c_void_p)), "project")
    Cref = Uq.T @ V.astype(np.float64)
    assert np.linalg.norm(Cg - Cref) / np.linalg.norm(Cref) <= 2e-5
    H = rng.standard_normal((r, B))
    Xd = torch.empty((n, B), dtype=torch.float32, device="cuda")
    gpu_ctx.check(lib().hd_eig_expand(gpu_ctx.handle, eig.handle, H.ctypes.data_as(C.c_void_p), B,
                                      C.c_void_p(Xd.data_ptr())), "expand")
    Xref = Uq @ H
    Xg = Xd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Xg - Xref) / np.linalg.norm(Xref) <= 2e-5


def test_eig_roundtrip_storage(gpu_ctx):
    import paper_1807_08692_gb300 as hd
    import synth
    rng = np.random.default_rng(1)
    n, r = 300, 20
    U = rng.standard_normal((n, r)).astype(np.float32)
    g = _graph(gpu_ctx, n)
    lam = np.linspace(1, 0.5, r)
    lam_b, Ub = hd.eig_from_host(gpu_ctx, g, lam, U, "bf16").export()
    assert np.array_equal(Ub, synth.round_bf16(U))
    assert np.array_equal(lam_b, lam)
    _, Uf = hd.eig_from_host(gpu_ctx, g, lam, U, "f32").export()
    assert np.array_equal(Uf, U)
    _, U8 = hd.eig_from_host(gpu_ctx, g, lam, U, "fp8").export()
    # e4m3 keeps 3 mantissa bits: relative error <= 2^-4 of the row scale
    scale = np.abs(U).max(axis=1, keepdims=True)
    assert np.all(np.abs(U8 - U) <= scale * 2.0 ** -4 + 1e-12)
