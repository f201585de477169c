"""hd_rank_static: the allocation-free top-K (for callers that cannot call
cudaMalloc at request time) returns exactly what hd_rank returns, on two calls
in a row that share its static scratch.  Named to be collected last."""
import ctypes as C
import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_rank_into(ctx, X, K, Kmax, idx, sc):
    import torch
    from paper_1807_08692_gb300.hd import lib
    n, B = X.shape
    Kh = np.ascontiguousarray(K, np.int32)
    rc = lib().hd_rank_static(ctx.handle, C.c_void_p(X.data_ptr()), n, B, X.stride(0), Kh.ctypes.data_as(C.c_void_p),
                              Kmax, C.c_void_p(idx.data_ptr()), C.c_void_p(sc.data_ptr()))
    ctx.check(rc, "hd_rank_static")
    torch.cuda.synchronize()


def _static_rank(ctx, X, K, Kmax):
    import torch
    n, B = X.shape
    idx = torch.empty((B, Kmax), dtype=torch.int32, device=X.device)
    sc = torch.empty((B, Kmax), dtype=torch.float32, device=X.device)
    _static_rank_into(ctx, X, K, Kmax, idx, sc)
    return idx.cpu().numpy(), sc.cpu().numpy()


def test_static_rank_equals_rank_twice():
    import torch
    import paper_1807_08692_gb300 as hd
    ctx = hd.Context(0)
    rng = np.random.default_rng(11)
    cases = [
        # many exact ties (scores on a coarse grid), ragged sizes, K up to Kmax, a K of 0
        ((rng.integers(0, 50, (7001, 9)) / 16.0).astype(np.float32), [1, 10, 100, 1000, 2048, 0, 37, 512, 5], 2048),
        # continuous scores, a different batch width: leftovers of the previous call must not matter
        (rng.standard_normal((30011, 3)).astype(np.float32), [100, 7, 100], 100),
    ]
    # one call first, so that every kernel it uses is loaded before memory is read
    warm = torch.from_numpy(cases[0][0]).cuda()
    _static_rank(ctx, warm, cases[0][1], cases[0][2])
    for x, K, Kmax in cases:
        Xd = torch.from_numpy(x).cuda()
        ref_idx, ref_sc = hd.rank(ctx, Xd, np.asarray(K, np.int32), Kmax=Kmax)
        torch.cuda.synchronize()
        outs = [(torch.empty((len(K), Kmax), dtype=torch.int32, device="cuda"),
                 torch.empty((len(K), Kmax), dtype=torch.float32, device="cuda")) for _ in range(2)]
        # the device's free memory, torch's reserved pool and the library's
        # workspace stay exactly as they were across the two calls: nothing is
        # allocated (unreferenced tensors are collected first, so that torch's
        # own bookkeeping does not move in between)
        gc.collect()
        torch.cuda.synchronize()
        before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(), ctx.workspace_bytes())
        for idx_t, sc_t in outs:
            _static_rank_into(ctx, Xd, K, Kmax, idx_t, sc_t)
        after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(), ctx.workspace_bytes())
        assert before == after, (before, after)
        for idx_t, sc_t in outs:
            idx, sc = idx_t.cpu().numpy(), sc_t.cpu().numpy()
            assert np.array_equal(idx, ref_idx)
            assert np.array_equal(sc.view(np.uint32), ref_sc.view(np.uint32))
    with pytest.raises(hd.HDError):
        _static_rank(ctx, torch.zeros((10, 257), device="cuda"), [1] * 257, 4)
    ctx.close()
