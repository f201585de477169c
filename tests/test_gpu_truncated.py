"""Temporal† (truncated temporal filtering, Sec. 3.1) on the device against the
oracle's subgraph solve."""
import numpy as np
import pytest

from _helpers import csr_of, rel_l2_cols, y_arrays
from oracle import rank as ORank
from oracle import truncated as T

pytestmark = pytest.mark.gpu


def _case(cfg1_data, sizes):
    X, Q = cfg1_data["X"], cfg1_data["Q"]
    sls = [T.shortlist(X, Q[j], s) for j, s in enumerate(sizes)]
    sl_ptr = np.concatenate([[0], np.cumsum([len(s) for s in sls])]).astype(np.int32)
    return sls, sl_ptr, np.concatenate(sls).astype(np.int32)


def test_truncated_matches_oracle(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    B = cfg1_data["Y"].shape[1]
    sizes = [300, 150, 2000, 17, 64, 1000, 500, 300, 10, 700, 300, 301, 299, 1500, 250, 128][:B]
    sls, sl_ptr, sl_idx = _case(cfg1_data, sizes)
    args = y_arrays(cfg1_data["yp"], cfg1_data["yi"], cfg1_data["yv"])
    tol = 1e-6
    Xg, it, rr, st = hd.temporal_truncated(gpu_ctx, g, sl_ptr, sl_idx, *args, 0.99, tol, 1000)
    Xg = Xg.cpu().numpy().astype(np.float64)
    for j in range(B):
        s = sizes[j]
        ref, _ = T.temporal_truncated(cfg1_data["A"], sls[j], cfg1_data["Y"][:, j], 0.99, 1e-12, 5000)
        assert rel_l2_cols(Xg[:s, j:j + 1], ref[:, None]).max() <= 1e-4, j
        # A column stops when its true residual meets tol.  On a small subgraph
        # x is about as large as y, and the exact solution rounded to fp32
        # already leaves a residual near c1 u ||x|| (~1e-6 of ||y||): there the
        # solver reports STAGNATED, and only where fp32 cannot do much better.
        W_S, _ = T.subsystem(cfg1_data["A"], sls[j])
        y_S = cfg1_data["Y"][sls[j], j]
        xr = ref.astype(np.float32).astype(np.float64)
        floor = np.linalg.norm(y_S - (xr - 0.99 * (W_S @ xr)) / 0.01) / np.linalg.norm(y_S)
        if st[j] == hd.hd.COL_CONVERGED:
            assert rr[j] <= tol, (j, rr[j])
        else:
            assert st[j] == hd.hd.COL_STAGNATED and floor > 0.3 * tol, (j, st[j], rr[j], floor)
            assert rr[j] <= 10 * floor, (j, rr[j], floor)
        assert np.all(Xg[s:, j] == 0.0)
        if s == 2000:
            # the whole graph: plain temporal filtering, in shortlist order
            assert rel_l2_cols(Xg[:s, j:j + 1], cfg1_data["xstar"][sls[j], j:j + 1]).max() <= 1e-4
    # ranking within each shortlist, mapped back to database ids
    ids, sc = hd.rank_shortlists(gpu_ctx, hd_tensor(Xg), sl_ptr, sl_idx, 10)
    for j in range(B):
        ref, _ = T.temporal_truncated(cfg1_data["A"], sls[j], cfg1_data["Y"][:, j], 0.99, 1e-12, 5000)
        k = min(10, sizes[j])
        top, _ = ORank.topk(ref, k)
        # scores are the solver's fp32 values at the shortlist positions, exactly
        xg = Xg[:sizes[j], j].astype(np.float32)
        assert ORank.ranks_match(_local(ids[j][:k], sls[j]), top, ref, 1e-5 * ref.max(), scores=sc[j][:k],
                                 x=xg), j


def hd_tensor(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _local(ids, S):
    where = {int(i): t for t, i in enumerate(S)}
    return np.array([where[int(i)] for i in ids])


def test_truncated_rejects_bad_shortlists(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    yp = np.array([0, 1], np.int32)
    yi = np.array([5], np.int32)
    yv = np.array([1.0], np.float32)
    with pytest.raises(hd.HDError):
        hd.temporal_truncated(gpu_ctx, g, np.array([0, 3], np.int32), np.array([5, 7, 5], np.int32), yp, yi, yv,
                              0.99, 1e-6, 100)
    with pytest.raises(hd.HDError):
        hd.temporal_truncated(gpu_ctx, g, np.array([0, 2], np.int32), np.array([5, 2000], np.int32), yp, yi, yv,
                              0.99, 1e-6, 100)
    # an observation outside the shortlist is dropped: y_S = 0 gives x_S = 0
    X, it, _, st = hd.temporal_truncated(gpu_ctx, g, np.array([0, 2], np.int32), np.array([8, 9], np.int32), yp, yi,
                                         yv, 0.99, 1e-6, 100)
    assert np.all(X.cpu().numpy() == 0.0)
