"""GPU parity: k-NN search, graph construction, normalisation, observations."""
import numpy as np
import pytest

import synth
from _helpers import check_graph, check_knn_lists, csr_of, near_tie_rows
from oracle import graph, observe

pytestmark = pytest.mark.gpu


def test_knn_f32_cuda_cores(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    X = np.ascontiguousarray(cfg1_data["X"], np.float32)
    idx, sim = hd.knn(gpu_ctx, X, X, 30, exclude_self=True)
    differ = check_knn_lists(idx, sim, X, X, 30, True, 2e-6)
    assert differ <= 2


@pytest.mark.parametrize("n,nq,d,k", [(1337, 1337, 200, 30), (600, 257, 2048, 50), (3000, 129, 64, 10)])
def test_knn_bf16_tensor_cores(gpu_ctx, n, nq, d, k):
    import torch
    import paper_1807_08692_gb300 as hd
    X, _ = synth.database(41, n, d, 13, 30.0, 300.0)
    Xb = synth.round_bf16(X)
    same = nq == n
    Q = Xb if same else synth.round_bf16(synth.queries(41, nq, d, 13, 30.0, 300.0))
    Xt = torch.from_numpy(Xb).to(torch.bfloat16).cuda()
    Qt = Xt if same else torch.from_numpy(Q).to(torch.bfloat16).cuda()
    idx, sim = hd.knn(gpu_ctx, Xt, Qt, k, exclude_self=same)
    differ = check_knn_lists(idx.cpu().numpy(), sim.cpu().numpy(), Xb, Q, k, same, 2e-5)
    assert differ <= max(2, nq // 100)


def test_build_graph_matches_oracle(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    c = cfg1_data["cfg"]
    X = np.ascontiguousarray(cfg1_data["X"], np.float32)
    g = hd.build_graph(gpu_ctx, X, c.k, c.gamma)
    rp, col, val, dinv = g.export()
    unc = near_tie_rows(X, c.k, 5e-6)
    assert len(unc) <= 20
    touched = check_graph(rp, col, val, dinv, cfg1_data["A"], unc)
    if len(unc) == 0:
        assert touched == 0


def test_build_graph_mutual_and_bf16(gpu_ctx):
    import torch
    import paper_1807_08692_gb300 as hd
    X, _ = synth.database(7, 900, 64, 6, 60.0, 60.0)
    Xb = synth.round_bf16(X)
    g = hd.build_graph(gpu_ctx, torch.from_numpy(Xb).to(torch.bfloat16).cuda(), 12, 3.0, hd.hd.SYM_MUTUAL)
    rp, col, val, dinv = g.export()
    A = graph.adjacency(Xb, 12, 3.0, "mutual")
    check_graph(rp, col, val, dinv, A, near_tie_rows(Xb, 12, 2e-5))


def test_graph_from_csr_normalises(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    rp, col, val = csr_of(cfg1_data["A"])
    # shuffle column order inside rows: the library sorts them
    rng = np.random.default_rng(0)
    col2, val2 = col.copy(), val.copy()
    for i in range(len(rp) - 1):
        s, e = rp[i], rp[i + 1]
        p = rng.permutation(e - s)
        col2[s:e], val2[s:e] = col[s:e][p], val[s:e][p]
    g = hd.graph_from_csr(gpu_ctx, rp, col2, val2)
    rpg, colg, valg, dinvg = g.export()
    W = cfg1_data["W"]
    assert np.array_equal(rpg, W.indptr) and np.array_equal(colg, W.indices)
    assert np.allclose(valg, W.data, rtol=2e-6, atol=1e-9)
    assert np.allclose(dinvg, cfg1_data["dinv"], rtol=1e-6)


def test_graph_from_csr_rejects_bad_input(gpu_ctx):
    import paper_1807_08692_gb300 as hd
    with pytest.raises(hd.HDError):
        hd.graph_from_csr(gpu_ctx, np.array([0, 2, 1], np.int32), np.array([1, 0], np.int32),
                          np.array([1.0, 1.0], np.float32))
    with pytest.raises(hd.HDError):
        hd.graph_from_csr(gpu_ctx, np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32),
                          np.array([1.0, 1.0], np.float32))


def test_observe_matches_oracle(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    c = cfg1_data["cfg"]
    X = np.ascontiguousarray(cfg1_data["X"], np.float32)
    Q = np.ascontiguousarray(cfg1_data["Q"], np.float32)
    yp, yi, yv = hd.observe(gpu_ctx, X, Q, c.k_y, c.gamma)
    assert np.array_equal(yp, cfg1_data["yp"])
    assert np.array_equal(yi, cfg1_data["yi"])
    assert np.allclose(yv, cfg1_data["yv"], rtol=2e-5)
