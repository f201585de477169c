"""Checkpoints of the graph and eigenpairs (bit-identical reload) and the
bounded-wait self-test of the tensor-core pipelines (no GPU fault: the waits
give up and report)."""
import time

import numpy as np
import pytest

from _helpers import csr_of, y_arrays

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_checkpoint_roundtrip_gives_identical_results(gpu_ctx, cfg1_data, tmp_path, storage):
    import paper_1807_08692_gb300 as hd
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    eig = hd.eig_from_host(gpu_ctx, g, cfg1_data["lam"][:40], cfg1_data["U"][:, :40], storage)
    g.save(tmp_path / "g.bin")
    eig.save(tmp_path / "e.bin")
    g2 = hd.graph_load(gpu_ctx, tmp_path / "g.bin")
    e2 = hd.eig_load(gpu_ctx, tmp_path / "e.bin")
    assert (g2.n, g2.nnz) == (g.n, g.nnz) and (e2.r, e2.storage) == (eig.r, eig.storage)
    for a, b in zip(g.export(), g2.export()):
        assert np.array_equal(a, b)
    la, Ua = eig.export()
    lb, Ub = e2.export()
    assert np.array_equal(la, lb) and np.array_equal(Ua, Ub)
    args = y_arrays(cfg1_data["yp"], cfg1_data["yi"], cfg1_data["yv"])
    X1, *_ = hd.query_batch(gpu_ctx, g, eig, "pcg", *args, 0.99, 1e-6, 500)
    X2, *_ = hd.query_batch(gpu_ctx, g2, e2, "pcg", *args, 0.99, 1e-6, 500)
    assert np.array_equal(X1.cpu().numpy().view(np.uint32), X2.cpu().numpy().view(np.uint32))


def test_checkpoint_errors(gpu_ctx, cfg1_data, tmp_path):
    import paper_1807_08692_gb300 as hd
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    g.save(tmp_path / "g.bin")
    with pytest.raises(hd.HDError):
        hd.eig_load(gpu_ctx, tmp_path / "g.bin")            # not an eigenpair file
    with pytest.raises(hd.HDError):
        hd.graph_load(gpu_ctx, tmp_path / "missing.bin")
    raw = (tmp_path / "g.bin").read_bytes()
    (tmp_path / "short.bin").write_bytes(raw[: len(raw) // 2])
    with pytest.raises(hd.HDError):
        hd.graph_load(gpu_ctx, tmp_path / "short.bin")
    # a column index out of range is caught by the structure check
    bad = bytearray(raw)
    off = 32 + 4 * (g.n + 1)
    bad[off:off + 4] = np.int32(10 ** 6).tobytes()
    (tmp_path / "bad.bin").write_bytes(bytes(bad))
    with pytest.raises(hd.HDError):
        hd.graph_load(gpu_ctx, tmp_path / "bad.bin")
    es = hd.eig_from_host(gpu_ctx, g, cfg1_data["lam"][:8], cfg1_data["U"][:, :8], "bf16").sparsify(0.5)
    with pytest.raises(hd.HDError):
        es.save(tmp_path / "sparse.bin")


def test_bounded_waits_give_up(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    t0 = time.perf_counter()
    timeout, aborted = hd.selftest_wait(gpu_ctx, 20000)   # 20 ms limit
    dt = time.perf_counter() - t0
    assert timeout and aborted
    assert 0.015 <= dt < 2.0
    # the context is still usable afterwards
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    X, it, rr, st = hd.query_batch(gpu_ctx, g, None, "paper",
                                   *y_arrays(cfg1_data["yp"], cfg1_data["yi"], cfg1_data["yv"]), 0.99, 1e-6, 500)
    assert np.all(st == 0)
