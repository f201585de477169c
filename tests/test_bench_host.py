"""Host logic of the benchmark that needs no GPU: the NumPy readers of the
library's checkpoint files (the reference arm's inputs), the clock summary of
the nvidia-smi samples, the algorithmic byte counts behind the roofline, and
the rule that withholds the ncu traffic figure once the SpMM source changed."""
import numpy as np
import pytest

import bench


def _write_graph(path, rp, col, val, dinv):
    n, nnz = len(rp) - 1, len(col)
    with open(path, "wb") as f:
        f.write(b"HDGRAPH1")
        f.write(np.array([n, nnz, 0], np.int64).tobytes())
        f.write(np.asarray(rp, np.int32).tobytes())
        f.write(np.asarray(col, np.int32).tobytes())
        f.write(np.asarray(val, np.float32).tobytes())
        f.write(np.asarray(dinv, np.float32).tobytes())


def test_graph_checkpoint_reader(tmp_path):
    # rows of different lengths, one empty row, values that fp32 holds exactly
    rp = [0, 2, 2, 5, 6]
    col = [1, 3, 0, 1, 3, 2]
    val = [0.5, 0.25, 0.5, 0.125, 0.75, 0.75]
    p = tmp_path / "g.hdg"
    _write_graph(p, rp, col, val, [1.0, 0.5, 0.25, 2.0])
    W = bench.read_graph_checkpoint(p)
    dense = np.zeros((4, 4))
    for i in range(4):
        for t in range(rp[i], rp[i + 1]):
            dense[i, col[t]] = val[t]
    assert W.shape == (4, 4) and W.dtype == np.float64
    assert np.array_equal(W.toarray(), dense)
    bad = tmp_path / "bad.hdg"
    bad.write_bytes(b"HDGRAPH0" + bytes(24))
    with pytest.raises(ValueError):
        bench.read_graph_checkpoint(bad)


def _write_eig(path, lam, U, ldu, storage=0):
    n, r = U.shape
    Up = np.zeros((n, ldu), np.float32)
    Up[:, :r] = U
    with open(path, "wb") as f:
        f.write(b"HDEIG001")
        f.write(np.array([n], np.int64).tobytes())
        f.write(np.array([r, storage, ldu, 0], np.int32).tobytes())
        f.write(np.asarray(lam, np.float64).tobytes())
        f.write(Up.tobytes())


def test_eig_checkpoint_reader(tmp_path):
    rng = np.random.default_rng(3)
    U = rng.standard_normal((5, 3)).astype(np.float32)
    lam = np.array([1.0, 0.5, -0.25])
    p = tmp_path / "e.hde"
    _write_eig(p, lam, U, ldu=16)
    lam2, U2 = bench.read_eig_checkpoint(p)
    assert np.array_equal(lam2, lam)
    assert U2.shape == (5, 3) and np.array_equal(U2, U.astype(np.float64))
    q = tmp_path / "e8.hde"
    _write_eig(q, lam, U, ldu=16, storage=2)
    with pytest.raises(ValueError):
        bench.read_eig_checkpoint(q)


def test_clock_summary_reports_median_max_and_reasons():
    c = bench.Clocks(0)
    row = lambda sm, mx, reason: ["0", sm, mx, "900.0", "0x0", "Not Active", "Not Active", "Not Active", reason]
    c.samples = [row("2070", "2070", "Not Active"), row("1980", "2070", "Active"), row("2070", "2070", "Not Active"),
                 row("[N/A]", "2070", "Not Active")]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4


class _G:
    def __init__(self, nnz):
        self.nnz = nnz


def test_algorithmic_bytes_per_launch():
    n, nnz, B = 1000, 54000, 62
    ab = bench.algorithmic_bytes({"n": n, "g": _G(nnz)}, B, None)
    vec = n * 64 * 4  # B rounded up to a multiple of 4
    assert ab["spmm"] == 8 * nnz + 4 * (n + 1) + 2 * vec
    assert ab["update"] == 6 * vec and ab["dot"] == 2 * vec and ab["rank"] == vec
    assert ab["spmm_h"] == 8 * nnz + 4 * (n + 1) + vec // 2 + 2 * vec
    assert ab["lr_reduce"] == vec and ab["lr_expand"] == 3 * vec  # no eigenpairs: no U bytes


def test_spmm_traffic_needs_the_profiled_kernel_and_shape(monkeypatch):
    class G:
        nnz = bench.SPMM_NCU["nnz"] * 2

        def tuning(self, B):
            return (bench.SPMM_NCU["slab"], 1)

    wl = {"g": G()}
    monkeypatch.setattr(bench, "spmm_source_sha1", lambda: bench.SPMM_NCU["src_sha1"])
    assert bench.spmm_traffic(wl, bench.SPMM_NCU["B"]) == 2 * bench.SPMM_NCU["dram_bytes"]
    assert bench.spmm_traffic(wl, bench.SPMM_NCU["B"] * 2) is None
    monkeypatch.setattr(bench, "spmm_source_sha1", lambda: "0" * 40)
    assert bench.spmm_traffic(wl, bench.SPMM_NCU["B"]) is None

