"""Replicas on several GPUs: the query stream shards by query and the job's
throughput is timed by the slowest replica.  The host logic runs here as two
gloo ranks on the CPU (127.0.0.1 rendezvous)."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(1.0 + 0.5 * rank)   # rank 1 is the slower replica
    qps = bench.replica_throughput(world, 64, 20, slowest)
    dist.barrier()
    q.put((rank, slowest, qps))
    dist.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.5, 1.5]
    assert all(o[2] == 2 * 64 * 20 / 1.5 for o in out)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_throughput(1, 64, 20, 0.5) == 64 * 20 / 0.5


def test_replicas_draw_disjoint_query_streams():
    import bench
    import synth
    c = synth.get_config("cfg1")
    q0 = synth.queries(bench.query_seed(c.seed, 0), 8, c.d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes)
    q1 = synth.queries(bench.query_seed(c.seed, 1), 8, c.d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes)
    assert q0.shape == q1.shape and not np.allclose(q0, q1)
    # and every replica is reproducible
    assert np.array_equal(q0, synth.queries(bench.query_seed(c.seed, 0), 8, c.d, c.ncl, c.kappa_lo, c.kappa_hi,
                                            c.sizes))
