"""Continuous-batching server: each request's result is the same alone and in
a mix (bitwise), rankings match the fp64 oracle, per-request tolerance and K
are honoured, and admission respects the memory budget."""
import numpy as np
import pytest

import synth
from _helpers import csr_of
from oracle import diffusion as D
from oracle import observe
from oracle import rank as ORank

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(gpu_ctx, cfg1_data):
    import paper_1807_08692_gb300 as hd
    c = cfg1_data["cfg"]
    g = hd.graph_from_csr(gpu_ctx, *csr_of(cfg1_data["A"]))
    r = 50
    eig = hd.eig_from_host(gpu_ctx, g, cfg1_data["lam"][:r], cfg1_data["U"][:, :r], "bf16")
    # 40 extra observation vectors from fresh queries of the same mixture
    Qx = synth.queries(c.seed + 77, 40, c.d, c.ncl, c.kappa_lo, c.kappa_hi)
    yp, yi, yv = observe.observe(cfg1_data["X"], Qx, c.k_y, c.gamma)
    reqs = [(yi[yp[j]:yp[j + 1]], yv[yp[j]:yp[j + 1]]) for j in range(40)]
    return g, eig, reqs


def _run(server, items, iters=2, max_steps=2000):
    """items: list of (step_to_submit, idx, val, tol, K); returns results by position."""
    tickets = {}
    out = {}
    waiting = list(range(len(items)))
    step = 0
    while (waiting or len(out) < len(items)) and step < max_steps:
        for pos in [p for p in waiting if items[p][0] <= step]:
            at, idx, val, tol, K = items[pos]
            tickets[pos] = (server.submit(idx, val, tol, K), K)
            waiting.remove(pos)
        server.step(iters)
        for pos, (t, K) in list(tickets.items()):
            if pos not in out:
                res = server.poll(t, K)
                if res is not None:
                    out[pos] = res
        step += 1
    assert len(out) == len(items)
    return [out[i] for i in range(len(items))]


def test_alone_equals_mix_bitwise(gpu_ctx, served):
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    q_idx, q_val = reqs[0]
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=12, max_iter=500, Kmax=200)
    alone = _run(srv, [(0, q_idx, q_val, 1e-6, 100)])[0]
    mix_items = [(s // 3, i, v, [1e-2, 1e-4, 1e-6][s % 3], [10, 100, 200][s % 3]) for s, (i, v) in enumerate(reqs[1:])]
    mix_items.insert(17, (4, q_idx, q_val, 1e-6, 100))
    mixed = _run(srv, mix_items)
    m = mixed[17]
    assert np.array_equal(alone[0], m[0])
    assert np.array_equal(alone[1].view(np.uint32), m[1].view(np.uint32))
    assert alone[2]["iters"] == m[2]["iters"] and alone[2]["status"] == 0
    # columns ran in several slots while others were admitted and retired
    slots = {r[2]["slot"] for r in mixed}
    assert len(slots) > 4
    srv.close()


def test_served_rankings_match_oracle(gpu_ctx, cfg1_data, served):
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    W = cfg1_data["W"]
    n = cfg1_data["cfg"].n
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=8, max_iter=500, Kmax=100)
    items = [(s // 4, i, v, 1e-6, 100) for s, (i, v) in enumerate(reqs[:16])]
    res = _run(srv, items)
    for (at, i, v, tol, K), (ids, sc, st) in zip(items, res):
        Y = np.zeros((n, 1))
        np.add.at(Y[:, 0], i, v.astype(np.float64))
        x = D.closed_form(W, Y, 0.99)[:, 0]
        ref, _ = ORank.topk(x, K)
        # scores of the served x (not returned) against the closed form at the same ids
        assert ORank.ranks_match(ids, ref, x, 1e-5 * x.max(), scores=sc, x=x, score_tol=1e-3)
        assert st["status"] == 0 and st["relres"] <= 1e-6 * 1.01
        assert st["done_s"] >= st["admit_s"] >= st["submit_s"]
    srv.close()


def test_tolerance_and_k_per_request(gpu_ctx, served):
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, None, "paper", 0.99, max_slots=4, max_iter=800, Kmax=1000)
    i, v = reqs[3]
    loose, tight = _run(srv, [(0, i, v, 1e-2, 10), (0, i, v, 1e-6, 1000)])
    assert loose[2]["iters"] < tight[2]["iters"]
    assert len(loose[0]) == 10 and len(tight[0]) == 1000
    assert loose[2]["relres"] <= 1e-2 and tight[2]["relres"] <= 1e-6 * 1.01
    srv.close()


def test_admission_by_memory_and_errors(gpu_ctx, served, cfg1_data):
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    n = cfg1_data["cfg"].n
    per_slot = 4 * n * 4 + 100 * 8
    srv = hd.Server(gpu_ctx, g, None, "paper", 0.99, max_slots=64, mem_budget=3 * per_slot + 7, Kmax=100)
    assert srv.slots == 3
    with pytest.raises(hd.HDError):
        srv.submit(np.array([n], np.int32), np.array([1.0], np.float32), 1e-6, 10)
    with pytest.raises(hd.HDError):
        srv.submit(np.array([0], np.int32), np.array([1.0], np.float32), 1e-6, 101)
    items = [(0, i, v, 1e-4, 10) for i, v in reqs[:7]]
    res = _run(srv, items)
    assert {r[2]["slot"] for r in res} <= {0, 1, 2}
    srv.close()
    with pytest.raises(hd.HDError):
        hd.Server(gpu_ctx, g, None, "paper", 0.99, max_slots=4, mem_budget=100, Kmax=10)


def test_completed_reports_each_ticket_once(gpu_ctx, served):
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=4, max_iter=500, Kmax=50)
    tickets = [srv.submit(i, v, [1e-2, 1e-4, 1e-6][k % 3], 20) for k, (i, v) in enumerate(reqs[:9])]
    seen = []
    for _ in range(500):
        busy = srv.step(1)
        seen += srv.completed(max_tickets=3)
        if not busy:
            break
    seen += srv.completed()
    assert sorted(seen) == sorted(tickets) and len(set(seen)) == len(seen)
    assert srv.completed() == []
    for t in seen:
        ids, sc, st = srv.poll(t, 20)
        assert st["status"] == 0 and len(ids) == 20
    srv.close()


def test_narrow_and_wide_lanes_agree(gpu_ctx, served):
    # one request alone runs in the narrow lane (slots >= 12 here), the same
    # request submitted with a crowd runs in the wide lane: same bits
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=12, max_iter=500, Kmax=50)
    q_idx, q_val = reqs[5]
    alone = _run(srv, [(0, q_idx, q_val, 1e-6, 50)], iters=1)[0]
    assert alone[2]["slot"] >= 12  # narrow lane
    crowd = [(0, i, v, 1e-4, 20) for i, v in reqs[10:20]] + [(0, q_idx, q_val, 1e-6, 50)]
    out = _run(srv, crowd, iters=1)
    m = out[-1]
    assert m[2]["slot"] < 12  # wide lane
    assert np.array_equal(alone[0], m[0])
    assert np.array_equal(alone[1].view(np.uint32), m[1].view(np.uint32))
    assert alone[2]["iters"] == m[2]["iters"]
    srv.close()


def test_served_request_equals_batch_solve(gpu_ctx, served):
    # a request alone is taken by a free column at the scalar step of one
    # iteration (whose direction forms z0 = M^-1 y) and then runs the batch
    # solver's PCG iterations for the same y, with the same ranking
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=8, max_iter=500, Kmax=20)
    for q in (7, 8):
        i, v = reqs[q]
        t = srv.submit(i, v, 1e-6, 20)
        steps, res = 0, None
        while res is None and steps < 100:
            srv.step(1)
            steps += 1
            res = srv.poll(t, 20)
        assert res is not None and res[2]["status"] == 0
        assert steps == res[2]["iters"] + 1
        X, it, rr, st = hd.query_batch(gpu_ctx, g, eig, "pcg", np.array([0, len(i)], np.int32), i, v, 0.99, 1e-6, 500)
        assert st[0] == 0 and abs(int(it[0]) - res[2]["iters"]) <= 1
        x = X[:, 0].cpu().numpy().astype(np.float64)
        ref, _ = ORank.topk(x, 20)
        assert ORank.ranks_match(res[0], ref, x, 1e-5 * x.max(), scores=res[1], x=x, score_tol=1e-3)
    srv.close()


def test_stopping_column_takes_the_next_request(gpu_ctx, served):
    # one column: the request queued behind another is taken at the scalar step
    # of the iteration where its predecessor stops, so the column never idles
    # between them, and its result is the same bits as alone
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=1, max_iter=500, Kmax=20)
    assert srv.slots == 1
    alone = _run(srv, [(0, *reqs[21], 1e-6, 20)], iters=1)[0]
    srv.completed()
    ta = srv.submit(*reqs[20], 1e-4, 20)
    tb = srv.submit(*reqs[21], 1e-6, 20)
    done, step = {}, 0
    while len(done) < 2 and step < 300:
        srv.step(1)
        step += 1
        for tk in srv.completed():
            done[tk] = (step, srv.poll(tk, 20))
    (sa, ra), (sb, rb) = done[ta], done[tb]
    assert ra[2]["status"] == 0 and rb[2]["status"] == 0
    assert sa == ra[2]["iters"] + 1
    assert sb == sa + rb[2]["iters"]
    assert ra[2]["slot"] == rb[2]["slot"] == 0
    assert np.array_equal(rb[0], alone[0])
    assert np.array_equal(rb[1].view(np.uint32), alone[1].view(np.uint32))
    assert rb[2]["iters"] == alone[2]["iters"]
    srv.close()


def test_requests_that_need_no_iteration(gpu_ctx, served):
    # y = 0 and tol >= 1 finish at staging with x = 0: ids 0 .. K-1, score 0
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=4, max_iter=500, Kmax=20)
    t0 = srv.submit(np.zeros(0, np.int32), np.zeros(0, np.float32), 1e-6, 5)
    t1 = srv.submit(np.array([3, 3], np.int32), np.array([1.0, -1.0], np.float32), 1e-6, 5)
    t2 = srv.submit(*reqs[4], 1.0, 5)
    t3 = srv.submit(*reqs[4], 1e-4, 5)
    srv.step(1)
    for t, status in ((t0, hd.COL_EMPTY), (t1, hd.COL_EMPTY), (t2, hd.COL_CONVERGED)):
        ids, sc, st = srv.poll(t, 5)
        assert st["status"] == status and st["iters"] == 0
        assert list(ids) == [0, 1, 2, 3, 4] and not sc.any()
    assert srv.poll(t3, 5) is None
    while srv.step(1):
        pass
    ids, sc, st = srv.poll(t3, 5)
    assert st["status"] == 0 and st["iters"] > 0
    srv.close()


def test_cancel_queued_and_running_requests(gpu_ctx, served):
    # a queued request leaves the queue, a running one frees its column at
    # once; neither is ranked, and the others get exactly their results alone
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=4, max_iter=500, Kmax=20)
    alone = _run(srv, [(0, *reqs[11], 1e-6, 20)], iters=1)[0]
    srv.completed()                  # already polled by _run
    t = [srv.submit(i, v, 1e-6, 20) for i, v in (reqs[11], reqs[12], reqs[13], reqs[14], reqs[15], reqs[16])]
    srv.step(1)                      # four running (wide lane), two queued
    srv.cancel(t[5])                 # queued
    srv.cancel(t[1])                 # running
    with pytest.raises(hd.HDError):
        srv.cancel(12345)
    done = {}
    for _ in range(200):
        busy = srv.step(1)
        for tk in srv.completed():
            done[tk] = srv.poll(tk, 20)
        if not busy:
            break
    for tk in srv.completed():
        done[tk] = srv.poll(tk, 20)
    assert sorted(done) == sorted(t)
    assert done[t[1]][2]["status"] == 4 and done[t[5]][2]["status"] == 4
    for k in (0, 2, 3, 4):
        assert done[t[k]][2]["status"] == 0
    assert np.array_equal(done[t[0]][0], alone[0])
    assert np.array_equal(done[t[0]][1].view(np.uint32), alone[1].view(np.uint32))
    # the queued request that followed got the cancelled one's column
    assert done[t[4]][2]["slot"] == done[t[1]][2]["slot"]
    srv.close()


def test_non_finite_observations_rejected(gpu_ctx, served):
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    i, v = reqs[2]
    bad = np.array(v, np.float32)
    bad[1] = np.nan
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=4, max_iter=500, Kmax=20)
    with pytest.raises(hd.HDError):
        srv.submit(i, bad, 1e-6, 20)
    srv.close()
    y_ptr = np.array([0, len(i)], np.int32)
    with pytest.raises(hd.HDError):
        hd.query_batch(gpu_ctx, g, eig, "pcg", y_ptr, i, bad, 0.99, 1e-6, 100)
    bad[1] = np.inf
    with pytest.raises(hd.HDError):
        hd.query_batch(gpu_ctx, g, None, "paper", y_ptr, i, bad, 0.99, 1e-6, 100)
    # the context stays usable
    X, it, rr, st = hd.query_batch(gpu_ctx, g, eig, "pcg", y_ptr, i, v, 0.99, 1e-6, 500)
    assert st[0] == 0


def test_random_traffic_with_cancellations(gpu_ctx, served):
    # 60 requests at seeded random steps with mixed tolerances and K, a queue
    # longer than the free columns at times (staged requests that no column
    # takes go back to the queue), 1 or 3 iterations per step, and 8 requests
    # cancelled while queued or running: every ticket is reported once, the
    # cancelled ones with status CANCELLED, and every other request gets the
    # bits it gets alone
    import paper_1807_08692_gb300 as hd
    g, eig, reqs = served
    rng = np.random.default_rng(1807)
    n_req = 60
    at = np.sort(rng.integers(0, 40, n_req))
    tols = rng.choice([1e-2, 1e-4, 1e-6], n_req)
    Ks = rng.choice([5, 20, 50], n_req)
    which = rng.integers(0, len(reqs), n_req)
    cancel_at = {int(p): int(at[p] + rng.integers(0, 6)) for p in rng.choice(n_req, 8, replace=False)}
    srv = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=8, max_iter=500, Kmax=50)
    tickets, out, seen = {}, {}, []
    step = 0
    while (len(tickets) < n_req or len(out) < n_req) and step < 3000:
        for p in range(n_req):
            if at[p] == step and p not in tickets:
                tickets[p] = srv.submit(*reqs[which[p]], float(tols[p]), int(Ks[p]))
        for p, s in cancel_at.items():
            if s == step and p in tickets and p not in out:
                srv.cancel(tickets[p])
        srv.step(1 + 2 * (step % 5 == 4))
        for t in srv.completed():
            seen.append(t)
        for p, t in tickets.items():
            if p not in out and t in seen:
                res = srv.poll(t, int(Ks[p]))
                assert res is not None
                out[p] = res
        step += 1
    assert len(out) == n_req and sorted(seen) == sorted(tickets.values())
    assert len(set(seen)) == len(seen)
    srv.close()
    cancelled = [p for p in range(n_req) if out[p][2]["status"] == hd.COL_CANCELLED]
    assert set(cancelled) <= set(cancel_at)
    solo = hd.Server(gpu_ctx, g, eig, "pcg", 0.99, max_slots=8, max_iter=500, Kmax=50)
    for p in range(n_req):
        if p in cancelled:
            continue
        ids, sc, st = out[p]
        assert st["status"] == 0
        a_ids, a_sc, a_st = _run(solo, [(0, *reqs[which[p]], float(tols[p]), int(Ks[p]))], iters=1)[0]
        assert np.array_equal(ids, a_ids), p
        assert np.array_equal(sc.view(np.uint32), a_sc.view(np.uint32)), p
        assert st["iters"] == a_st["iters"], p
    solo.close()
