"""Throughput of the hybrid diffusion query path on GB300.

One step = one batch of B queries through the whole online path: observation
scatter, spectral term, CG iterations of the temporal term (Eq. 17-20) and
the top-K ranking (Sec. 3), with inputs resident in HBM.  The workload is the
1,000,000-node k=50 graph of synthetic d=2048 bf16 vMF descriptors.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the query stream shards by query; there is no exchange step).  Rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/sec and p50/p99 latency at 1M nodes, hybrid BF16-U_r vs pure CG, equal FP64 error"
TOL_REL = 1e-4
LADDER = [1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg3")
    ap.add_argument("--n", type=int, default=0, help="override n (smaller profiling case)")
    ap.add_argument("--d", type=int, default=0)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--r", type=int, default=200)
    ap.add_argument("--mode", default="pcg")
    ap.add_argument("--storage", default="bf16")
    ap.add_argument("--topk", type=int, default=100)
    ap.add_argument("--restarts", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=2, help="query columns timed on the oracle")
    ap.add_argument("--calib-cols", type=int, default=32,
                    help="calibration queries solved by the fp64 oracle (the accuracy reference)")
    ap.add_argument("--check-cols", type=int, default=8,
                    help="queries of the timed batch whose scores are checked against the fp64 oracle")
    ap.add_argument("--export-inputs", default="",
                    help="(reference arm) write the workload's graph, eigenpairs and observations here and exit")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the r=0 leg and calibration (profiling runs)")
    ap.add_argument("--serve-rates", default="100,300,1000,3000,10000,20000",
                    help="Poisson arrival rates (req/s) of the serving leg; empty to skip")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests per rate after warm-up (the serving protocol asks for 10000)")
    ap.add_argument("--serve-slots", type=int, default=128)
    ap.add_argument("--serve-saturated", type=int, default=0,
                    help="requests queued at once for a saturated-server step profile (0: skip)")
    ap.add_argument("--sweep", type=int, default=1, help="run the storage / rank / batch sweep")
    ap.add_argument("--sweep-batches", default="1,16,256")
    ap.add_argument("--shortlist", type=int, default=75000, help="Temporal† shortlist size (0: skip the leg)")
    ap.add_argument("--sweep-r400", type=int, default=1, help="add an r=400 leg (its own Lanczos) to the sweep")
    ap.add_argument("--trunc-iters", type=int, default=20, help="Temporal† CG iterations (Table 1: 20)")
    ap.add_argument("--small-leg", type=int, default=1,
                    help="time the 2,000-node clustered workload (d=128; r=50 against r=0) as well")
    ap.add_argument("--converged-r", type=int, default=1,
                    help="rank of the eigenpairs converged to residual 1e-5 for the paper's-form leg (0: skip)")
    ap.add_argument("--converged-restarts", type=int, default=30,
                    help="restart limit of that Lanczos run")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class Clocks:
    """Sample nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi's start-up (NVML initialisation) must not overlap the timed
        # steps: wait for its first sample (at most 3 s)
        t0 = time.time()
        while not self.samples and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for nm, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ------------------------------------------------------------------ workload
def build_workload(args, ctx, rank):
    """Descriptors, graph, observations and eigenpairs of the benchmark workload."""
    import torch
    import paper_1807_08692_gb300 as hd
    import synth
    c = synth.get_config(args.workload)
    n = args.n or c.n
    d = args.d or c.d
    t0 = time.time()
    R = c.regions
    if R > 1:
        # regional workload: images of R region descriptors, image-major rows
        n = n // R * R
        X, _ = synth.regional_database(c.seed, n // R, R, d, c.ncl, c.kappa_lo, c.kappa_hi,
                                       c.extra.get("p_stay", 0.8))
    else:
        X, _ = synth.database(c.seed, n, d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes, c.zipf_s)
    Xt = torch.from_numpy(X).to(torch.bfloat16 if c.dtype == "bf16" else torch.float32).cuda()
    del X
    t_gen = time.time() - t0
    t0 = time.time()
    g = hd.build_graph(ctx, Xt, c.k, c.gamma)
    torch.cuda.synchronize()
    t_graph = time.time() - t0
    # queries: one calibration batch and the timed batch (different draws), sized
    # for the largest batch of the sweep
    bmax = max([args.batch] + ([int(b) for b in args.sweep_batches.split(",") if b] if args.sweep else []))
    nq = 2 * bmax
    if R > 1:
        # query images drawn like the database's (own seed), one observation per image
        Qv, _ = synth.regional_database(query_seed(c.seed + 7000, rank), nq, R, d, c.ncl, c.kappa_lo, c.kappa_hi,
                                        c.extra.get("p_stay", 0.8))
        Qt = torch.from_numpy(Qv).to(Xt.dtype).cuda()
        yp, yi, yv = hd.observe_regional(ctx, Xt, Qt, R, c.k_y, c.gamma)
    else:
        Qv = synth.queries(query_seed(c.seed, rank), nq, d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes, c.zipf_s)
        Qt = torch.from_numpy(Qv).to(Xt.dtype).cuda()
        yp, yi, yv = hd.observe(ctx, Xt, Qt, c.k_y, c.gamma)
    yall = (yp, yi, yv)
    B = args.batch
    cal, tim = split_batches(yall, B, bmax)
    t0 = time.time()
    eig, lam, res, conv, U32 = None, None, None, None, None
    wl_restarts = None
    if args.r > 0:
        # fp32 Ritz vectors once; each storage format is made from them
        e32, lam, res, conv = hd.eigendecompose(ctx, g, args.r, block=32, tol=1e-5, max_restarts=args.restarts,
                                                storage="f32")
        wl_restarts = e32.restarts
        _, U32 = e32.export()
        e32.close()
        eig = hd.eig_from_host(ctx, g, lam, U32, args.storage)
    torch.cuda.synchronize()
    t_eig = time.time() - t0
    return {"cfg": c, "n": n, "d": d, "g": g, "Xt": Xt, "Qt": Qt, "pool": R if R > 1 else 0, "cal": cal, "tim": tim,
            "yall": yall, "bmax": bmax,
            "eig": eig, "lam": lam, "U32": U32, "res": res, "conv": conv, "restarts": wl_restarts, "t_gen": t_gen,
            "t_graph": t_graph, "t_eig": t_eig}


def split_batches(yall, B, bmax):
    """Calibration batch = queries [0, B), timed batch = queries [bmax, bmax + B)."""
    yp, yi, yv = yall

    def take(q0):
        s, e = yp[q0], yp[q0 + B]
        return ((yp[q0:q0 + B + 1] - s).astype(np.int32), yi[s:e].copy(), yv[s:e].copy())

    return take(0), take(bmax)


def calibrate(ctx, wl, eig, mode, alpha, cal=None):
    """Loosest ladder tolerance whose max rel-l2 against the fp64 oracle's
    solution (wl["ref_cal"], calibration queries 0 .. calib_cols - 1, solved to
    relres 1e-12) is <= TOL_REL over the calibration columns the batch holds.
    The timed batch's own error against the oracle is measured separately
    (accuracy).  Returns (tol, max rel-l2 at it, most iterations)."""
    import paper_1807_08692_gb300 as hd
    g = wl["g"]
    yp, yi, yv = wl["cal"] if cal is None else cal
    B = len(yp) - 1
    ref = wl["ref_cal"]
    m = min(B, ref.shape[1])
    refn = np.linalg.norm(ref[:, :m], axis=0)
    err = None
    for tol in LADDER:
        X, it, rr, st = hd.query_batch(ctx, g, eig, mode, yp, yi, yv, alpha, tol, 2000)
        x = X[:, :m].double().cpu().numpy()
        err = float((np.linalg.norm(x - ref[:, :m], axis=0) / refn).max())
        if err <= TOL_REL:
            return tol, err, int(np.max(it))
    return LADDER[-1], err, int(np.max(it))


# ------------------------------------------------------------------ timed legs
FAMILIES = ["spmm", "spmm_h", "to_half", "resid", "dot", "update", "direction", "colsq", "lr_reduce", "lr_expand",
            "scalar", "rank"]


def time_leg(ctx, wl, eig, mode, tol, alpha, K, W, B, topk, profile, tim=None):
    import torch
    import paper_1807_08692_gb300 as hd
    g = wl["g"]
    yp, yi, yv = wl["tim"] if tim is None else tim
    # inputs resident in HBM
    ypd = torch.from_numpy(yp).cuda()
    yid = torch.from_numpy(yi).cuda()
    yvd = torch.from_numpy(yv).cuda()
    told = torch.full((B,), tol, dtype=torch.float32, device="cuda")
    X = torch.empty((wl["n"], (B + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    itd = torch.zeros(B, dtype=torch.int32, device="cuda")
    rrd = torch.zeros(B, dtype=torch.float32, device="cuda")
    std = torch.zeros(B, dtype=torch.int32, device="cuda")
    idx = torch.empty((B, topk), dtype=torch.int32, device="cuda")
    sc = torch.empty((B, topk), dtype=torch.float32, device="cuda")
    Kh = np.full(B, topk, np.int32)

    def step():
        hd.query_batch(ctx, g, eig, mode, ypd, yid, yvd, alpha, told, 2000, X=X, ldx=X.shape[1], iters=itd,
                       relres=rrd, status=std)
        hd.rank(ctx, X[:, :B], Kh, topk, pool=wl["pool"], idx=idx, score=sc)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    if profile:
        ctx.profile(True)
        for f in FAMILIES:
            ctx.profile_read(f)
    l0 = ctx.launches()
    s = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push(f"timed_{mode}_r{0 if eig is None else eig.r}")
    evs[0].record(s)
    for k in range(K):
        step()
        evs[k + 1].record(s)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = ctx.launches() - l0
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(K)]
    fam = {}
    if profile:
        for f in FAMILIES:
            cnt, ms, busy = ctx.profile_read(f, busy=True)
            fam[f] = (cnt, ms, busy)
        ctx.profile(False)
    total_ms = evs[0].elapsed_time(evs[K])
    return {"ms": per, "total_ms": total_ms, "launches": launches, "fam": fam,
            "iters": itd.cpu().numpy(), "status": std.cpu().numpy(), "relres": rrd.cpu().numpy(),
            "X": X[:, :B], "idx": idx, "sc": sc}


def e2e_leg(ctx, wl, eig, mode, tol, alpha, K, B, topk):
    """Same metric through the public API with HOST buffers: the observation
    arrays go host->device and the rankings device->host inside each step, from
    and into pinned host memory (numpy views of page-locked torch tensors)."""
    import torch
    import paper_1807_08692_gb300 as hd
    g = wl["g"]

    def pinned(a, dtype):
        t = torch.empty(a.shape if hasattr(a, "shape") else a, dtype=dtype, pin_memory=True)
        if hasattr(a, "shape"):
            t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
        return t.numpy()

    yp, yi, yv = (pinned(a, dt) for a, dt in zip(wl["tim"], (torch.int32, torch.int32, torch.float32)))
    tolh = pinned(np.full(B, tol, np.float32), torch.float32)
    X = torch.empty((wl["n"], (B + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    Kh = np.full(B, topk, np.int32)
    idx = pinned((B, topk), torch.int32)
    sc = pinned((B, topk), torch.float32)
    times = []
    for k in range(K + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hd.query_batch(ctx, g, eig, mode, yp, yi, yv, alpha, tolh, 2000, X=X, ldx=X.shape[1])
        hd.rank(ctx, X[:, :B], Kh, topk, pool=wl["pool"], idx=idx, score=sc)
        torch.cuda.synchronize()
        if k:
            times.append(time.perf_counter() - t0)
    h2d = yp.nbytes + yi.nbytes + yv.nbytes + tolh.nbytes
    d2h = idx.nbytes + sc.nbytes + 3 * 4 * B
    return float(np.sum(times)), h2d, d2h


# DRAM bytes per launch of the SpMM measured by ncu (the SpMM summary under profiles/):
# k_spmm<32> on a 1M-node k=50 graph (d=256 descriptors, nnz 62,097,728), B=64.
# Scaled to another graph by nnz (the gathered rows dominate); reported only
# while the kernel source still hashes to the value the counters were taken on.
SPMM_NCU = {"dram_bytes": 8468885888, "nnz": 62097728, "n": 1000000, "B": 64, "slab": 32,
            "src_sha1": "b0a31b960a82f4637d356dc47bf415d4c28ca76d"}


def spmm_source_sha1():
    import hashlib
    src = open(os.path.join(ROOT, "paper_1807_08692_gb300", "csrc", "hd_solve.cu")).read()
    a = src.index("k_spmm(const int32_t* rp,")
    b = src.index("\n}\n", a)
    return hashlib.sha1(src[a:b].encode()).hexdigest()


def spmm_traffic(wl, B):
    tun = wl["g"].tuning(B)
    if SPMM_NCU["dram_bytes"] is None or SPMM_NCU["src_sha1"] != spmm_source_sha1() or B != SPMM_NCU["B"] \
            or tun is None or tun[0] != SPMM_NCU["slab"] or tun[1] != 1:
        return None
    return int(SPMM_NCU["dram_bytes"] * wl["g"].nnz / SPMM_NCU["nnz"])


def algorithmic_bytes(wl, B, eig):
    """Algorithmic bytes per launch of each kernel family (each operand once)."""
    n = wl["n"]
    nnz = wl["g"].nnz
    Bp = (B + 3) // 4 * 4
    vec = n * Bp * 4
    su = {"f32": 4, "bf16": 2, "fp8": 1}
    ub = 0
    if eig is not None:
        ldu = (eig.r + 15) // 16 * 16
        ub = n * ldu * su[{0: "f32", 1: "bf16", 2: "fp8"}[eig.storage]]
    return {
        "spmm": 8 * nnz + 4 * (n + 1) + 2 * vec,      # W (col + val), row_ptr, P once, Q
        "resid": 8 * nnz + 4 * (n + 1) + 2 * vec,     # the same for b - A x (X once, T)
        "spmm_h": 8 * nnz + 4 * (n + 1) + vec // 2 + 2 * vec,  # fp16 copy of P once, own rows of P, Q
        "to_half": 2 * vec + vec // 2,                 # max |P_j| (read P), convert (read P, write the copy)
        "dot": 2 * vec,                                 # read P, Q (P^T Q partials)
        "update": 6 * vec,                              # read X, R, P, Q; write X, R
        "direction": 3 * vec,                           # read R, P; write P
        "lr_reduce": ub + vec,                          # U and R once
        "lr_expand": ub + 3 * vec,                      # U, R, P; write P
        "rank": vec,                                    # X once (top-K)
    }


# ------------------------------------------------------------------ the fp64 oracle (cpu_baseline leg)
# The oracle runs only in this section: untimed, it solves the accuracy
# references of the metric ("equal FP64 error"); timed on a bounded sample, it
# is the CPU baseline.  Its inputs are the workload's graph W (rows checked
# against the oracle's brute-force k-NN in the tests) and, for the timed
# hybrid sample, the fp32 eigenpairs; the references use plain CG, which
# needs no eigenpairs.

def oracle_threads():
    return max(1, os.cpu_count() or 1)


def oracle_inputs(wl):
    """W (fp64 CSR) and the fp32 eigenpairs, exported from the device once."""
    import scipy.sparse as sp
    n = wl["n"]
    if "oracle_inputs" not in wl:
        rp, col, val, _ = wl["g"].export()
        W = sp.csr_matrix((val.astype(np.float64), col, rp), shape=(n, n))
        if wl.get("U32") is not None:
            lam, U = wl["lam"], wl["U32"].astype(np.float64)
        elif wl["eig"] is not None:
            lam, U = wl["eig"].export()
            U = U.astype(np.float64)
        else:
            lam, U = np.zeros(0), np.zeros((n, 0))
        wl["oracle_inputs"] = (W, lam, U)
    return wl["oracle_inputs"]


def oracle_references(wl, args, alpha):
    """x* = (1 - alpha)(I - alpha W)^-1 y (Eq. 3) by the oracle's fp64 CG on
    L_alpha(W) to relres 1e-12, for calibration queries 0 .. calib_cols - 1 and
    the first check_cols queries of the timed batch."""
    from oracle import diffusion, observe
    W, _, _ = oracle_inputs(wl)
    n = wl["n"]

    def dense(batch, m):
        yp, yi, yv = batch
        m = min(m, len(yp) - 1)
        return observe.dense(n, yp[:m + 1], yi[:yp[m]], yv[:yp[m]].astype(np.float64))

    Yc, Yt = dense(wl["cal"], args.calib_cols), dense(wl["tim"], args.check_cols)
    t0 = time.perf_counter()
    X, it, rel = diffusion.cg_columns(diffusion.laplacian_op(W, alpha, oracle_threads()), np.hstack([Yc, Yt]),
                                      1e-12, 1000)
    wl["ref_cal"], wl["ref_tim"] = X[:, :Yc.shape[1]], X[:, Yc.shape[1]:]
    return {"columns": int(X.shape[1]), "relres_max": float(rel.max()), "iters_max": int(it.max()),
            "seconds": round(time.perf_counter() - t0, 1), "threads": oracle_threads()}


def cpu_oracle(W, lam, U, Y, alpha, tol, with_cg=False):
    """Time the fp64 oracle's hybrid PCG (Form S) on the columns of Y, and
    optionally its pure CG (r = 0) on the same columns."""
    from oracle import diffusion
    t0 = time.perf_counter()
    x, iters = diffusion.hybrid_pcg(W, U, lam, Y, alpha, tol, 2000)
    dt = time.perf_counter() - t0
    if not with_cg:
        return dt, iters
    t0 = time.perf_counter()
    _, it0, _ = diffusion.temporal(W, Y, alpha, tol, 2000)
    dt0 = time.perf_counter() - t0
    return dt, iters, dt0, it0


def accuracy(wl, X, idx, sc, topk, rankings=True):
    """The timed batch's first check_cols columns against the oracle's
    references: rel-l2 of the scores (max, median), and how many top-K lists
    are valid rankings of the oracle's scores (distinct ids, nothing missing,
    order up to ties within 1e-5 of the largest score, scores equal to the
    ranked vector's); per image for the regional workload."""
    from oracle import rank as ORank
    ref = wl["ref_tim"]
    m = min(ref.shape[1], X.shape[1])
    x = X[:, :m].double().cpu().numpy()
    err = np.linalg.norm(x - ref[:, :m], axis=0) / np.linalg.norm(ref[:, :m], axis=0)
    out = {"oracle_rel_l2_max": float(err.max()), "oracle_rel_l2_median": float(np.median(err)),
           "oracle_columns": int(m)}
    if not rankings:
        return out
    ids, scs = idx[:m].cpu().numpy(), sc[:m].cpu().numpy()
    pool = wl["pool"]
    ok = 0
    for j in range(m):
        rj = ORank.pooled(ref[:, j], pool) if pool else ref[:, j]
        xj = ORank.pooled(x[:, j], pool) if pool else X[:, j].cpu().numpy()
        top, _ = ORank.topk(rj, topk)
        ok += bool(ORank.ranks_match(ids[j], top, rj, 1e-5 * rj.max(), scores=scs[j], x=xj,
                                     score_tol=1e-5 if pool else 0.0))
    out[f"top{topk}_valid"] = f"{ok}/{m}"
    return out


def timed_columns(wl, columns):
    from oracle import observe
    yp, yi, yv = wl["tim"]
    return observe.dense(wl["n"], yp[:columns + 1], yi[:yp[columns]], yv[:yp[columns]].astype(np.float64))


# ------------------------------------------------------------------ sweep (storage, rank, batch)
def sweep_leg(ctx, wl, args, alpha):
    """Short timed legs over the recipe's knobs, each at its own calibrated
    tolerance: U storage (f32 / bf16 / fp8 at r), a smaller rank, the paper's
    form with bf16 U, and batch sizes."""
    import paper_1807_08692_gb300 as hd
    out = []
    g, lam, U32 = wl["g"], wl["lam"], wl["U32"]

    def run(label, eig, mode, B, **kw):
        cal, tim = split_batches(wl["yall"], B, wl["bmax"])
        tol, err, _ = calibrate(ctx, wl, eig, mode, alpha, cal=cal)
        leg = time_leg(ctx, wl, eig, mode, tol, alpha, 5, 2, B, args.topk, False, tim=tim)
        ms = leg["total_ms"] / 5
        acc = accuracy(wl, leg["X"], leg["idx"], leg["sc"], args.topk, rankings=False)
        out.append({"leg": label, "mode": mode, "B": B, "tol": tol, "calib_rel_err": err,
                    "meets_1e-4": bool(err is not None and err <= TOL_REL and acc["oracle_rel_l2_max"] <= TOL_REL),
                    "timed_rel_l2_max": acc["oracle_rel_l2_max"], "iters_max": int(leg["iters"].max()),
                    "ms_per_batch": round(ms, 3), "qps": round(B / ms * 1e3, 1), **kw})

    if U32 is not None:
        r = U32.shape[1]
        for st in ("f32", "fp8"):
            e = hd.eig_from_host(ctx, g, lam, U32, st)
            run(f"pcg r={r} {st}", e, "pcg", args.batch, r=r, storage=st)
            e.close()
        for r2 in sorted({1, min(50, r), min(100, r)}):
            if r2 == r:
                continue
            e = hd.eig_from_host(ctx, g, lam[:r2], np.ascontiguousarray(U32[:, :r2]), "bf16")
            run(f"pcg r={r2} bf16", e, "pcg", args.batch, r=r2, storage="bf16")
            e.close()
        if args.sweep_r400 and r < 400:
            # the top of the rank range of the paper's sweep: its own Lanczos run
            t0 = time.time()
            e4, lam4, res4, conv4 = hd.eigendecompose(ctx, g, 400, block=32, tol=1e-5, max_restarts=args.restarts,
                                                      storage="bf16")
            t_l = time.time() - t0
            run("pcg r=400 bf16", e4, "pcg", args.batch, r=400, storage="bf16", lanczos_s=round(t_l, 1),
                lambda_r=round(float(lam4[-1]), 5))
            e4.close()
        run(f"paper r={r} {args.storage}", wl["eig"], "paper", args.batch, r=r, storage=args.storage)
        # SHybrid (Sec. 5.3): 99% of the embedding's entries dropped
        es = wl["eig"].sparsify(0.99)
        run(f"pcg r={r} {args.storage} sparse 0.99", es, "pcg", args.batch, r=r, storage=args.storage,
            sparsity=0.99, u_nnz=es.nnz)
        run(f"paper r={r} {args.storage} sparse 0.99", es, "paper", args.batch, r=r, storage=args.storage,
            sparsity=0.99, u_nnz=es.nnz)
        es.close()
        rc_ = args.converged_r
        if rc_ > 0:
            # Theorem 1 (Eq. 15) holds for exact eigenpairs: the paper's form on
            # eigenpairs converged to ||W u - l u|| <= 1e-5, stored in fp32.  On
            # this graph only lambda_1 = 1 is isolated (lambda_2 .. lambda_200 lie
            # within 0.002 of each other), so the default rank is 1.
            t0 = time.time()
            ec, lamc, resc, convc = hd.eigendecompose(ctx, g, rc_, block=32, tol=1e-5,
                                                      max_restarts=args.converged_restarts, storage="f32")
            t_c = time.time() - t0
            info = dict(r=rc_, storage="f32", lanczos_s=round(t_c, 1), lanczos_restarts=ec.restarts,
                        lanczos_converged=bool(convc), lanczos_max_resid=float(np.max(resc)),
                        lambda_r=round(float(lamc[-1]), 5))
            run(f"paper r={rc_} f32 converged", ec, "paper", args.batch, **info)
            run(f"pcg r={rc_} f32 converged", ec, "pcg", args.batch, **info)
            ec.close()
    for b in [int(x) for x in args.sweep_batches.split(",") if x]:
        run(f"{args.mode} r={args.r} B={b}", wl["eig"], args.mode, b, r=args.r, storage=args.storage)
        run(f"cg r=0 B={b}", None, "paper", b, r=0, storage=None)
    return out


def small_leg(ctx, args, alpha):
    """The 2,000-node workload (d=128, 20 vMF components, k=30, 16 queries, top-10
    observations): real clusters, so lambda_2 .. lambda_20 sit near 0.6-0.7 and the
    hybrid's rank matters.  Graph on the device, eigenpairs by Lanczos; both legs
    calibrated against the oracle's fp64 CG like the headline."""
    import torch
    import paper_1807_08692_gb300 as hd
    import synth
    from oracle import diffusion, observe
    c = synth.get_config("cfg1")
    X, _ = synth.database(c.seed, c.n, c.d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes)
    Q = synth.queries(c.seed, 2 * c.batch, c.d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes)
    Xt = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Qt = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).cuda()
    g = hd.build_graph(ctx, Xt, c.k, c.gamma)
    yp, yi, yv = hd.observe(ctx, Xt, Qt, c.k_y, c.gamma)
    B = c.batch
    sub = {"n": c.n, "g": g, "pool": 0, "yall": (yp, yi, yv), "bmax": B}
    sub["cal"], sub["tim"] = split_batches(sub["yall"], B, B)
    rp, col, val, _ = g.export()
    import scipy.sparse as sp
    W = sp.csr_matrix((val.astype(np.float64), col, rp), shape=(c.n, c.n))

    def dense(batch):
        p, i, v = batch
        return observe.dense(c.n, p, i, v.astype(np.float64))

    Y = np.hstack([dense(sub["cal"]), dense(sub["tim"])])
    Xr, _, _ = diffusion.cg_columns(diffusion.laplacian_op(W, alpha), Y, 1e-12, 5000)
    sub["ref_cal"], sub["ref_tim"] = Xr[:, :B], Xr[:, B:]
    eig, lam, res, conv = hd.eigendecompose(ctx, g, 50, block=16, tol=1e-5, max_restarts=50, storage="bf16")
    out = {"workload": f"{c.name}: n={c.n}, d={c.d}, k={c.k}, nnz={g.nnz}, B={B}", "lambda_2": round(float(lam[1]), 4),
           "lambda_50": round(float(lam[-1]), 4), "lanczos_converged": bool(conv)}
    for label, e, mode in (("hybrid PCG r=50 bf16", eig, "pcg"), ("pure CG r=0", None, "paper")):
        tol, err, _ = calibrate(ctx, sub, e, mode, alpha)
        leg = time_leg(ctx, sub, e, mode, tol, alpha, 50, 5, B, 10, False)
        ms = leg["total_ms"] / 50
        acc = accuracy(sub, leg["X"], leg["idx"], leg["sc"], 10)
        out[label] = {"tol": tol, "iters_max": int(leg["iters"].max()), "ms_per_batch": round(ms, 4),
                      "qps": round(B / ms * 1e3, 1), "timed_rel_l2_max": acc["oracle_rel_l2_max"],
                      "top10_valid": acc["top10_valid"]}
    eig.close()
    return out


def truncated_leg(ctx, wl, args, alpha, tol_ref):
    """Temporal† (Sec. 3.1; Table 1: 20 iterations, 75k shortlist): CG on each
    query's shortlist subgraph.  The shortlists (top-s database items by
    descriptor similarity, the paper's excluded NN search) are prepared
    outside the timed region.  Reported with its truncation error against the
    full-graph solution on the shortlist."""
    import torch
    import paper_1807_08692_gb300 as hd
    B, s = args.batch, min(args.shortlist, wl["n"])
    bmax = wl["bmax"]
    Q = wl["Qt"][bmax:bmax + B]
    sims = (Q.float() @ wl["Xt"].float().T) if wl["Xt"].dtype == torch.float32 else (Q @ wl["Xt"].T).float()
    sl = torch.topk(sims, s, dim=1).indices.to(torch.int32)
    del sims
    sl_idx = sl.reshape(-1).contiguous()
    sl_ptr = np.arange(B + 1, dtype=np.int32) * s
    yp, yi, yv = wl["tim"]
    ypd, yid, yvd = (torch.from_numpy(a).cuda() for a in (yp, yi, yv))
    X = torch.empty((s, B), dtype=torch.float32, device="cuda")
    for _ in range(2):
        hd.temporal_truncated(ctx, wl["g"], sl_ptr, sl_idx, ypd, yid, yvd, alpha, 1e-12, args.trunc_iters, X=X)
    torch.cuda.synchronize()
    steps = 5
    t0 = time.perf_counter()
    for _ in range(steps):
        _, it, _, st = hd.temporal_truncated(ctx, wl["g"], sl_ptr, sl_idx, ypd, yid, yvd, alpha, 1e-12,
                                             args.trunc_iters, X=X)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / steps * 1e3
    # truncation error: the full solution restricted to each shortlist
    ref, *_ = hd.query_batch(ctx, wl["g"], wl["eig"], "pcg", yp, yi, yv, alpha, tol_ref, 2000)
    full = torch.gather(ref, 0, sl.T.long())
    err = (torch.linalg.norm(full - X, dim=0) / torch.linalg.norm(full, dim=0)).cpu().numpy()
    return {"shortlist": s, "B": B, "iters": int(np.max(it)), "ms_per_batch": round(ms, 3),
            "qps": round(B / ms * 1e3, 1), "truncation_rel_err_median": float(np.median(err)),
            "truncation_rel_err_max": float(np.max(err)),
            "timing": "host wall clock around the call (subsystem build + CG), inputs resident"}


def convergence_leg(ctx, wl, rows_in, alpha):
    """Sec. 4.4 on the benchmark graph: lambda_n by Lanczos on -W, then the
    Eq. 21-23 iteration bound for each measured (r, tol) leg.  lambda_{r+1} is
    taken as lambda_r when only r eigenvalues are known (a larger kappa, so
    the bound stays an upper bound)."""
    import paper_1807_08692_gb300 as hd
    t0 = time.perf_counter()
    lam_min, conv = hd.spectrum_min(ctx, wl["g"], tol=1e-4, max_restarts=30)
    t_min = time.perf_counter() - t0
    lam = wl["lam"]
    out = []
    for row in rows_in:
        r, mode, tol, measured = row[:4]
        if r == 0:
            lam_next = 1.0
        elif len(row) > 4 and row[4] is not None:
            lam_next = float(row[4])  # lambda_r of the leg's own eigenpairs (lambda_{r+1} <= it)
        else:
            lam_next = float(lam[min(r, len(lam) - 1)])
        kap, ia, ir = hd.cg_bound(mode if r > 0 else "paper", alpha, lam_next, min(lam_min, lam_next), tol)
        out.append({"r": r, "mode": mode, "tol": tol, "lambda_next": round(lam_next, 5), "kappa": round(kap, 3),
                    "bound_iters_anorm": ia, "bound_iters_resid": ir, "measured_iters": measured})
    return {"lambda_min": round(lam_min, 5), "lambda_min_converged": conv, "lambda_min_s": round(t_min, 2),
            "rows": out}


# ------------------------------------------------------------------ serving (continuous batching)
def serve_leg(ctx, wl, eig, args, rates, alpha):
    """Open-loop Poisson arrivals into the continuous-batching server; each
    request draws its tolerance from {1e-2, 1e-4, 1e-6} and K from {10, 100,
    1000}.  Latency = completion (ranking on the host) - scheduled arrival."""
    import torch
    import paper_1807_08692_gb300 as hd
    import synth
    c = wl["cfg"]
    nreq = args.serve_requests
    Qv = synth.queries(c.seed + 5000, nreq, wl["d"], c.ncl, c.kappa_lo, c.kappa_hi, c.sizes, c.zipf_s)
    yp, yi, yv = hd.observe(ctx, wl["Xt"], torch.from_numpy(Qv).to(wl["Xt"].dtype).cuda(), c.k_y, c.gamma)
    tols, Ks = synth.request_draws(c.seed, nreq)
    out = []
    for rate in rates:
        srv = hd.Server(ctx, wl["g"], eig, "pcg" if eig is not None else "paper", alpha, max_slots=args.serve_slots,
                        max_iter=2000, Kmax=1000)
        arr = synth.poisson_arrivals(c.seed + int(rate), rate, nreq)
        lat, tick = [], {}
        # warm-up: a few requests through the server before the clock starts
        for j in range(min(8, nreq)):
            tick[srv.submit(yi[yp[j]:yp[j + 1]], yv[yp[j]:yp[j + 1]], 1e-4, 10)] = (10, None)
        while srv.step(2):
            pass
        for t in srv.completed():
            srv.poll(t, 10)
        tick.clear()
        t0 = time.monotonic()
        nxt = 0
        done = 0
        last_done = t0
        iters = []
        while done < nreq:
            now = time.monotonic() - t0
            while nxt < nreq and arr[nxt] <= now:
                t = srv.submit(yi[yp[nxt]:yp[nxt + 1]], yv[yp[nxt]:yp[nxt + 1]], float(tols[nxt]), int(Ks[nxt]))
                tick[t] = (int(Ks[nxt]), t0 + arr[nxt])
                nxt += 1
            busy = srv.step(1)
            for t in srv.completed():
                res = srv.poll(t, tick[t][0])
                lat.append(res[2]["done_s"] - tick[t][1])
                iters.append(res[2]["iters"])
                last_done = max(last_done, res[2]["done_s"])
                del tick[t]
                done += 1
            if not busy and nxt < nreq:
                time.sleep(max(0.0, min(arr[nxt] - (time.monotonic() - t0), 0.002)))
        span = last_done - (t0 + arr[0])
        lat_ms = 1e3 * np.asarray(lat)
        out.append({"rate": rate, "requests": nreq, "qps": round(nreq / span, 1),
                    "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                    "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
                    "mean_iters": round(float(np.mean(iters)), 2), "slots": srv.slots})
        srv.close()
    return {"rates": out, "batch_same_mix": batch_same_mix(ctx, wl, eig, args, yp, yi, yv, tols, Ks, alpha)}


def serve_saturated(ctx, wl, eig, args, alpha, nreq):
    """Where a saturated server's time goes: nreq requests of the serving mix
    queued at once, one CG iteration per step until all are done; wall time in
    step() and in completed() + poll(), and the per-family kernel time per step
    (a second pass with CUDA-event profiling on)."""
    import torch
    import paper_1807_08692_gb300 as hd
    import synth
    c = wl["cfg"]
    Qv = synth.queries(c.seed + 5000, nreq, wl["d"], c.ncl, c.kappa_lo, c.kappa_hi, c.sizes, c.zipf_s)
    yp, yi, yv = hd.observe(ctx, wl["Xt"], torch.from_numpy(Qv).to(wl["Xt"].dtype).cuda(), c.k_y, c.gamma)
    tols, Ks = synth.request_draws(c.seed, nreq)
    out = {"requests": nreq, "slots": args.serve_slots}
    for prof in (False, True):
        srv = hd.Server(ctx, wl["g"], eig, "pcg" if eig is not None else "paper", alpha, max_slots=args.serve_slots,
                        max_iter=2000, Kmax=1000)
        for j in range(min(16, nreq)):
            srv.submit(yi[yp[j]:yp[j + 1]], yv[yp[j]:yp[j + 1]], 1e-4, 10)
        while srv.step(1):
            pass
        for t in srv.completed():
            srv.poll(t, 10)
        tick = {srv.submit(yi[yp[j]:yp[j + 1]], yv[yp[j]:yp[j + 1]], float(tols[j]), int(Ks[j])): int(Ks[j])
                for j in range(nreq)}
        if prof:
            ctx.profile(True)
            for f in FAMILIES:
                ctx.profile_read(f)
        t_step = t_poll = 0.0
        steps = done = 0
        t0 = time.perf_counter()
        while done < nreq:
            a = time.perf_counter()
            srv.step(1)
            b = time.perf_counter()
            fin = srv.completed()
            for t in fin:
                srv.poll(t, tick[t])
            done += len(fin)
            t_poll += time.perf_counter() - b
            t_step += b - a
            steps += 1
        wall = time.perf_counter() - t0
        if not prof:
            out.update({"qps": round(nreq / wall, 1), "steps": steps, "ms_per_step": round(wall / steps * 1e3, 3),
                        "step_ms": round(t_step / steps * 1e3, 3), "completed_poll_ms": round(t_poll / steps * 1e3, 3),
                        "retirements_per_step": round(nreq / steps, 1)})
        else:
            out["families_ms_per_step"] = {f: round(ms / steps, 3) for f in FAMILIES
                                           for (cnt, ms) in [ctx.profile_read(f)] if cnt}
            ctx.profile(False)
        srv.close()
    return out


def batch_same_mix(ctx, wl, eig, args, yp, yi, yv, tols, Ks, alpha):
    """The batch solver on the serving leg's request mix: batches of
    serve_slots requests with their own tolerances and K (hd_query_batch +
    hd_rank), requests back to back; the throughput continuous batching is
    compared with."""
    import torch
    import paper_1807_08692_gb300 as hd
    B = args.serve_slots
    nb = max(1, min(len(yp) - 1, 4 * B) // B)
    X = torch.empty((wl["n"], (B + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    Kmax = int(max(Ks))
    idx = torch.empty((B, Kmax), dtype=torch.int32, device="cuda")
    sc = torch.empty((B, Kmax), dtype=torch.float32, device="cuda")

    def run(q0):
        p = (yp[q0:q0 + B + 1] - yp[q0]).astype(np.int32)
        hd.query_batch(ctx, wl["g"], eig, "pcg" if eig is not None else "paper", p, yi[yp[q0]:yp[q0 + B]],
                       yv[yp[q0]:yp[q0 + B]], alpha, tols[q0:q0 + B].astype(np.float32), 2000, X=X, ldx=X.shape[1])
        hd.rank(ctx, X[:, :B], Ks[q0:q0 + B].astype(np.int32), Kmax, idx=idx, score=sc)

    run(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(nb):
        run(b * B)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"batch": B, "batches": nb, "qps": round(nb * B / dt, 1)}


# ------------------------------------------------------------------ replicas
def max_over_ranks(value: float) -> float:
    """The largest value over the ranks (the slowest replica's time); the
    value itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, batch: int, steps: int, slowest_s: float) -> float:
    """Whole-job queries/s of `world` replicas that each ran `steps` batches of
    `batch` queries, timed by the slowest replica."""
    return world * batch * steps / slowest_s


def query_seed(cfg_seed: int, rank: int) -> int:
    """Each replica draws its own query stream (the stream shards by query)."""
    return cfg_seed + 1000 * rank


# ------------------------------------------------------------------ main
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.export_inputs:
        return export_inputs(args)
    if args.impl == "reference":
        return reference_arm(args, world, rank, local)
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1807_08692_gb300 as hd
    ctx = hd.Context(local)
    alpha = 0.99
    wl = build_workload(args, ctx, rank)
    B = args.batch
    eig = wl["eig"]
    # ---- calibration: loosest ladder tolerance meeting 1e-4 against the fp64 oracle for each method
    # (with replicas, rank 0 calibrates on its queries and the others take its tolerances)
    refs = None
    tol_h, err_h, it_h = 1e-5, None, None
    tol_0, err_0, it_0 = 1e-5, None, None
    if not args.quick and rank == 0:
        refs = oracle_references(wl, args, alpha)
        tol_h, err_h, it_h = calibrate(ctx, wl, eig, args.mode, alpha)
        tol_0, err_0, it_0 = calibrate(ctx, wl, None, "paper", alpha)
    if world > 1 and not args.quick:
        t = torch.tensor([tol_h, tol_0], dtype=torch.float64, device="cuda")
        torch.distributed.broadcast(t, 0)
        tol_h, tol_0 = float(t[0]), float(t[1])
    # ---- timed hybrid leg (the headline) with clocks
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    t_wall0 = time.perf_counter()
    hyb = time_leg(ctx, wl, eig, args.mode, tol_h, alpha, args.steps, args.warmup, B, args.topk, False)
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_s = max_over_ranks(hyb["total_ms"] / 1e3)
    qps = replica_throughput(world, B, args.steps, total_s)
    acc_h = accuracy(wl, hyb["X"], hyb["idx"], hyb["sc"], args.topk) if refs else None
    # per-kernel event timing for the roofline in a separate pass: profiling
    # brackets every launch with events, so it runs without the CUDA graphs
    prof_steps = min(args.steps, 10)
    hprof = time_leg(ctx, wl, eig, args.mode, tol_h, alpha, prof_steps, 1, B, args.topk, True)
    # ---- r = 0 pure CG leg
    cg = None
    if not args.quick:
        cgl = time_leg(ctx, wl, None, "paper", tol_0, alpha, args.steps, args.warmup, B, args.topk, False)
        cg = {"value": replica_throughput(world, B, args.steps, max_over_ranks(cgl["total_ms"] / 1e3)),
              "ms_per_step": cgl["total_ms"] / args.steps,
              "tol": tol_0, "calib_rel_err": err_0, "iters_max": int(cgl["iters"].max()),
              "accuracy": accuracy(wl, cgl["X"], cgl["idx"], cgl["sc"], args.topk) if refs else None,
              "p50_ms": float(np.percentile(cgl["ms"], 50)), "p99_ms": float(np.percentile(cgl["ms"], 99))}
    # ---- e2e through host buffers
    e2e = None
    if not args.no_e2e:
        es, h2d, d2h = e2e_leg(ctx, wl, eig, args.mode, tol_h, alpha, args.steps, B, args.topk)
        e2e = {"value": replica_throughput(world, B, args.steps, max_over_ranks(es)), "unit": "queries/s",
               "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
    # ---- sweep over storage, rank and batch
    sweep = sweep_leg(ctx, wl, args, alpha) if (args.sweep and not args.quick and refs) else None
    # ---- Temporal† baseline (truncated temporal filtering)
    trunc = None
    if not args.quick and args.shortlist > 0 and not wl["pool"]:
        trunc = truncated_leg(ctx, wl, args, alpha, 1e-7)
    # ---- the 2,000-node clustered workload, where the hybrid's rank matters
    small = small_leg(ctx, args, alpha) if (args.small_leg and not args.quick and rank == 0) else None
    # ---- convergence analysis (Eq. 21-23) against the measured iteration counts
    conv = None
    if not args.quick and wl["lam"] is not None:
        rows_in = [(args.r, args.mode, tol_h, int(hyb["iters"].max()))]
        if cg is not None:
            rows_in.append((0, "paper", tol_0, cg["iters_max"]))
        for sw in sweep or []:
            if sw["mode"] == args.mode and sw.get("storage") == args.storage and sw["B"] == B \
                    and "sparsity" not in sw and sw["r"] != args.r:
                rows_in.append((sw["r"], sw["mode"], sw["tol"], sw["iters_max"], sw.get("lambda_r")))
        conv = convergence_leg(ctx, wl, rows_in, alpha)
    # ---- serving: continuous batching under Poisson load
    serving = None
    rates = [float(x) for x in args.serve_rates.split(",") if x.strip()] if not wl["pool"] else []
    if rates:
        serving = serve_leg(ctx, wl, eig, args, rates, alpha)
    if args.serve_saturated > 0 and not wl["pool"]:
        serving = dict(serving or {}, saturated=serve_saturated(ctx, wl, eig, args, alpha, args.serve_saturated))
    # ---- roofline of the dominant kernel
    ab = algorithmic_bytes(wl, B, eig)
    fam = hprof["fam"]
    dom = max((f for f in fam if f in ab), key=lambda f: fam[f][1])
    cnt, ms, busy = fam[dom]
    avg_s = ms / 1e3 / max(busy, 1)  # per launch that did work (idle launches return at once)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = ab[dom] / avg_s / 1e9
    nnz = wl["g"].nnz
    gather = nnz * ((B + 3) // 4 * 4) * 4 + 8 * nnz + 4 * (wl["n"] + 1) + 2 * wl["n"] * ((B + 3) // 4 * 4) * 4
    spmm_ms = fam["spmm"][1] / max(fam["spmm"][2], 1)
    traffic = spmm_traffic(wl, B) if dom == "spmm" else None
    # the whole step against a fully fused design's bytes: per CG iteration W
    # once (8 nnz), U twice (U^T P and U H) and nine n x B vector passes; once per
    # step the spectral term (U, one vector) and the top-K (one vector)
    s_u = {0: 4, 1: 2, 2: 1}[eig.storage] if eig is not None else 0
    r_u = eig.r if eig is not None else 0
    n_, vb = wl["n"], wl["n"] * B * 4
    # plus once per step the true residual b - A x (W once, X, T written and read back)
    path_bytes = int(hyb["iters"].max()) * (8 * nnz + 2 * n_ * r_u * s_u + 9 * vb) + n_ * r_u * s_u + 2 * vb \
        + 8 * nnz + 3 * vb
    path_gbs = path_bytes / (hyb["total_ms"] / args.steps / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                # the same launch measured by its DRAM bytes (random gathers re-read rows; see profiles/)
                "dram_gbs": round(traffic / avg_s / 1e9, 1) if traffic else None,
                "dram_frac": round(traffic / avg_s / 1e9 / peak, 4) if traffic else None,
                "spmm_gather_bytes_per_launch": int(gather),
                "spmm_gather_gbs": round(gather / (spmm_ms / 1e3) / 1e9, 1) if spmm_ms > 0 else None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_launch": int(ab[dom]), "avg_launch_ms": round(avg_s * 1e3, 4),
                "share_of_step": round(ms / hprof["total_ms"], 4),
                "path_algorithmic_bytes_per_step": int(path_bytes), "path_gbs": round(path_gbs, 1),
                "path_frac": round(path_gbs / peak, 4),
                "profiled_steps": prof_steps,
                "profiled_ms_per_step": round(hprof["total_ms"] / prof_steps, 4),
                "profiled_launches_per_step": round(hprof["launches"] / prof_steps, 1),
                "families_ms": {f: round(v[1], 3) for f, v in fam.items()},
                "families_launches": {f: v[0] for f, v in fam.items()},
                "families_busy_launches": {f: v[2] for f, v in fam.items()},
                # each iteration launches the fp32 and the fp16-gather SpMM and
                # one of them returns at once (the choice is made on the
                # device): busy launches of both per CG iteration run
                "spmm_busy_per_iteration": round((fam["spmm"][2] + fam["spmm_h"][2])
                                                 / max(1, int(hprof["iters"].max()) * prof_steps), 3)}
    # ---- CPU baseline: the oracle on host cores, bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        Wo, lamo, Uo = oracle_inputs(wl)
        dt, iters, dt0, it0 = cpu_oracle(Wo, lamo, Uo, timed_columns(wl, args.cpu_sample), alpha, min(tol_h, 1e-6),
                                         with_cg=True)
        cpu = {"value": args.cpu_sample / dt, "unit": "queries/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{args.cpu_sample} query columns of the timed batch, oracle fp64 hybrid PCG "
                         f"(scipy CSR SpMV, numpy BLAS) on the same graph and r={args.r} eigenpairs, "
                         f"{dt:.1f} s, iterations {list(map(int, iters))}",
               "cg_r0": {"value": args.cpu_sample / dt0, "unit": "queries/s",
                         "sample": f"same columns, oracle fp64 CG (r = 0), {dt0:.1f} s, "
                                   f"iterations {list(map(int, it0))}"}}
    line = {
        "metric": METRIC, "value": round(qps, 2), "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(hyb["total_ms"] / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (U bf16)" if args.storage == "bf16" else "f32",
        "data": "synthetic vMF mixture (seeded), built on the device",
        "config": {"workload": f"{wl['cfg'].name}: n={wl['n']}, d={wl['d']}, k={wl['cfg'].k}, nnz={wl['g'].nnz}, "
                               f"B={B} queries/step, k_y={wl['cfg'].k_y}, top-{args.topk}"
                               + (f", regional: {wl['pool']} regions per image, pooled ranking of "
                                  f"{wl['n'] // wl['pool']} images" if wl["pool"] else ""),
                   "mode": args.mode, "r": args.r, "storage": args.storage, "alpha": alpha, "tol": tol_h,
                   "spmm_tuning": dict(zip(("slab", "segments"), wl["g"].tuning(B) or (None, None))),
                   "calib_rel_err": err_h, "calib_reference": "fp64 oracle CG to relres 1e-12" if refs else None,
                   "oracle_references": refs, "accuracy": acc_h, "iters_max": int(hyb["iters"].max()),
                   "l2": "inputs larger than L2 (graph + U + vectors per step > 129 MB)",
                   "parallelism": f"replicas x{world}",
                   "lambda_top": [round(float(v), 5) for v in (wl["lam"][:3] if wl["lam"] is not None else [])],
                   "lambda_r": round(float(wl["lam"][-1]), 5) if wl["lam"] is not None else None,
                   "lanczos_max_resid": float(np.max(wl["res"])) if wl["res"] is not None else None,
                   "lanczos_restarts": wl["restarts"],
                   "setup_s": {"gen": round(wl["t_gen"], 1), "graph": round(wl["t_graph"], 1),
                               "eig": round(wl["t_eig"], 1)}},
        "p50_ms": round(float(np.percentile(hyb["ms"], 50)), 4), "p99_ms": round(float(np.percentile(hyb["ms"], 99)), 4),
        "cg_r0": cg, "sweep": sweep, "small_workload": small, "temporal_truncated": trunc, "convergence": conv, "serving": serving, "e2e": e2e, "gpu_launches": int(hyb["launches"]), "roofline": roofline, "cpu_baseline": cpu,
        "clocks": clocks, "wall_s_timed": round(t_wall, 3),
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def export_inputs(args):
    """Reference arm, first process: build the workload with the library and
    write what the oracle needs to args.export_inputs: the graph and the fp32
    eigenpairs as library checkpoints, the timed batch's observations."""
    import torch
    import paper_1807_08692_gb300 as hd
    out = args.export_inputs
    os.makedirs(out, exist_ok=True)
    torch.cuda.set_device(0)
    ctx = hd.Context(0)
    wl = build_workload(args, ctx, 0)
    wl["g"].save(os.path.join(out, "graph.hdg"))
    if wl["U32"] is not None:
        e32 = hd.eig_from_host(ctx, wl["g"], wl["lam"], wl["U32"], "f32")
        e32.save(os.path.join(out, "eig.hde"))
        e32.close()
    yp, yi, yv = wl["tim"]
    np.savez(os.path.join(out, "y.npz"), yp=yp, yi=yi, yv=yv, n=wl["n"], d=wl["d"], k=wl["cfg"].k,
             name=wl["cfg"].name)
    ctx.close()


def read_graph_checkpoint(path):
    """W from a graph checkpoint: "HDGRAPH1", n, nnz (int64), one reserved
    int64, then row_ptr int32[n+1], col int32[nnz], val float32[nnz] (= W),
    dinv float32[n]."""
    import scipy.sparse as sp
    with open(path, "rb") as f:
        if f.read(8) != b"HDGRAPH1":
            raise ValueError(f"{path}: not a graph checkpoint")
        n, nnz, _ = np.frombuffer(f.read(24), np.int64)
        rp = np.frombuffer(f.read(4 * (n + 1)), np.int32)
        col = np.frombuffer(f.read(4 * nnz), np.int32)
        val = np.frombuffer(f.read(4 * nnz), np.float32)
    return sp.csr_matrix((val.astype(np.float64), col, rp), shape=(n, n))


def read_eig_checkpoint(path):
    """(lambda, U) from an fp32 eigenpair checkpoint: "HDEIG001", n (int64),
    r, storage, ldu, pad (int32), lambda float64[r], U float32[n][ldu]."""
    with open(path, "rb") as f:
        if f.read(8) != b"HDEIG001":
            raise ValueError(f"{path}: not an eigenpair checkpoint")
        n = int(np.frombuffer(f.read(8), np.int64)[0])
        r, storage, ldu, _ = np.frombuffer(f.read(16), np.int32)
        if storage != 0:
            raise ValueError(f"{path}: fp32 eigenpairs expected")
        lam = np.frombuffer(f.read(8 * r), np.float64).copy()
        U = np.frombuffer(f.read(4 * n * ldu), np.float32).reshape(n, ldu)[:, :r].astype(np.float64)
    return lam, U


def reference_arm(args, world, rank, local):
    """The oracle (fp64, host cores) on this arm's workload and metric.  The
    workload is built by a separate, earlier process (export_inputs); this
    process reads its files with NumPy and never loads the library."""
    if rank != 0:
        return
    import shutil
    import tempfile
    from oracle import observe
    tmp = tempfile.mkdtemp(prefix="hd_ref_")
    try:
        # same workload and query split as this arm's own run (--sweep sets the batch offsets)
        cmd = [sys.executable, os.path.abspath(__file__), "--export-inputs", tmp, "--workload", args.workload,
               "--batch", str(args.batch), "--r", str(args.r), "--restarts", str(args.restarts),
               "--sweep", str(args.sweep), "--sweep-batches", args.sweep_batches]
        if args.n:
            cmd += ["--n", str(args.n)]
        if args.d:
            cmd += ["--d", str(args.d)]
        env = {k: v for k, v in os.environ.items() if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE")}
        subprocess.run(cmd, check=True, env=env)
        W = read_graph_checkpoint(os.path.join(tmp, "graph.hdg"))
        eig_path = os.path.join(tmp, "eig.hde")
        lam, U = read_eig_checkpoint(eig_path) if os.path.exists(eig_path) else (np.zeros(0), np.zeros((W.shape[0], 0)))
        z = np.load(os.path.join(tmp, "y.npz"))
        yp, yi, yv, n = z["yp"], z["yi"], z["yv"], int(z["n"])
        workload = f"{z['name']}: n={n}, d={int(z['d'])}, k={int(z['k'])}, nnz={W.nnz}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    alpha, tol = 0.99, 1e-6

    def cols(c0, m):
        return observe.dense(n, (yp[c0:c0 + m + 1] - yp[c0]).astype(np.int64), yi[yp[c0]:yp[c0 + m]],
                             yv[yp[c0]:yp[c0 + m]].astype(np.float64))

    for w in range(args.warmup):
        cpu_oracle(W, lam, U, cols(w % (len(yp) - 1), 1), alpha, tol)
    times, its = [], []
    # one oracle column takes about a second: keep the whole run to a few minutes
    per_step = args.cpu_sample if args.steps <= 40 else 1
    nb = len(yp) - 1
    for s in range(args.steps):
        c0 = (s * per_step) % max(1, nb - per_step + 1)
        dt, it = cpu_oracle(W, lam, U, cols(c0, per_step), alpha, tol)
        times.append(dt)
        its.extend(it)
    value = args.steps * per_step / float(np.sum(times))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": round(1e3 * float(np.mean(times)), 2),
            "config": {"workload": workload, "mode": "pcg", "r": int(lam.size)},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": round(value, 4),
                             "unit": "queries/s",
                             "sample": f"{per_step} query column(s) per step of the timed batch, fp64 hybrid PCG "
                                       f"(Form S) to relres {tol}, iterations {its[:8]}; inputs read from "
                                       f"checkpoint files written by a separate process"},
            "e2e": {"value": round(value, 4), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
