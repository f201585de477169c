"""von Mises-Fisher mixture sampling and other seeded draws.

Every generator here is deterministic given (seed, stream) and independent of
the number of worker threads: rows are produced in fixed blocks, each block
with its own PCG64 stream derived from SeedSequence([seed, stream, block]).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# Stream ids (one independent random stream per kind of draw).
STREAM_MEANS = 0
STREAM_DATABASE = 1
STREAM_QUERIES = 2
STREAM_ARRIVALS = 3
STREAM_LABELS = 4
STREAM_KAPPAS = 5

BLOCK_ROWS = 16384


def _rng(seed: int, stream: int, block: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream), int(block)])))


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def wood_radial(kappa: np.ndarray, d: int, rng: np.random.Generator) -> np.ndarray:
    """Cosine w = mu^T x of vMF(mu, kappa) samples on S^{d-1}, one per entry of kappa.

    Wood (1994), "Simulation of the von Mises Fisher distribution", rejection
    sampler with a Beta((d-1)/2, (d-1)/2) envelope.  `kappa` may vary per row.
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    m = d - 1.0
    # b = (-2k + sqrt(4k^2 + m^2)) / m, written without cancellation.
    b = m / (2.0 * kappa + np.sqrt(4.0 * kappa * kappa + m * m))
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + m * np.log1p(-x0 * x0)
    out = np.empty(kappa.shape, dtype=np.float64)
    todo = np.arange(kappa.size)
    while todo.size:
        z = rng.beta(m / 2.0, m / 2.0, size=todo.size)
        bb = b[todo]
        w = (1.0 - (1.0 + bb) * z) / (1.0 - (1.0 - bb) * z)
        u = rng.uniform(size=todo.size)
        ok = kappa[todo] * w + m * np.log1p(-x0[todo] * w) - c[todo] >= np.log(u)
        out[todo[ok]] = w[ok]
        todo = todo[~ok]
    return out


def sample_vmf_rows(mu: np.ndarray, kappa: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """One vMF sample per row: mean direction mu[i] (unit), concentration kappa[i].

    x = w mu + sqrt(1 - w^2) v with w from Wood's sampler and v uniform on the
    unit sphere orthogonal to mu.  Returns float32 rows.
    """
    rows, d = mu.shape
    w = wood_radial(kappa, d, rng)
    g = rng.standard_normal((rows, d), dtype=np.float32)
    proj = np.einsum("ij,ij->i", g, mu, dtype=np.float32)
    g -= proj[:, None] * mu
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    x = w[:, None].astype(np.float32) * mu + np.sqrt(1.0 - w * w)[:, None].astype(np.float32) * g
    return x.astype(np.float32, copy=False)


def mixture_means(seed: int, ncl: int, d: int) -> np.ndarray:
    """Cluster mean directions: normalised standard Gaussians (float32)."""
    g = _rng(seed, STREAM_MEANS).standard_normal((ncl, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def mixture_kappas(seed: int, ncl: int, kappa_lo: float, kappa_hi: float) -> np.ndarray:
    if kappa_lo == kappa_hi:
        return np.full(ncl, float(kappa_lo))
    return _rng(seed, STREAM_KAPPAS).uniform(kappa_lo, kappa_hi, size=ncl)


def mixture_labels(seed: int, n: int, ncl: int, sizes: str = "equal", zipf_s: float = 1.1,
                   stream: int = STREAM_LABELS) -> np.ndarray:
    """Cluster label per row.  'equal': uniform over clusters; 'zipf': p_i ~ i^-s."""
    rng = _rng(seed, stream)
    if sizes == "equal":
        return rng.integers(0, ncl, size=n).astype(np.int64)
    if sizes == "zipf":
        p = np.arange(1, ncl + 1, dtype=np.float64) ** (-zipf_s)
        p /= p.sum()
        return rng.choice(ncl, size=n, p=p).astype(np.int64)
    raise ValueError(f"unknown cluster-size law {sizes!r}")


def _blocked(seed: int, stream: int, n: int, d: int, mu_of_row, kappa_of_row) -> np.ndarray:
    out = np.empty((n, d), dtype=np.float32)
    nblk = (n + BLOCK_ROWS - 1) // BLOCK_ROWS

    def work(b):
        s, e = b * BLOCK_ROWS, min(n, (b + 1) * BLOCK_ROWS)
        rng = _rng(seed, stream, b)
        out[s:e] = sample_vmf_rows(mu_of_row(s, e), kappa_of_row(s, e), rng)

    if nblk == 1:
        work(0)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(nblk)))
    return out


def database(seed: int, n: int, d: int, ncl: int, kappa_lo: float, kappa_hi: float,
             sizes: str = "equal", zipf_s: float = 1.1) -> tuple[np.ndarray, np.ndarray]:
    """n unit-norm float32 descriptors from a vMF mixture; returns (X, labels)."""
    mu = mixture_means(seed, ncl, d)
    kap = mixture_kappas(seed, ncl, kappa_lo, kappa_hi)
    lab = mixture_labels(seed, n, ncl, sizes, zipf_s)
    X = _blocked(seed, STREAM_DATABASE, n, d, lambda s, e: mu[lab[s:e]], lambda s, e: kap[lab[s:e]])
    return X, lab


def queries(seed: int, nq: int, d: int, ncl: int, kappa_lo: float, kappa_hi: float,
            sizes: str = "equal", zipf_s: float = 1.1) -> np.ndarray:
    """nq fresh query descriptors from the same mixture as `database` (float32)."""
    mu = mixture_means(seed, ncl, d)
    kap = mixture_kappas(seed, ncl, kappa_lo, kappa_hi)
    lab = mixture_labels(seed, nq, ncl, sizes, zipf_s, stream=STREAM_QUERIES + 100)
    return _blocked(seed, STREAM_QUERIES, nq, d, lambda s, e: mu[lab[s:e]], lambda s, e: kap[lab[s:e]])


def regional_database(seed: int, n_img: int, regions: int, d: int, ncl: int, kappa_lo: float,
                      kappa_hi: float, p_stay: float = 0.8, stream: int = STREAM_DATABASE,
                      label_stream: int = STREAM_LABELS) -> tuple[np.ndarray, np.ndarray]:
    """Regional descriptors: n_img images x `regions` rows each, image-major.

    Each image draws a cluster; each of its regions keeps that cluster with
    probability p_stay, otherwise takes a uniformly drawn other cluster.
    Returns (X of shape (n_img*regions, d), image id per row).
    """
    mu = mixture_means(seed, ncl, d)
    kap = mixture_kappas(seed, ncl, kappa_lo, kappa_hi)
    rng = _rng(seed, label_stream)
    img_cl = rng.integers(0, ncl, size=n_img)
    lab = np.repeat(img_cl, regions)
    move = rng.uniform(size=lab.size) >= p_stay
    other = rng.integers(0, ncl - 1, size=lab.size)
    other = other + (other >= lab)  # uniform over clusters != own
    lab = np.where(move, other, lab).astype(np.int64)
    X = _blocked(seed, stream, lab.size, d, lambda s, e: mu[lab[s:e]], lambda s, e: kap[lab[s:e]])
    return X, np.repeat(np.arange(n_img, dtype=np.int64), regions)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 values rounded to the nearest bfloat16 (ties to even), as float32."""
    bits = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (bits >> 16) & 1
    rounded = (bits + np.uint32(0x7FFF) + lsb) & np.uint32(0xFFFF0000)
    return rounded.view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 bfloat16 encodings of float32 values already representable in bf16."""
    return (np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def poisson_arrivals(seed: int, rate: float, count: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    gaps = _rng(seed, STREAM_ARRIVALS).exponential(1.0 / rate, size=count)
    return np.cumsum(gaps)


def request_draws(seed: int, count: int, tols=(1e-2, 1e-4, 1e-6), ks=(10, 100, 1000)):
    """Per-request residual tolerance and K, each uniform over its set."""
    rng = _rng(seed, STREAM_ARRIVALS + 10)
    tol = np.asarray(tols, dtype=np.float64)[rng.integers(0, len(tols), size=count)]
    K = np.asarray(ks, dtype=np.int64)[rng.integers(0, len(ks), size=count)]
    return tol, K


def a_d_kappa(d: int, kappa: float) -> float:
    """Mean resultant length of vMF on S^{d-1}: I_{d/2}(k) / I_{d/2-1}(k).

    Evaluated with the backward recurrence of the Bessel-ratio continued
    fraction, R_v = k / (2v + k R_{v+1}), which does not underflow for large d.
    """
    nu = d / 2.0
    R = 0.0
    for m in range(2000, -1, -1):
        R = kappa / (2.0 * (nu + m) + kappa * R)
    return float(R)

