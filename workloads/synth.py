"""Seeded synthetic stand-ins for the paper's datasets.

The paper evaluates on SIFT100M / DEEP100M (uint8), SIFT1M and GIST1M
(Section 5.1 and Table 3). None of those sets is available here, so each
workload below is a seeded synthetic distribution with the shape of one of
them (dimension, value range, cluster structure, list-length skew). All draws
use numpy's PCG64; the mixture parameters and the base vectors come from
``seed``, queries from ``seed + 100`` (training queries from ``seed + 200``).

Nothing here computes any part of the search; it only produces arrays.
"""
from __future__ import annotations

import numpy as np

# Five workloads. ``nprobe`` of the SIFT-shaped workload is a sweep; the
# GIST-shaped one draws nprobe and k per query.
CONFIGS = {
    "A": dict(name="gauss-mix-20k-d128", n=20_000, dim=128, nlist=64, M=16,
              nprobe=8, k=10, nq=100, seed=1),
    "B": dict(name="sift-shaped-1m-d128", n=1_000_000, dim=128, nlist=1024, M=32,
              nprobe=32, nprobe_sweep=(16, 32, 64), k=10, nq=10_000, seed=2),
    "C": dict(name="deep-shaped-10m-d96", n=10_000_000, dim=96, nlist=4096, M=48,
              nprobe=32, k=10, nq=10_000, seed=3),
    "D": dict(name="gist-shaped-uneven-1m-d960", n=1_000_000, dim=960, nlist=1024,
              M=120, nprobe=128, k=100, nq=4096, seed=4),
    "E": dict(name="embedding-5m-d768", n=5_000_000, dim=768, nlist=8192, M=96,
              nprobe=64, k=100, nq=20_000, ntrain=50_000, seed=5),
}
KSUB = 256


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


class _Mixture:
    """Mixture parameters drawn once from the workload seed."""

    def __init__(self, key: str, dim: int, seed: int, ncomp: int | None = None):
        self.key, self.dim = key, dim
        r = _rng(seed)
        self.r = r  # base vectors continue this stream after the parameters
        if key == "A":
            k = ncomp or 64
            self.means = r.uniform(-1.0, 1.0, size=(k, dim))
            self.sigma = r.uniform(0.05, 0.3, size=k)
            self.weights = np.full(k, 1.0 / k)
        elif key == "B":
            k = ncomp or 1024
            self.w = r.uniform(0.25, 2.0, size=(k, dim))
            self.weights = np.full(k, 1.0 / k)
        elif key == "C":
            k = ncomp or 4096
            self.mu = r.standard_normal((k, dim)) / np.sqrt(dim)
            self.sig = r.uniform(0.05, 0.2, size=k)
            g = r.standard_normal((k, dim, dim))
            q, rr = np.linalg.qr(g)
            # fix the sign so that the rotation is a deterministic function of g
            q = q * np.sign(np.diagonal(rr, axis1=1, axis2=2))[:, None, :]
            self.rot = q.astype(np.float64)
            self.decay = 1.0 / np.sqrt(np.arange(1, dim + 1))
            self.weights = np.full(k, 1.0 / k)
        elif key == "D":
            k = ncomp or 1024
            w = 1.0 / np.arange(1, k + 1)  # Zipf(s=1) cluster sizes
            self.weights = w / w.sum()
            self.lam = r.uniform(0.5, 4.0, size=(k, dim))
        elif key == "E":
            k = ncomp or 8192
            mu = r.standard_normal((k, dim))
            self.mu = mu / np.linalg.norm(mu, axis=1, keepdims=True)
            self.kappa = r.uniform(20.0, 200.0, size=k)
            self.weights = np.full(k, 1.0 / k)
        else:
            raise KeyError(key)
        self.ncomp = len(self.weights)

    def sample(self, n: int, r: np.random.Generator, chunk: int = 1 << 18) -> np.ndarray:
        out = np.empty((n, self.dim), dtype=np.float32)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            out[s:e] = self._sample(e - s, r)
        return out

    def _sample(self, n, r):
        lab = r.choice(self.ncomp, size=n, p=self.weights)
        d = self.dim
        if self.key == "A":
            return self.means[lab] + self.sigma[lab, None] * r.standard_normal((n, d))
        if self.key == "B":
            x = r.gamma(0.5, 40.0 * self.w[lab])
            return np.clip(np.rint(x), 0, 255)
        if self.key == "C":
            z = r.standard_normal((n, d)) * (self.sig[lab, None] * self.decay[None, :])
            x = np.empty((n, d))
            # x = mu_c + R_c z, one matrix product per component present
            order = np.argsort(lab, kind="stable")
            cut = np.flatnonzero(np.diff(lab[order])) + 1
            for idx in np.split(order, cut):
                if idx.size:
                    c = lab[idx[0]]
                    x[idx] = self.mu[c] + z[idx] @ self.rot[c].T
            return x / np.linalg.norm(x, axis=1, keepdims=True)
        if self.key == "D":
            return r.exponential(1.0 / self.lam[lab])
        if self.key == "E":
            return _vmf(self.mu[lab], self.kappa[lab], r)
        raise KeyError(self.key)


def _vmf(mu: np.ndarray, kappa: np.ndarray, r: np.random.Generator) -> np.ndarray:
    """von Mises-Fisher draws by Wood (1994): rejection-sample w = cos(angle to
    mu), then add a uniform direction orthogonal to mu."""
    n, d = mu.shape
    b = (d - 1) / (2.0 * kappa + np.sqrt(4.0 * kappa ** 2 + (d - 1) ** 2))
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + (d - 1) * np.log(1.0 - x0 ** 2)
    w = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        z = r.beta((d - 1) / 2.0, (d - 1) / 2.0, size=todo.size)
        u = r.uniform(size=todo.size)
        bb, xx, cc, kk = b[todo], x0[todo], c[todo], kappa[todo]
        ww = (1.0 - (1.0 + bb) * z) / (1.0 - (1.0 - bb) * z)
        ok = kk * ww + (d - 1) * np.log(1.0 - xx * ww) - cc >= np.log(u)
        w[todo[ok]] = ww[ok]
        todo = todo[~ok]
    v = r.standard_normal((n, d))
    v -= np.sum(v * mu, axis=1, keepdims=True) * mu
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return w[:, None] * mu + np.sqrt(np.maximum(0.0, 1.0 - w ** 2))[:, None] * v


def make_dataset(key: str, n: int | None = None, nq: int | None = None,
                 ntrain: int | None = None, ncomp: int | None = None) -> dict:
    """Base vectors, evaluation queries and (optionally) training queries.

    ``n``/``nq``/``ntrain`` override the workload's sizes for scaled-down
    test cases; ``ncomp`` overrides the number of mixture components.
    """
    cfg = CONFIGS[key]
    n = cfg["n"] if n is None else n
    nq = cfg["nq"] if nq is None else nq
    mix = _Mixture(key, cfg["dim"], cfg["seed"], ncomp)
    base = mix.sample(n, mix.r)
    queries = mix.sample(nq, _rng(cfg["seed"] + 100))
    out = dict(base=base, queries=queries)
    if ntrain:
        out["train"] = mix.sample(ntrain, _rng(cfg["seed"] + 200))
    return out


def make_queries(key: str, nq: int, stream: int = 100, ncomp: int | None = None) -> np.ndarray:
    """Extra queries from the workload's mixture (``stream`` picks the seed offset)."""
    cfg = CONFIGS[key]
    mix = _Mixture(key, cfg["dim"], cfg["seed"], ncomp)
    return mix.sample(nq, _rng(cfg["seed"] + stream))


def zipf_nprobe(nq: int, seed: int, lo: int = 1, hi: int = 128, s: float = 1.1) -> np.ndarray:
    """Per-query nprobe ~ Zipf(s) truncated to [lo, hi] (mean 19.69 for the defaults)."""
    v = np.arange(lo, hi + 1)
    p = v ** (-s)
    p /= p.sum()
    return _rng(seed + 300).choice(v, size=nq, p=p).astype(np.int32)


def mixed_k(nq: int, seed: int, choices=(1, 10, 100)) -> np.ndarray:
    """Per-query k drawn uniformly from ``choices``."""
    return _rng(seed + 400).choice(np.asarray(choices), size=nq).astype(np.int32)
