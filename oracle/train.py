"""CPU oracle of IVF-PQ index training — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.

The index of Section 2.1 (Fig. 1): a coarse quantiser of nlist centroids
found by k-means, and a product quantiser whose M codebooks of 256 entries
are found by k-means on the residuals x - c_list(x) cut into M sub-vectors;
every vector is stored as its list and its M code indices. The paper trains
this index offline and states neither the sampling, the initialisation nor
the rounding of the means; the readings below fix them so that training is
a deterministic function of the data and the seed.

* Sample: row i of an n-row matrix is drawn when key(i) < floor(target *
  2^64 / n), key(i) the SplitMix64 output (Steele, Lea and Flood, 2014) of
  the state seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64); drawn rows keep
  their row order. (Every row when target >= n.)
* Initial centroids: centroid j is sample row floor(j * S / k), S rows drawn.
* Lloyd iteration: every sample row goes to its nearest centroid by the FP32
  distance rule of CL (ties to the lower centroid index); a centroid with
  members becomes their mean coordinate by coordinate, computed as the
  exact sum of the members' FP32 values rounded once to FP32, then one IEEE
  FP32 division by the member count; the e-th empty centroid (ascending
  index) takes the e-th farthest sample row from its own centroid (FP32
  rule distance of this iteration's assignment; ties to the lower row).
* PQ: a second sample (seed + 1) whose residuals to their nearest centroid
  (fl32(x - c) per coordinate) train one k-means of 256 centroids per
  sub-space, on that sub-space's coordinates.
* Encoding: list = nearest centroid, code_m = nearest codebook entry of the
  residual's sub-vector m (FP32 rule, ties to the lower index).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import ivfpq

F32 = np.float32
F64 = np.float64
M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(z: int) -> int:
    """The SplitMix64 output function of the state z."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def sample_rows(n: int, target: int, seed: int) -> np.ndarray:
    """Rows drawn by the keyed Bernoulli rule (module docstring), ascending."""
    if target >= n:
        return np.arange(n, dtype=np.int64)
    thr = (target << 64) // n
    return np.array([i for i in range(n) if splitmix64(seed + (i + 1) * GOLDEN) < thr], dtype=np.int64)


def _exact_mean(values: np.ndarray) -> np.float32:
    """fl32(fl32(exact sum) / count) of FP32 values (count >= 1)."""
    scaled = sum(int(F64(v) * F64(2.0) ** 149) for v in values)   # every FP32 value is k * 2^-149
    s32 = ivfpq.nearest_f32(Fraction(scaled, 1 << 149))
    return F32(s32 / F32(len(values)))


def assign(X: np.ndarray, C: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Nearest centroid of each row (FP32 rule, ties to the lower index) and its distance."""
    D = ivfpq.coarse_d2_fp32(X, C)
    a = np.argmin(D, axis=1)                      # first minimum: the lower index
    return a.astype(np.int64), D[np.arange(len(X)), a]


def kmeans(X: np.ndarray, k: int, iters: int) -> np.ndarray:
    """Lloyd k-means of the rows of X (FP32) by the rules of the module docstring."""
    X = np.asarray(X, F32)
    S = len(X)
    assert S >= k >= 1
    C = X[(np.arange(k) * S) // k].copy()
    for _ in range(iters):
        a, d = assign(X, C)
        newC = C.copy()
        empty = []
        for j in range(k):
            mem = np.flatnonzero(a == j)
            if len(mem) == 0:
                empty.append(j)
                continue
            for c in range(X.shape[1]):
                newC[j, c] = _exact_mean(X[mem, c])
        if empty:
            order = np.lexsort((np.arange(S), -d.astype(F64)))   # farthest first, ties to the lower row
            for e, j in enumerate(empty):
                newC[j] = X[order[e]]
        C = newC
    return C


def train(base: np.ndarray, nlist: int, M: int, iters: int = 10, pq_iters: int = 10, seed: int = 0,
          per_centroid: int = 256, pq_sample: int = 65536, ksub: int = 256) -> dict:
    """Centroids, codebooks [M, 256, dsub], codes [n, M] and lists [n] of the base."""
    base = np.asarray(base, F32)
    n, dim = base.shape
    assert dim % M == 0
    dsub = dim // M
    S = base[sample_rows(n, nlist * per_centroid, seed)]
    cent = kmeans(S, nlist, iters)
    R = base[sample_rows(n, pq_sample, seed + 1)]
    a, _ = assign(R, cent)
    res = (R - cent[a]).astype(F32)
    books = np.empty((M, ksub, dsub), dtype=F32)
    for m in range(M):
        books[m] = kmeans(res[:, m * dsub:(m + 1) * dsub], ksub, pq_iters)
    return dict(centroids=cent, codebooks=books, **encode(base, cent, books))


def encode(base: np.ndarray, cent: np.ndarray, books: np.ndarray) -> dict:
    """List of each row and the codes of its residual (FP32 rules)."""
    base = np.asarray(base, F32)
    M, _, dsub = books.shape
    lst, _ = assign(base, cent)
    res = (base - cent[lst]).astype(F32)
    codes = np.empty((len(base), M), dtype=np.uint8)
    for m in range(M):
        c, _ = assign(res[:, m * dsub:(m + 1) * dsub], books[m])
        codes[:, m] = c
    return dict(codes=codes, list_of=lst.astype(np.int32))
