"""Seeded IVF-PQ index construction (k-means coarse quantiser + PQ on residuals).

The index of Section 2.1 (Fig. 1): the corpus is split into ``nlist`` clusters,
each vector's residual to its centroid is cut into ``M`` sub-vectors, and each
sub-vector is replaced by the index of its nearest entry in a per-sub-space
codebook shared by all clusters. The arrays produced here are inputs to both
the CUDA library and the CPU oracle; parity between them does not depend on
k-means quality.

Initialisation: the first ``k`` distinct rows of a seeded permutation of the
training sample. An empty cluster is re-seeded with the sample point farthest
from its current centroid. Ten Lloyd iterations by default.
"""
from __future__ import annotations

import numpy as np
import torch


def _device(device):
    if device is not None:
        return torch.device(device)
    return torch.device("cuda" if torch.cuda.is_available() else "cpu")


def _nearest(X: torch.Tensor, C: torch.Tensor, chunk: int = 1 << 16):
    """Index of and squared distance to the nearest row of C, for each row of X."""
    cn = (C * C).sum(1)
    idx = torch.empty(X.shape[0], dtype=torch.int64, device=X.device)
    dist = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    for s in range(0, X.shape[0], chunk):
        x = X[s:s + chunk]
        d = (x * x).sum(1, keepdim=True) - 2.0 * (x @ C.T) + cn[None, :]
        v, i = d.min(1)
        idx[s:s + chunk] = i
        dist[s:s + chunk] = v.clamp_min(0)
    return idx, dist


def _distinct_prefix(X: np.ndarray, k: int) -> np.ndarray:
    """Positions of the first k distinct rows of X (fewer if X has fewer)."""
    seen, keep = set(), []
    for i in range(X.shape[0]):
        key = X[i].tobytes()
        if key not in seen:
            seen.add(key)
            keep.append(i)
            if len(keep) == k:
                break
    return np.asarray(keep, dtype=np.int64)


def kmeans(X: np.ndarray, k: int, iters: int = 10, seed: int = 0,
           max_per_centroid: int = 256, device=None) -> np.ndarray:
    """Lloyd k-means on a seeded sample of at most ``k * max_per_centroid`` rows."""
    dev = _device(device)
    r = np.random.Generator(np.random.PCG64(seed))
    perm = r.permutation(X.shape[0])
    perm = perm[: min(X.shape[0], k * max_per_centroid)]
    S = np.ascontiguousarray(X[perm], dtype=np.float32)
    first = _distinct_prefix(S, k)
    C0 = S[first]
    if C0.shape[0] < k:  # fewer distinct points than clusters: repeat them
        C0 = C0[np.arange(k) % max(1, C0.shape[0])]
    Xs = torch.from_numpy(S).to(dev)
    C = torch.from_numpy(np.ascontiguousarray(C0)).to(dev)
    for _ in range(iters):
        a, dist = _nearest(Xs, C)
        cnt = torch.bincount(a, minlength=k).to(torch.float32)
        sums = torch.zeros_like(C).index_add_(0, a, Xs)
        newC = sums / cnt.clamp_min(1)[:, None]
        empty = torch.nonzero(cnt == 0).flatten()
        if empty.numel():
            far = torch.argsort(dist, descending=True)[: empty.numel()]
            newC[empty] = Xs[far]
        C = newC
    return C.cpu().numpy().astype(np.float32)


def train_ivfpq(base: np.ndarray, nlist: int, M: int, ksub: int = 256, iters: int = 10,
                seed: int = 0, max_per_centroid: int = 256, device=None) -> dict:
    """Train centroids and PQ codebooks on ``base`` and encode it.

    Returns float32 ``centroids [nlist, D]``, float32 ``codebooks [M, ksub, D/M]``,
    uint8 ``codes [N, M]`` and int32 ``list_of [N]``.
    """
    dev = _device(device)
    n, dim = base.shape
    assert dim % M == 0, "D must be a multiple of M"
    dsub = dim // M
    cent = kmeans(base, nlist, iters, seed, max_per_centroid, dev)
    X = torch.from_numpy(np.ascontiguousarray(base, dtype=np.float32))
    C = torch.from_numpy(cent).to(dev)
    list_of = np.empty(n, dtype=np.int32)
    codes = np.empty((n, M), dtype=np.uint8)
    # codebooks from a residual sample
    r = np.random.Generator(np.random.PCG64(seed + 1))
    samp = np.sort(r.permutation(n)[: min(n, ksub * 256)])
    xs = X[samp].to(dev)
    a, _ = _nearest(xs, C)
    res_s = (xs - C[a]).cpu().numpy()
    books = np.empty((M, ksub, dsub), dtype=np.float32)
    for m in range(M):
        books[m] = kmeans(res_s[:, m * dsub:(m + 1) * dsub], ksub, iters, seed + 17 * (m + 1),
                          max_per_centroid, dev)
    B = torch.from_numpy(books).to(dev)
    chunk = 1 << 17
    for s in range(0, n, chunk):
        x = X[s:s + chunk].to(dev)
        a, _ = _nearest(x, C)
        list_of[s:s + chunk] = a.cpu().numpy().astype(np.int32)
        res = x - C[a]
        for m in range(M):
            i, _ = _nearest(res[:, m * dsub:(m + 1) * dsub].contiguous(), B[m])
            codes[s:s + chunk, m] = i.cpu().numpy().astype(np.uint8)
    return dict(centroids=cent, codebooks=books, codes=codes, list_of=list_of)
