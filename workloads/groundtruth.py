"""Exact k-nearest-neighbour ground truth for recall measurement.

Squared L2 distance, ties broken by ascending row index. Candidates are found
with an FP32 GEMM-form distance, then the best ``k * 4 + 64`` per query are
re-ranked with a direct FP64 difference so the returned order is exact unless
an FP32 error exceeds the gap to the 4k+64-th candidate.
"""
from __future__ import annotations

import numpy as np
import torch


def exact_knn(base: np.ndarray, queries: np.ndarray, k: int, device=None,
              qchunk: int = 256) -> tuple[np.ndarray, np.ndarray]:
    """Returns (ids int64 [nq, k], squared distances float64 [nq, k])."""
    dev = torch.device(device) if device else torch.device(
        "cuda" if torch.cuda.is_available() else "cpu")
    X = torch.from_numpy(np.ascontiguousarray(base, dtype=np.float32)).to(dev)
    xn = (X * X).sum(1)
    n = X.shape[0]
    kc = min(n, 4 * k + 64)
    ids = np.empty((len(queries), k), dtype=np.int64)
    dst = np.empty((len(queries), k), dtype=np.float64)
    base64 = np.asarray(base, dtype=np.float64)
    for s in range(0, len(queries), qchunk):
        q = torch.from_numpy(np.ascontiguousarray(queries[s:s + qchunk], dtype=np.float32)).to(dev)
        d = xn[None, :] - 2.0 * (q @ X.T) + (q * q).sum(1, keepdim=True)
        cand = torch.topk(d, kc, dim=1, largest=False).indices.cpu().numpy()
        q64 = np.asarray(queries[s:s + qchunk], dtype=np.float64)
        for i in range(cand.shape[0]):
            c = cand[i]
            diff = base64[c] - q64[i][None, :]
            dd = np.einsum("ij,ij->i", diff, diff)
            order = np.lexsort((c, dd))[:k]
            ids[s + i] = c[order]
            dst[s + i] = dd[order]
    return ids, dst


def recall_at(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """Mean |found[:, :k] ∩ truth[:, :k]| / k over queries."""
    tot = 0
    for f, t in zip(found[:, :k], truth[:, :k]):
        tot += len(set(int(x) for x in f if x >= 0) & set(int(x) for x in t))
    return tot / (k * len(found))
