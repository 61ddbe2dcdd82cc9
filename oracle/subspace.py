"""CPU oracle of the paper's sub-space precision granularity — TEST
INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.

Section 3.2 divides the vector space in two ways at once: the dimensions
into slices, and, inside each slice, the vectors into clusters (sub-spaces).
Eq. 1 says a neighbour in sub-space C1 beats one in C2 when d > 3 r1 + r2, so
sub-spaces far from the query need less precision; Section 3.3 turns this
into features (d', r1, r2, n1, n2) per sub-space, d' measured from the
query; Section 4.2 applies the precision by keeping the most significant
bits of the (uint8) operands; Section 5.3 (Fig. 13) sweeps the number of
slices and of sub-spaces per slice in CL, and notes that LC behaves alike
with the codebook entries of each PQ sub-space as its vectors.

Readings (the paper states none of these):
* Partition: in CL, slice s (S slices of D/S consecutive dimensions) of the
  nlist centroids is clustered into K sub-spaces by oracle.train.kmeans
  (its deterministic Lloyd rules, `iters` iterations); in LC, the 256 entries
  of codebook m are clustered into K_lc groups the same way.
* Statistics per sub-space: its centre (the k-means centroid), its size n
  (members) and its covering radius r = max over members of the distance to
  the centre (FP64: squares summed over dimensions in ascending order, IEEE
  square root, rounded to FP32).
* Operands in uint8 fixed point: x8 = clamp(rint(fl32(fl32(x - lo) * inv)),
  0, 255) (round half to even) with inv = fl32(255 / fl32(hi - lo)); in CL,
  lo / hi are the smallest / largest centroid coordinate, and queries use the
  same map; in LC the map is the codebook's and applies to the residual
  r = fl32(q - c_l). Keeping b bits: x_b = (x8 >> (8 - b)) << (8 - b).
* Bits per (query, slice, sub-space): the FP32 distance rule gives
  d_k = fl32(sqrt(D_k)), D_k the squared distance from the query's slice to
  centre k; k1 = the nearest centre (ties to the lower index); Eq. 2 with the
  query distance measured beyond the nearest centre, g = fl32(fl32(fl32(d_k -
  d_k1) - fl32(3 r_k1)) - r_k) / r_k (FP32; g = -inf when r_k = 0); bits 2,
  4 or 6 when g >= th2, th4 or th6 (checked in that order), else 8. The
  nearest sub-space always gets g < 0 and so 8 bits.
* CL: D2_int[l] = sum over slices s and their dimensions j of
  (q_b,j - c_b,l,j)^2 with b the bits of (q, s, sub-space of c_l's slice s),
  an exact integer; the nprobe smallest (D2_int, l) are probed, then
  re-ordered by their FP32-rule coarse distance (ties by l), which the
  later stages use.
* LC + DC: per probed pair, T_int[m][c] = sum over the dsub dimensions of
  (r_b,j - y_b,c,j)^2, b the bits of (pair, m, group of entry c), with r the
  pair's residual; the vector's distance S = sum_m T_int[m][code_m] (exact
  integer), the top-k by (S, id), reported as fl32(fl32(S) * fl32(1 / inv^2)).
"""
from __future__ import annotations

import numpy as np

from . import ivfpq, train

F32 = np.float32
F64 = np.float64


def fixed_point(lo: float, hi: float) -> tuple[np.float32, np.float32]:
    """(lo, inv) of the uint8 map: inv = fl32(255 / fl32(hi - lo)) (1 if hi == lo)."""
    lo, hi = F32(lo), F32(hi)
    span = F32(hi - lo)
    return lo, (F32(F32(255.0) / span) if span > 0 else F32(1.0))


def to_u8(x: np.ndarray, lo, inv) -> np.ndarray:
    """clamp(rint(fl32(fl32(x - lo) * inv)), 0, 255)."""
    y = ((np.asarray(x, F32) - F32(lo)).astype(F32) * F32(inv)).astype(F32)
    return np.clip(np.rint(y), 0, 255).astype(np.int64)


def keep_bits(x8: np.ndarray, b) -> np.ndarray:
    """The b most significant bits of the uint8 values (b broadcastable)."""
    t = 8 - np.asarray(b, np.int64)
    return (np.asarray(x8, np.int64) >> t) << t


def partition(X: np.ndarray, K: int, iters: int) -> dict:
    """Sub-spaces of the rows of X: centres, assignment, size and radius."""
    X = np.asarray(X, F32)
    C = train.kmeans(X, K, iters)
    a, _ = train.assign(X, C)
    size = np.bincount(a, minlength=K).astype(np.int64)
    rad = np.zeros(K, F64)
    for k in range(K):
        mem = X[a == k].astype(F64)
        if len(mem):
            acc = np.zeros(len(mem), F64)          # FP64 sum over dimensions, ascending
            for j in range(X.shape[1]):
                e = mem[:, j] - F64(C[k, j])
                acc = acc + e * e
            rad[k] = np.sqrt(acc).max()
    return dict(centres=C, assign=a, size=size, radius=rad.astype(F32))


def build(index: ivfpq.Index, S: int, K: int, K_lc: int, iters: int) -> dict:
    """CL partitions (one per slice of the centroids) and LC partitions (one
    per codebook), with the two uint8 maps."""
    D = index.dim
    assert D % S == 0
    w = D // S
    cl = [partition(index.centroids[:, s * w:(s + 1) * w], K, iters) for s in range(S)]
    lc = [partition(index.books[m], K_lc, iters) for m in range(index.M)]
    cl_map = fixed_point(index.centroids.min(), index.centroids.max())
    lc_map = fixed_point(index.books.min(), index.books.max())
    return dict(S=S, w=w, K=K, K_lc=K_lc, cl=cl, lc=lc, cl_map=cl_map, lc_map=lc_map,
                c8=to_u8(index.centroids, *cl_map), y8=to_u8(index.books, *lc_map))


def sub_bits(xs: np.ndarray, part: dict, th) -> np.ndarray:
    """Bits of every sub-space of one partition for one query slice xs."""
    C = part["centres"]
    D = ivfpq.coarse_d2_fp32(np.asarray(xs, F32)[None, :], C)[0]
    d = np.sqrt(D).astype(F32)
    k1 = int(np.argmin(D))
    r = part["radius"]
    f = ((d - d[k1]).astype(F32) - (F32(3.0) * r[k1]).astype(F32)).astype(F32)
    f = (f - r).astype(F32)
    g = np.where(r > 0, (f / np.where(r > 0, r, F32(1))).astype(F32), F32(-np.inf))
    bits = np.full(len(C), 8, np.int64)
    for b, t in ((6, th[2]), (4, th[1]), (2, th[0])):   # later (narrower) checks win
        bits = np.where(g >= F32(t), b, bits)
    return bits


def cl_bits(ss: dict, q: np.ndarray, th) -> np.ndarray:
    """Bits [S, K] of every (slice, sub-space) for query q."""
    w = ss["w"]
    return np.stack([sub_bits(q[s * w:(s + 1) * w], ss["cl"][s], th) for s in range(ss["S"])])


def locate(index: ivfpq.Index, ss: dict, Q: np.ndarray, nprobe: int, th):
    """Sub-space CL: probes [nq, nprobe], their FP32-rule distances, and the
    fraction of partial distances (query, list, slice) computed below 8 bits."""
    Q = np.asarray(Q, F32)
    S, w = ss["S"], ss["w"]
    q8 = to_u8(Q, *ss["cl_map"])
    c8 = ss["c8"]
    probes = np.empty((len(Q), nprobe), np.int32)
    pd = np.empty((len(Q), nprobe), F32)
    low = 0
    for i in range(len(Q)):
        B = cl_bits(ss, Q[i], th)                                     # [S, K]
        tot = np.zeros(index.nlist, np.int64)
        for s in range(S):
            b = B[s][ss["cl"][s]["assign"]]                           # bits per list
            low += int(np.sum(b < 8))
            sl = slice(s * w, (s + 1) * w)
            diff = keep_bits(q8[i, sl][None, :], b[:, None]) - keep_bits(c8[:, sl], b[:, None])
            tot += (diff * diff).sum(1)
        sel = np.lexsort((np.arange(index.nlist), tot))[:nprobe]
        d32 = ivfpq.coarse_d2_fp32(Q[i:i + 1], index.centroids[sel])[0]
        order = np.lexsort((sel, d32))
        probes[i], pd[i] = sel[order], d32[order]
    return probes, pd, low / (len(Q) * index.nlist * S)


def search(index: ivfpq.Index, ss: dict, Q: np.ndarray, nprobe: int, k: int, th_cl, th_lc,
           cl: bool = True, lc: bool = True):
    """The search with sub-space CL (else the FP32 CL) and sub-space LC + DC
    (else the FP32 LUT). Returns ids, dists and the low-precision shares."""
    Q = np.asarray(Q, F32)
    if cl:
        probes, pd, cl_low = locate(index, ss, Q, nprobe, th_cl)
    else:
        probes, pd = ivfpq.locate(ivfpq.coarse_d2_fp32(Q, index.centroids), nprobe)
        cl_low = 0.0
    M, dsub = index.M, index.dsub
    lo, inv = ss["lc_map"]
    scale = F32(F32(1.0) / F32(inv * inv))
    y8 = ss["y8"]                                                      # [M, 256, dsub]
    out_i = np.full((len(Q), k), -1, np.int64)
    out_d = np.full((len(Q), k), np.inf, F32)
    low, entries = 0, 0
    for i in range(len(Q)):
        ds, idl = [], []
        for j in range(nprobe):
            l = int(probes[i, j])
            mem = index.members[l]
            if len(mem) == 0:
                continue
            cd = index.codes[mem].astype(np.int64)
            if lc:
                r = (Q[i] - index.centroids[l]).astype(F32)
                r8 = to_u8(r, lo, inv).reshape(M, dsub)
                T = np.zeros((M, 256), np.int64)
                for m in range(M):
                    bg = sub_bits(r[m * dsub:(m + 1) * dsub], ss["lc"][m], th_lc)   # bits per group
                    b = bg[ss["lc"][m]["assign"]]                                   # bits per entry
                    low += int(np.sum(b < 8))
                    entries += 256
                    diff = keep_bits(r8[m][None, :], b[:, None]) - keep_bits(y8[m], b[:, None])
                    T[m] = (diff * diff).sum(1)
                Sv = T[np.arange(M)[None, :], cd].sum(1)
                d = ((Sv.astype(F32)) * scale).astype(F32)
                key = Sv
            else:
                T32 = ivfpq.lut_fp32(Q[i], index.centroids[l], index.books)
                d = ivfpq.adc_fp32(T32, cd, pd[i, j])
                key = d
            ds.append((key, d))
            idl.append(index.ids[mem])
        if ds:
            keys = np.concatenate([a for a, _ in ds])
            dd = np.concatenate([b for _, b in ds])
            ids = np.concatenate(idl)
            sel = np.lexsort((ids, keys))[:k]
            out_i[i, :len(sel)] = ids[sel]
            out_d[i, :len(sel)] = dd[sel]
    return out_i, out_d, dict(cl_low=cl_low, lc_low=(low / entries if entries else 0.0))
