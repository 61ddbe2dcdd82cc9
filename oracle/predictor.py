"""CPU oracle of the precision choice — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.

Section 3.3 turns the separation condition of Eq. 1, P(d1 <= d2) >= P(d > 3 r1 + r2),
into the precision function f(d, r1, r2) = d - 3 r1 - r2 (Eq. 2): the larger f,
the lower the precision a cluster needs. It then replaces the centre-to-centre
distance d by the query-to-cluster distance d' and adds cluster sizes, giving
features {d', r1, r2, n1, n2} where cluster 1 is the query's nearest. A learned
model maps features to a precision (Section 3.4 uses an SVR; this build uses a
5-32-32-5 MLP classifier over the bit widths 4/6/8/12/16).

Readings (the paper fixes none of these):
* feature vector of probe rank j (0-based) of a query with nprobe probes:
  (sqrt(D2_j) - sqrt(D2_0), r_0, r_j, sqrt(n_j), j / nprobe), all FP32, with
  D2 the FP32 coarse distances, r the covering radius of a list and n its size;
  features are normalised as fl32(fl32(x - mean) * inv_std).
* Eq. 2 heuristic ("the method without the network"): g = f / r_j with
  f = d' - 3 r_0 - r_j; the pair gets the fewest bits whose threshold g
  reaches.
* labels (Section 3.3, Fig. 6, read as "fewest bits that keep the top-k"):
  tau = (d_k + d_{k+1}) / 2 of the FP32 top-(k+1) over the probed lists;
  margin_l = min_{x in l} |d(x) - tau|; E_l(b) = max_{x in l} |dhat_b(x) - d(x)|;
  label = fewest b with E_l(b) < margin_l, else "needs FP32".
* MLP inference: FP16 operands (weights, biases, inputs, hidden activations),
  FP32 accumulation in ascending input order starting from the bias, ReLU on
  the hidden layers, FP32 logits; the width is the fewest bits c with
  fl32(max_{i<=c} z_i - max_{i>c} z_i) >= tau, else 16 bits (decide_bits).
"""
from __future__ import annotations

import numpy as np

from . import ivfpq

F16 = np.float16
F32 = np.float32
F64 = np.float64
BITS = ivfpq.BITS
NFEAT, H1, H2, NCLS = 5, 32, 32, 5


# ----------------------------------------------------------------- Eq. 1 / Eq. 2

def eq1_bound_holds(d, r1, r2) -> np.ndarray:
    """Eq. 1's sufficient condition for a neighbour in C1 to beat one in C2: d > 3 r1 + r2."""
    return np.asarray(d, dtype=F64) > 3.0 * np.asarray(r1, dtype=F64) + np.asarray(r2, dtype=F64)


def eq2(d, r1, r2) -> np.ndarray:
    """Eq. 2: f(d, r1, r2) = d - 3 r1 - r2 (FP64)."""
    return np.asarray(d, dtype=F64) - 3.0 * np.asarray(r1, dtype=F64) - np.asarray(r2, dtype=F64)


def eq2_fp32(dprime, r1, r2) -> np.ndarray:
    """FP32 rule for Eq. 2: fl32(fl32(d' - fl32(3 * r1)) - r2)."""
    a = (F32(3.0) * np.asarray(r1, dtype=F32)).astype(F32)
    return ((np.asarray(dprime, dtype=F32) - a).astype(F32) - np.asarray(r2, dtype=F32)).astype(F32)


# ----------------------------------------------------------------- features

def features(probe_d2: np.ndarray, probes: np.ndarray, radius: np.ndarray,
             sizes: np.ndarray, nprobe_per_q=None) -> np.ndarray:
    """Raw FP32 features [nq, nprobe, 5] of every (query, probe rank) pair."""
    pd = np.asarray(probe_d2, dtype=F32)
    nq, npb = pd.shape
    s = np.sqrt(pd).astype(F32)
    rad = np.asarray(radius, dtype=F32)
    out = np.zeros((nq, npb, NFEAT), dtype=F32)
    out[:, :, 0] = (s - s[:, :1]).astype(F32)
    out[:, :, 1] = rad[probes[:, :1]]
    out[:, :, 2] = rad[probes]
    out[:, :, 3] = np.sqrt(np.asarray(sizes, dtype=F32)[probes]).astype(F32)
    npq = np.full(nq, npb) if nprobe_per_q is None else np.asarray(nprobe_per_q)
    for i in range(nq):
        j = np.arange(npb, dtype=F32)
        out[i, :, 4] = (j / F32(npq[i])).astype(F32)
    return out


def normalise(x: np.ndarray, mean: np.ndarray, inv_std: np.ndarray) -> np.ndarray:
    """fl32(fl32(x - mean) * inv_std)."""
    return ((np.asarray(x, dtype=F32) - np.asarray(mean, dtype=F32)).astype(F32)
            * np.asarray(inv_std, dtype=F32)).astype(F32)


def eq2_bits(feat: np.ndarray, thresholds) -> np.ndarray:
    """Eq. 2 heuristic: g = f / r_j with f = d' - 3 r_0 - r_j (FP32 rule); the
    fewest bits b_i whose threshold g >= thresholds[i] holds (thresholds for
    4, 6, 8, 12 bits, non-increasing); otherwise 16."""
    f = eq2_fp32(feat[..., 0], feat[..., 1], feat[..., 2])
    rj = feat[..., 2].astype(F32)
    g = np.where(rj > 0, (f / np.where(rj > 0, rj, F32(1))).astype(F32), F32(-np.inf))
    out = np.full(f.shape, 16, dtype=np.uint8)
    for b, th in reversed(list(zip((4, 6, 8, 12), thresholds))):
        out = np.where(g >= F32(th), np.uint8(b), out)
    return out


# ------------------------------------------------------------------- labels

def labels_for_query(index: ivfpq.Index, q: np.ndarray, probes_q: np.ndarray, k: int):
    """Label sweep for one query over its probed lists (reading in the docstring).

    Returns (label bits per probe, 0 = needs FP32; tau; per-probe margins;
    per-probe E[b] for b in BITS as an array [nprobe, 5]).
    """
    T = []
    dl = []
    d2s = ivfpq.coarse_d2_fp32(np.asarray(q)[None], index.centroids[np.asarray(probes_q)])[0]
    for j, l in enumerate(probes_q):
        l = int(l)
        T32 = ivfpq.lut_fp32(q, index.centroids[l], index.books)
        T.append(T32)
        mem = index.members[l]
        dl.append(ivfpq.adc_fp32(T32, index.codes[mem], d2s[j]) if len(mem) else np.zeros(0, F32))
    alld = np.concatenate(dl) if dl else np.zeros(0, F32)
    allid = np.concatenate([index.ids[index.members[int(l)]] for l in probes_q]) if dl else np.zeros(0, np.int64)
    if alld.size > k:
        sel = ivfpq.smallest(alld, allid, k + 1)
        tau = (F64(alld[sel[k - 1]]) + F64(alld[sel[k]])) / 2.0
    else:
        tau = F64(np.inf)
    out = np.zeros(len(probes_q), dtype=np.uint8)
    margins = np.full(len(probes_q), np.inf)
    errs = np.zeros((len(probes_q), len(BITS)))
    for j, l in enumerate(probes_q):
        l = int(l)
        mem = index.members[l]
        if len(mem) == 0:
            out[j] = BITS[0]
            continue
        d = dl[j].astype(F64)
        margin = np.min(np.abs(d - tau))
        margins[j] = margin
        cd = index.codes[mem]
        lab = 0
        for bi, b in enumerate(BITS):
            qz = ivfpq.quantize_lut(T[j], b, d2s[j])
            dh = ivfpq.dequant32(ivfpq.adc_int(qz["t"], cd), qz["delta32"], qz["B32"]).astype(F64)
            errs[j, bi] = np.max(np.abs(dh - d))
            if lab == 0 and errs[j, bi] < margin:
                lab = b
        out[j] = lab
    return out, tau, margins, errs


def labels(index: ivfpq.Index, Q: np.ndarray, nprobe: int, k: int) -> np.ndarray:
    """Label bits [nq, nprobe] for training queries (0 = needs FP32)."""
    D2 = ivfpq.coarse_d2_fp32(Q, index.centroids)
    probes, _ = ivfpq.locate(D2, nprobe)
    return np.stack([labels_for_query(index, Q[i], probes[i], k)[0] for i in range(len(Q))])


# --------------------------------------------------------------------- MLP

def init_mlp(seed: int = 0) -> dict:
    """He-uniform initial weights (FP32 master copy)."""
    r = np.random.Generator(np.random.PCG64(seed))

    def lin(o, i):
        lim = np.sqrt(6.0 / i)
        return r.uniform(-lim, lim, size=(o, i)).astype(F32), np.zeros(o, dtype=F32)

    W1, b1 = lin(H1, NFEAT)
    W2, b2 = lin(H2, H1)
    W3, b3 = lin(NCLS, H2)
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def mlp_forward64(p: dict, X: np.ndarray) -> dict:
    """FP64 forward: z = W3 relu(W2 relu(W1 x + b1) + b2) + b3."""
    X = np.asarray(X, dtype=F64)
    a1 = X @ p["W1"].astype(F64).T + p["b1"].astype(F64)
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].astype(F64).T + p["b2"].astype(F64)
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].astype(F64).T + p["b3"].astype(F64)
    return dict(X=X, a1=a1, h1=h1, a2=a2, h2=h2, z=z)


def softmax_ce64(z: np.ndarray, y: np.ndarray) -> tuple[float, np.ndarray]:
    """Mean softmax cross-entropy and its gradient with respect to the logits."""
    z = np.asarray(z, dtype=F64)
    zm = z - z.max(axis=1, keepdims=True)
    e = np.exp(zm)
    p = e / e.sum(axis=1, keepdims=True)
    n = z.shape[0]
    loss = -np.mean(np.log(p[np.arange(n), y]))
    g = p.copy()
    g[np.arange(n), y] -= 1.0
    return float(loss), g / n


def mlp_backward64(p: dict, fw: dict, gz: np.ndarray) -> dict:
    """FP64 backward of mlp_forward64 given dLoss/dz."""
    g = {}
    g["W3"] = gz.T @ fw["h2"]
    g["b3"] = gz.sum(axis=0)
    gh2 = gz @ p["W3"].astype(F64)
    ga2 = gh2 * (fw["a2"] > 0)
    g["W2"] = ga2.T @ fw["h1"]
    g["b2"] = ga2.sum(axis=0)
    gh1 = ga2 @ p["W2"].astype(F64)
    ga1 = gh1 * (fw["a1"] > 0)
    g["W1"] = ga1.T @ fw["X"]
    g["b1"] = ga1.sum(axis=0)
    return g


def loss_and_grad64(p: dict, X: np.ndarray, y: np.ndarray):
    fw = mlp_forward64(p, X)
    loss, gz = softmax_ce64(fw["z"], y)
    return loss, mlp_backward64(p, fw, gz)


def loss_and_grad16(p: dict, Xn: np.ndarray, y: np.ndarray, high_weight: float = 1.0):
    """Softmax-CE loss and gradients of the network the GPU trains: FP16
    weights, biases and normalised inputs, hidden activations rounded to FP16
    after ReLU (the inference rule), evaluated in FP64 with those roundings.
    The loss is (1/n) sum_i w_i CE_i, w_i = high_weight for classes 3 and 4
    (12 and 16 bits), else 1."""
    p16 = {k: np.asarray(v, dtype=F32).astype(F16).astype(F64) for k, v in p.items()}
    X = np.asarray(Xn, dtype=F32).astype(F16).astype(F64)
    a1 = X @ p16["W1"].T + p16["b1"]
    h1 = np.maximum(a1, 0.0).astype(F16).astype(F64)
    a2 = h1 @ p16["W2"].T + p16["b2"]
    h2 = np.maximum(a2, 0.0).astype(F16).astype(F64)
    z = h2 @ p16["W3"].T + p16["b3"]
    y = np.asarray(y)
    w = np.where(y >= 3, float(high_weight), 1.0)
    zm = z - z.max(axis=1, keepdims=True)
    pr = np.exp(zm)
    pr /= pr.sum(axis=1, keepdims=True)
    n = z.shape[0]
    loss = float(np.mean(-w * np.log(pr[np.arange(n), y])))
    gz = pr.copy()
    gz[np.arange(n), y] -= 1.0
    gz *= (w / n)[:, None]
    fw = dict(X=X, a1=a1, h1=h1, a2=a2, h2=h2, z=z)
    return loss, mlp_backward64(p16, fw, gz)


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (FP64) of every parameter; returns new (p, m, v)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in p:
        mk = b1 * m[k] + (1 - b1) * g[k]
        vk = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = mk / (1 - b1 ** t)
        vh = vk / (1 - b2 ** t)
        out_p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v


def to_fp16(p: dict) -> dict:
    return {k: np.asarray(v, dtype=F32).astype(F16) for k, v in p.items()}


def _layer16(W16, b16, x16, relu: bool):
    """acc = b; for i ascending: acc = fl32(acc + W[o,i] * x[i]) (product exact in FP32)."""
    W = W16.astype(F32)
    acc = np.broadcast_to(b16.astype(F32), (x16.shape[0], W.shape[0])).astype(F32).copy()
    x = x16.astype(F32)
    for i in range(W.shape[1]):
        acc = (acc + (x[:, i:i + 1] * W[None, :, i]).astype(F32)).astype(F32)
    if relu:
        return np.maximum(acc, F32(0)).astype(F16)
    return acc


def mlp_logits16(p16: dict, Xn: np.ndarray) -> np.ndarray:
    """FP16-operand inference rule; Xn are normalised FP32 features [n, 5]."""
    x16 = np.asarray(Xn, dtype=F32).astype(F16)
    h1 = _layer16(p16["W1"], p16["b1"], x16, True)
    h2 = _layer16(p16["W2"], p16["b2"], h1, True)
    return _layer16(p16["W3"], p16["b3"], h2, False)


def decide_bits(z: np.ndarray, tau: float) -> np.ndarray:
    """Round-up rule on the FP32 logits of the widths 4, 6, 8, 12, 16: the
    fewest bits c such that fl32(max_{i <= c} z_i - max_{i > c} z_i) >= tau,
    16 bits when no narrower width qualifies. tau = 0 gives the argmax with
    ties to the narrower width; a larger tau moves uncertain pairs to wider
    tables (towards full precision)."""
    z = np.asarray(z, dtype=F32)
    n = z.shape[0]
    out = np.full(n, BITS[-1], dtype=np.uint8)
    done = np.zeros(n, dtype=bool)
    for c in range(len(BITS) - 1):
        lo = z[:, :c + 1].max(axis=1)
        hi = z[:, c + 1:].max(axis=1)
        ok = ~done & ((lo - hi).astype(F32) >= F32(tau))
        out[ok] = BITS[c]
        done |= ok
    return out


def gpu_width(bits: np.ndarray) -> np.ndarray:
    """Widths mapped to GB300 tables: 6 -> 8 bits, 12 and 16 -> FP32 (0)."""
    b = np.asarray(bits, dtype=np.uint8)
    return np.where(b == 6, np.uint8(8), np.where((b == 12) | (b == 16), np.uint8(0), b)).astype(np.uint8)


def bits_to_class(bits: np.ndarray, gpu: bool = False, nibble: bool = False) -> np.ndarray:
    """Training target: class of the label bits; "needs FP32" trains as 16 bits.
    With `gpu`, the two tables of the GB300 width map: 4, 6, 8 -> class 2
    (8 bits); 12, 16 and FP32 -> class 4 (16 bits). With `nibble`, its three
    tables: 4 -> class 0; 6, 8 -> class 2; 12, 16 and FP32 -> class 4."""
    b = np.asarray(bits)
    lut = {4: 0, 6: 1, 8: 2, 12: 3, 16: 4, 0: 4}
    if gpu:
        lut = {4: 2, 6: 2, 8: 2, 12: 4, 16: 4, 0: 4}
    if nibble:
        lut = {4: 0, 6: 2, 8: 2, 12: 4, 16: 4, 0: 4}
    return np.vectorize(lambda v: lut[int(v)])(b).astype(np.int64)
