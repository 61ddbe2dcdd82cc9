"""CPU oracle of the SVR-RBF precision predictor (Section 3.4) — TEST
INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.

Section 3.4 fits the precision function with support-vector regression on a
Gaussian (RBF) kernel, trained on a small sample (1280 feature/label pairs:
the kernel matrix is quadratic in the sample count), and evaluates the
exponential through a lookup table at inference. This module states that
model in FP64.

Readings (the paper fixes the kernel, the sample count and the lookup-table
idea; it fixes neither the solver nor the bias nor the table):
* model: f(x) = sum_i beta_i (K(x_i, x) + 1) with K(x, y) = exp(-gamma |x - y|^2);
  the constant 1 is the bias, absorbed into the kernel as a constant feature.
* training: epsilon-insensitive regression, as its dual over the box
  beta in [-C, C]^n:
      minimise  L(beta) = 1/2 beta^T K1 beta - y^T beta + eps * |beta|_1,
      K1 = K + 1 (the matrix of K(x_i, x_j) + 1).
  Solver: exact coordinate descent. Each step sets beta_i to the minimiser of
  L in that coordinate (a soft threshold of the Newton step, then a clip to
  the box), for i ascending in sweeps, until the largest change in a sweep is
  at most tol or max_sweeps sweeps ran. L is convex and each step exact, so
  the sweeps converge to the optimum. The optimum satisfies, with
  g_i = f(x_i) - y_i:  beta_i = 0 -> |g_i| <= eps;  0 < beta_i < C -> g_i = -eps;
  -C < beta_i < 0 -> g_i = eps;  beta_i = C -> g_i <= -eps;  beta_i = -C -> g_i >= eps.
* targets and widths: the label's index in (4, 6, 8, 12, 16, FP32) = 0..5;
  the predicted width is the one at index clip(ceil(f(x) - margin), 0, 5)
  (margin > 0 moves pairs towards narrower widths, margin < 0 towards wider
  ones).
* exponential by lookup table: exp(-t) for t >= 0 from a table of
  exp(-t_k) at t_k = k * step, k = 0..n-1, linearly interpolated; 0 past the
  table. Its error is bounded by step^2 / 8 (the second derivative of exp(-t)
  is at most 1 on t >= 0) plus the tail exp(-t_max) past the table.
* inference on the GPU (``predict32``): the same model as a fixed sequence of
  FP32 operations, one rounding each, so that the width it decides is exact.
  The table is the geometric sequence of a ratio rho = exp(-step) chosen as
  a dyadic number: e_0 = 1, e_k = fl64(e_{k-1} * rho), each entry rounded
  once to FP32 (no exponential function is evaluated, so no library's exp
  enters the table); 1/step is a model parameter.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64
WIDTHS = (4, 6, 8, 12, 16, 0)  # index 5: FP32 (0)


def rbf(X: np.ndarray, Y: np.ndarray, gamma: float) -> np.ndarray:
    """K(x, y) = exp(-gamma |x - y|^2) for every row pair, FP64."""
    X = np.asarray(X, F64)
    Y = np.asarray(Y, F64)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2)
    return np.exp(-gamma * d2)


def objective(beta: np.ndarray, K1: np.ndarray, y: np.ndarray, eps: float) -> float:
    """L(beta) of the dual (module docstring)."""
    beta = np.asarray(beta, F64)
    return float(0.5 * beta @ K1 @ beta - np.asarray(y, F64) @ beta + eps * np.abs(beta).sum())


def fit(X: np.ndarray, y: np.ndarray, C: float, gamma: float, eps: float,
        tol: float = 1e-10, max_sweeps: int = 10000) -> dict:
    """Coordinate descent on the dual; returns the model {"X", "beta", "gamma"}
    and the number of sweeps run."""
    X = np.asarray(X, F64)
    y = np.asarray(y, F64)
    n = len(y)
    K1 = rbf(X, X, gamma) + 1.0
    beta = np.zeros(n, F64)
    f = np.zeros(n, F64)  # f(x_i) = (K1 beta)_i, kept up to date
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        big = 0.0
        for i in range(n):
            a = K1[i, i]
            # L in coordinate i: 1/2 a b^2 + (f_i - a beta_i - y_i) b + eps |b|
            c = f[i] - a * beta[i] - y[i]
            if c < -eps:
                b = (-c - eps) / a
            elif c > eps:
                b = (-c + eps) / a
            else:
                b = 0.0
            b = min(max(b, -C), C)
            d = b - beta[i]
            if d != 0.0:
                f += d * K1[:, i]
                beta[i] = b
                big = max(big, abs(d))
        if big <= tol:
            break
    return {"X": X, "beta": beta, "gamma": float(gamma), "sweeps": sweeps}


def predict(model: dict, Xq: np.ndarray) -> np.ndarray:
    """f(x) = sum_i beta_i (K(x_i, x) + 1), FP64."""
    K1 = rbf(np.asarray(Xq, F64), model["X"], model["gamma"]) + 1.0
    return K1 @ model["beta"]


def kkt_violation(model: dict, y: np.ndarray, C: float, eps: float) -> float:
    """Largest violation of the optimality conditions (module docstring)."""
    beta = model["beta"]
    g = predict(model, model["X"]) - np.asarray(y, F64)
    v = np.zeros_like(g)
    inner = (beta > -C) & (beta < C)
    zero = beta == 0.0
    v[zero] = np.maximum(np.abs(g[zero]) - eps, 0.0)
    pos = inner & (beta > 0)
    v[pos] = np.abs(g[pos] + eps)
    neg = inner & (beta < 0)
    v[neg] = np.abs(g[neg] - eps)
    top = beta >= C
    v[top] = np.maximum(g[top] + eps, 0.0)
    bot = beta <= -C
    v[bot] = np.maximum(-(g[bot] - eps), 0.0)
    return float(v.max()) if len(v) else 0.0


def widths(f: np.ndarray, margin: float = 0.0) -> np.ndarray:
    """Predicted table widths (0 = FP32) from the regression values."""
    idx = np.clip(np.ceil(np.asarray(f, F64) - margin), 0, len(WIDTHS) - 1).astype(np.int64)
    return np.asarray(WIDTHS, np.uint8)[idx]


def width_index(bits: np.ndarray) -> np.ndarray:
    """Regression target of a label: its index in WIDTHS (0 = FP32 -> 5)."""
    lut = {w: i for i, w in enumerate(WIDTHS)}
    return np.array([lut[int(b)] for b in np.asarray(bits).reshape(-1)], F64).reshape(np.shape(bits))


def exp_table(n: int, t_max: float) -> tuple[np.ndarray, float]:
    """exp(-t_k) at t_k = k * step, k = 0..n-1, step = t_max / (n - 1)."""
    step = t_max / (n - 1)
    return np.exp(-np.arange(n, dtype=F64) * step), step


def exp_lut(t: np.ndarray, table: np.ndarray, step: float) -> np.ndarray:
    """exp(-t) by linear interpolation in the table; 0 past its end."""
    t = np.asarray(t, F64)
    u = t / step
    k = np.floor(u).astype(np.int64)
    inside = (k >= 0) & (k < len(table) - 1)
    kk = np.clip(k, 0, len(table) - 2)
    w = u - kk
    val = table[kk] * (1.0 - w) + table[kk + 1] * w
    return np.where(inside, val, np.where(k < 0, 1.0, 0.0))


def exp_lut_bound(step: float, t_max: float) -> float:
    """Bound on |exp_lut(t) - exp(-t)| for t >= 0."""
    return step * step / 8.0 + float(np.exp(-t_max))


# ------------------------------------------------- FP32 inference rule (GPU)

F32 = np.float32


def exp_table_geometric(n: int, rho: float) -> np.ndarray:
    """FP32 table of exp(-k step), step = -ln(rho): e_0 = 1, e_k = fl64(e_{k-1} rho)
    for k ascending, each entry rounded once to FP32."""
    out = np.empty(n, dtype=F32)
    e = F64(1.0)
    for k in range(n):
        out[k] = F32(e)
        e = F64(e * F64(rho))
    return out


def normalise32(f: np.ndarray, mean, inv_std) -> np.ndarray:
    """x = fl32(fl32(f - mean) * inv_std) per feature."""
    return ((np.asarray(f, F32) - np.asarray(mean, F32)).astype(F32) * np.asarray(inv_std, F32)).astype(F32)


def predict32(sv: np.ndarray, beta: np.ndarray, gamma: float, inv_step: float, table: np.ndarray,
              X: np.ndarray) -> np.ndarray:
    """FP32 rule of f(x) = sum_i beta_i (exp(-gamma |x - sv_i|^2) + 1) with the
    table exponential, for normalised FP32 rows X. Per row: f = 0; for i
    ascending: d2 = 0; for c ascending: e = fl32(x_c - sv_ic),
    d2 = fl32(d2 + fl32(e e)); t = fl32(gamma d2); u = fl32(t * inv_step);
    if u >= n - 1 the exponential is 0, else k = floor(u), w = fl32(u - k),
    ex = fl32(fl32(table_k fl32(1 - w)) + fl32(table_{k+1} w));
    f = fl32(f + fl32(beta_i fl32(ex + 1)))."""
    sv = np.asarray(sv, F32)
    beta = np.asarray(beta, F32)
    X = np.asarray(X, F32)
    table = np.asarray(table, F32)
    n = len(table)
    g, inv = F32(gamma), F32(inv_step)
    f = np.zeros(len(X), dtype=F32)
    for i in range(len(beta)):
        d2 = np.zeros(len(X), dtype=F32)
        for c in range(X.shape[1]):
            e = (X[:, c] - sv[i, c]).astype(F32)
            d2 = (d2 + (e * e).astype(F32)).astype(F32)
        t = (g * d2).astype(F32)
        u = (t * inv).astype(F32)
        inside = u < F32(n - 1)
        k = np.where(inside, np.floor(np.where(inside, u, F32(0))), 0).astype(np.int64)
        w = (u - k.astype(F32)).astype(F32)
        a = (table[k] * (F32(1) - w).astype(F32)).astype(F32)
        b = (table[np.minimum(k + 1, n - 1)] * w).astype(F32)
        ex = np.where(inside, (a + b).astype(F32), F32(0))
        term = (beta[i] * (ex + F32(1)).astype(F32)).astype(F32)
        f = (f + term).astype(F32)
    return f


def widths32(f: np.ndarray, margin: float) -> np.ndarray:
    """Widths from FP32 regression values: index clip(ceil(fl32(f - margin)), 0, 5)."""
    v = (np.asarray(f, F32) - F32(margin)).astype(F32)
    idx = np.clip(np.ceil(v), 0, len(WIDTHS) - 1).astype(np.int64)
    return np.asarray(WIDTHS, np.uint8)[idx]
