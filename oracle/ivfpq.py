"""CPU oracle of the IVF-PQ search stages — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module. It is deliberately plain numpy: one stage per function, in the
order Section 2.1 (Fig. 1) lists them.

  CL  cluster locating: squared L2 distance from the query to every centroid,
      then the ``nprobe`` nearest lists (Section 2.1).
  RC  residual r = q - c_l (Section 2.1).
  LC  lookup table T[m][c] = ||r_m - y_{m,c}||^2 over the M sub-spaces and the
      256 entries of the shared codebook (Section 2.1).
  DC  ADC distance d(x) = sum_m T[m][code_m(x)] (Section 2.1; the DRM adder tree
      of Section 4.1).
  TS  the k smallest distances (Section 2.1; TSM of Section 4.1).

Two families of functions:

* ``*_fp64``: the definitions in double precision. These are what the paper
  computes; float outputs of the library are checked against them with a
  tolerance.
* ``*_fp32`` and the quantiser: the single-precision evaluation rules that the
  library follows step for step wherever a rounding decides an integer (which
  lists are probed, which LUT level an entry maps to, which ids are returned).
  Each is written as an explicit sequence of IEEE operations with one rounding
  per operation, no fused multiply-add and a fixed summation order, so the
  library must reproduce it bit for bit.

The FP32 LUT follows the published IVFADC look-up-table decomposition for
residual PQ (Johnson, Douze and Jegou, "Billion-scale similarity search with
GPUs", 2017): with r = q - c_l and y = y_{m,c},
  ||r_m - y||^2 = ||q_m - c_{l,m}||^2 + (||y||^2 + 2 <c_{l,m}, y>) - 2 <q_m, y>
                =      term 1       +          term 2             + term 3.
Term 1 summed over m is the coarse distance D2 that CL already has; term 2
depends only on the list (it is tabulated once per list when the index is
built); term 3 depends only on the query (tabulated once per query and shared
by all its probes). The FP32 table of a pair is T'[m][c] = fl32(term2 + term3)
(the entry shifted by ||r_m||^2), and the ADC distance is D2 + sum_m T'. The
FP64 definitions keep the direct form ||r_m - y||^2 of Section 2.1.

Readings where the paper is silent (the paper states no quantiser, bit-width
set, tie rule or feature normalisation):

* Tie rule: ascending (distance, list id) in CL, ascending (distance, id) in TS.
* Quantiser of a (query, list) LUT at b bits: per sub-table bias_m = min_c T,
  one step Delta = range / (2^b - 1) shared by all sub-tables (so that integer
  sums over m are coherent), t = round-half-even((T - bias_m) * s) with
  s = fl32((2^b - 1) / range) clamped to [0, 2^b - 1]; the distance estimate is
  fl32(fl32(Delta32 * S) + B32) with S the exact integer sum. The offset B32
  is the exact (rational) sum of the pair's FP32 coarse distance and the M
  biases, rounded once to the nearest FP32 value (ties to even): a value
  that no summation order changes.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

F32 = np.float32
F64 = np.float64
KSUB = 256
BITS = (4, 6, 8, 12, 16)


# ---------------------------------------------------------------- CL (Section 2.1)

def coarse_d2_fp64(Q: np.ndarray, C: np.ndarray) -> np.ndarray:
    """D2[q, l] = sum_d (q_d - c_{l,d})^2 in FP64, by direct differences."""
    Q = np.asarray(Q, dtype=F64)
    C = np.asarray(C, dtype=F64)
    out = np.empty((Q.shape[0], C.shape[0]), dtype=F64)
    for i in range(Q.shape[0]):
        diff = C - Q[i][None, :]
        out[i] = np.einsum("ld,ld->l", diff, diff)
    return out


def coarse_d2_fp32(Q: np.ndarray, C: np.ndarray) -> np.ndarray:
    """FP32 rule for D2: acc = 0; for d = 0..D-1 ascending:
    e = fl32(q_d - c_d); acc = fl32(acc + fl32(e * e))."""
    Q = np.asarray(Q, dtype=F32)
    C = np.asarray(C, dtype=F32)
    acc = np.zeros((Q.shape[0], C.shape[0]), dtype=F32)
    for d in range(Q.shape[1]):
        e = (Q[:, d][:, None] - C[:, d][None, :]).astype(F32)
        acc = (acc + (e * e).astype(F32)).astype(F32)
    return acc


def smallest(d: np.ndarray, key: np.ndarray, n: int) -> np.ndarray:
    """Positions of the n smallest (d, key) pairs, in ascending order."""
    order = np.lexsort((np.asarray(key), np.asarray(d)))
    return order[:n]


def locate(D2: np.ndarray, nprobe: int) -> tuple[np.ndarray, np.ndarray]:
    """CL selection: per query the nprobe smallest (D2, list id)."""
    nq, nlist = D2.shape
    lists = np.arange(nlist)
    probes = np.empty((nq, nprobe), dtype=np.int32)
    pd = np.empty((nq, nprobe), dtype=D2.dtype)
    for i in range(nq):
        sel = smallest(D2[i], lists, nprobe)
        probes[i] = sel
        pd[i] = D2[i][sel]
    return probes, pd


# ------------------------------------------------------- RC + LC (Section 2.1)

def lut_fp64(q: np.ndarray, c: np.ndarray, books: np.ndarray) -> np.ndarray:
    """T[m][c'] = ||(q - c)_m - y_{m,c'}||^2 in FP64. ``books`` is [M, 256, dsub]."""
    M, ksub, dsub = books.shape
    r = np.asarray(q, dtype=F64) - np.asarray(c, dtype=F64)
    T = np.zeros((M, ksub), dtype=F64)
    for m in range(M):
        diff = r[m * dsub:(m + 1) * dsub][None, :] - np.asarray(books[m], dtype=F64)
        T[m] = np.einsum("cj,cj->c", diff, diff)
    return T


def lut_shift_fp64(q: np.ndarray, c: np.ndarray, books: np.ndarray) -> np.ndarray:
    """The shifted table T'[m][c'] = ||r_m - y_{m,c'}||^2 - ||r_m||^2 in FP64."""
    M, ksub, dsub = books.shape
    r = np.asarray(q, dtype=F64) - np.asarray(c, dtype=F64)
    rn = np.array([np.dot(r[m * dsub:(m + 1) * dsub], r[m * dsub:(m + 1) * dsub]) for m in range(M)])
    return lut_fp64(q, c, books) - rn[:, None]


def _dot_rule(a: np.ndarray, y: np.ndarray) -> np.ndarray:
    """acc = 0; for j ascending: acc = fl32(acc + fl32(a_j * y_j)); a is [M, dsub], y [M, 256, dsub]."""
    acc = np.zeros(y.shape[:2], dtype=F32)
    for j in range(y.shape[2]):
        acc = (acc + (a[:, j][:, None] * y[:, :, j]).astype(F32)).astype(F32)
    return acc


def query_table_fp32(q: np.ndarray, books: np.ndarray) -> np.ndarray:
    """FP32 rule for <q_m, y_{m,c}> (dot rule, j ascending); term 3 of the
    decomposition is -2 times this table."""
    M, _, dsub = books.shape
    return _dot_rule(np.asarray(q, dtype=F32).reshape(M, dsub), np.asarray(books, dtype=F32))


def list_table_fp32(c: np.ndarray, books: np.ndarray) -> np.ndarray:
    """FP32 rule for term 2 of the decomposition, fl32(||y||^2 + fl32(2 <c_{l,m}, y>)),
    both inner products by the dot rule."""
    M, _, dsub = books.shape
    y = np.asarray(books, dtype=F32)
    yn = np.zeros(y.shape[:2], dtype=F32)
    for j in range(dsub):
        yn = (yn + (y[:, :, j] * y[:, :, j]).astype(F32)).astype(F32)
    cy = _dot_rule(np.asarray(c, dtype=F32).reshape(M, dsub), y)
    return (yn + (F32(2.0) * cy).astype(F32)).astype(F32)


def lut_fp32(q: np.ndarray, c: np.ndarray, books: np.ndarray) -> np.ndarray:
    """FP32 rule for the shifted table: T' = fl32(P_l - fl32(2 Q_q))."""
    P = list_table_fp32(c, books)
    Qt = query_table_fp32(q, books)
    return (P - (F32(2.0) * Qt).astype(F32)).astype(F32)


# ----------------------------------------------- precision: the LUT quantiser

def quantize_lut(T32: np.ndarray, b: int, d2=0.0) -> dict:
    """Quantise one (query, list) FP32 LUT to b bits (rule in the module docstring).

    ``d2`` is the pair's FP32 coarse distance, folded into the offset. Returns
    the integer table ``t`` [M, 256] (int64), the FP32 biases, the FP32 range,
    the FP64 step ``delta64`` = fl64(range / L) and its FP32 rounding
    ``delta32``, the FP32 multiplier ``s32``, and the offset: ``B_exact`` (the
    exact rational d2 + sum of the biases), ``B64`` and ``B32`` (its nearest
    FP64 and FP32 values).
    """
    assert b in BITS
    T32 = np.asarray(T32, dtype=F32)
    L = (1 << b) - 1
    bias = T32.min(axis=1).astype(F32)                      # exact
    Tp = (T32 - bias[:, None]).astype(F32)
    rng = F32(Tp.max())
    if rng > 0:
        delta64 = F64(rng) / F64(L)
        s32 = F32(F64(L) / F64(rng))
    else:
        delta64 = F64(0.0)
        s32 = F32(0.0)
    y = (Tp * s32).astype(F32)
    t = np.minimum(np.rint(y), L).astype(np.int64)          # rint: half to even
    B_exact = exact_sum([F32(d2)] + list(bias))
    return dict(t=t, bias=bias, range=rng, delta64=delta64, s32=s32, B_exact=B_exact,
                B64=F64(float(B_exact)), delta32=F32(delta64), B32=nearest_f32(B_exact), L=L)


def exact_sum(values) -> Fraction:
    """The exact sum of finite floating-point values, as a rational number."""
    return sum((Fraction(float(v)) for v in values), Fraction(0))


def nearest_f32(x: Fraction) -> np.float32:
    """The FP32 value nearest to the rational ``x``; of two equally near ones
    the one with an even significand (IEEE 754 round to nearest, ties to even).
    Beyond the largest finite value by half an ulp or more: infinity."""
    big = Fraction(float(np.finfo(F32).max)) + Fraction(2) ** (127 - 24)
    if abs(x) >= big:
        return F32(np.inf) if x > 0 else F32(-np.inf)
    with np.errstate(over="ignore"):
        guess = F32(float(x))               # within one ulp of the answer
    if not np.isfinite(guess):
        guess = np.finfo(F32).max
    cands = [guess, np.nextafter(guess, F32(-np.inf)), np.nextafter(guess, F32(np.inf))]
    cands = [c for c in cands if np.isfinite(c)]
    best = min(abs(Fraction(float(c)) - x) for c in cands)
    near = [c for c in cands if abs(Fraction(float(c)) - x) == best]
    near.sort(key=lambda c: int(np.asarray(c, dtype=F32).view(np.uint32)) & 1)
    return F32(near[0])


def exact_sum_f32(values) -> np.float32:
    """The exact sum of finite FP32 values rounded once to FP32 (order-free)."""
    return nearest_f32(exact_sum(values))


# ----------------------------------------------------------- DC (Section 2.1)

def adc_fp64(T: np.ndarray, codes: np.ndarray) -> np.ndarray:
    """d(x) = sum_m T[m][code_m(x)] in FP64."""
    codes = np.asarray(codes)
    M = codes.shape[1]
    return np.asarray(T, dtype=F64)[np.arange(M)[None, :], codes.astype(np.int64)].sum(axis=1)


def adc_fp32(T32: np.ndarray, codes: np.ndarray, d2=0.0) -> np.ndarray:
    """FP32 rule: acc = 0; for m = 0..M-1 ascending: acc = fl32(acc + T'[m][code_m]);
    the distance is fl32(d2 + acc) with d2 the pair's FP32 coarse distance."""
    codes = np.asarray(codes).astype(np.int64)
    acc = np.zeros(codes.shape[0], dtype=F32)
    for m in range(codes.shape[1]):
        acc = (acc + T32[m][codes[:, m]]).astype(F32)
    return (F32(d2) + acc).astype(F32)


def adc_int(t: np.ndarray, codes: np.ndarray) -> np.ndarray:
    """S(x) = sum_m t[m][code_m(x)] as an exact integer."""
    codes = np.asarray(codes).astype(np.int64)
    M = codes.shape[1]
    return np.asarray(t, dtype=np.int64)[np.arange(M)[None, :], codes].sum(axis=1)


def dequant32(S: np.ndarray, delta32, B32) -> np.ndarray:
    """Distance estimate fl32(fl32(Delta32 * fl32(S)) + B32)."""
    s = np.asarray(S, dtype=np.int64)
    assert np.all(s < (1 << 24)), "S must be exact in FP32"
    return ((F32(delta32) * s.astype(F32)).astype(F32) + F32(B32)).astype(F32)


# ----------------------------------------------------------- TS (Section 2.1)

def topk(d: np.ndarray, ids: np.ndarray, k: int, dtype=F32) -> tuple[np.ndarray, np.ndarray]:
    """The k smallest (d, id), ascending; padded with (id -1, +inf)."""
    sel = smallest(d, ids, k)
    out_i = np.full(k, -1, dtype=np.int64)
    out_d = np.full(k, np.inf, dtype=dtype)
    out_i[:len(sel)] = np.asarray(ids)[sel]
    out_d[:len(sel)] = np.asarray(d)[sel]
    return out_i, out_d


# --------------------------------------------------------------- the index

class Index:
    """The IVF-PQ index as plain arrays grouped by list (Section 2.1).

    Per list: member rows in ascending row order, n_l, and the covering
    radius r_l = max over members of ||x_hat - c_l|| where x_hat is the PQ
    reconstruction c_l + concat_m y_{m, code_m} (FP64).
    """

    def __init__(self, centroids, codebooks, codes, list_of, ids=None):
        self.centroids = np.asarray(centroids, dtype=F32)
        self.books = np.asarray(codebooks, dtype=F32)
        self.codes = np.asarray(codes, dtype=np.uint8)
        self.list_of = np.asarray(list_of, dtype=np.int64)
        n = self.codes.shape[0]
        self.ids = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, dtype=np.int64)
        self.nlist, self.dim = self.centroids.shape
        self.M, ksub, self.dsub = self.books.shape
        assert ksub == KSUB and self.M * self.dsub == self.dim
        order = np.argsort(self.list_of, kind="stable")
        bounds = np.searchsorted(self.list_of[order], np.arange(self.nlist + 1))
        self.members = [order[bounds[l]:bounds[l + 1]] for l in range(self.nlist)]
        self.sizes = np.array([len(m) for m in self.members], dtype=np.int64)
        # ||y_{m,c}||^2 in FP64, j ascending; then per member, m ascending.
        y = self.books.astype(F64)
        ynorm2 = np.zeros((self.M, ksub), dtype=F64)
        for j in range(self.dsub):
            ynorm2 = ynorm2 + y[:, :, j] * y[:, :, j]
        self.radius = np.zeros(self.nlist, dtype=F64)
        for l in range(self.nlist):
            if len(self.members[l]):
                cd = self.codes[self.members[l]].astype(np.int64)
                rn2 = np.zeros(len(cd), dtype=F64)
                for m in range(self.M):
                    rn2 = rn2 + ynorm2[m, cd[:, m]]
                self.radius[l] = np.sqrt(rn2.max())

    def reconstruct(self, rows: np.ndarray) -> np.ndarray:
        """x_hat = c_{list(x)} + concat_m y_{m, code_m(x)} in FP64."""
        rows = np.asarray(rows)
        cd = self.codes[rows].astype(np.int64)
        parts = self.books.astype(F64)[np.arange(self.M)[None, :], cd]   # [n, M, dsub]
        return self.centroids[self.list_of[rows]].astype(F64) + parts.reshape(len(rows), self.dim)


def search(index: Index, Q: np.ndarray, nprobe: int, k: int, bits=0,
           nprobe_per_q=None, k_per_q=None, fp64: bool = False,
           return_probes: bool = False):
    """Full search: CL -> RC -> LC -> (quantise) -> DC -> TS for every query.

    ``bits`` is 0 (plain FP32 LUT), one of 4/6/8/12/16 for every pair, or an
    int array [nq, nprobe] giving the bits of each (query, probe rank) pair.
    With ``fp64=True`` every stage uses its FP64 definition and ``bits`` must
    be 0. Outputs ids [nq, k] int64 and dists [nq, k] (padding id -1, +inf).
    """
    Q = np.asarray(Q)
    nq = Q.shape[0]
    bits_arr = np.broadcast_to(np.asarray(bits), (nq, nprobe))
    D2 = coarse_d2_fp64(Q, index.centroids) if fp64 else coarse_d2_fp32(Q, index.centroids)
    probes, pd = locate(D2, nprobe)
    dt = F64 if fp64 else F32
    out_i = np.full((nq, k), -1, dtype=np.int64)
    out_d = np.full((nq, k), np.inf, dtype=dt)
    for i in range(nq):
        npq = nprobe if nprobe_per_q is None else int(nprobe_per_q[i])
        kq = k if k_per_q is None else int(k_per_q[i])
        ds, idl = [], []
        for j in range(npq):
            l = int(probes[i, j])
            mem = index.members[l]
            if len(mem) == 0:
                continue
            cd = index.codes[mem]
            b = int(bits_arr[i, j])
            if fp64:
                assert b == 0
                d = adc_fp64(lut_fp64(Q[i], index.centroids[l], index.books), cd)
            else:
                T32 = lut_fp32(Q[i], index.centroids[l], index.books)
                d2 = pd[i, j]
                if b == 0:
                    d = adc_fp32(T32, cd, d2)
                else:
                    qz = quantize_lut(T32, b, d2)
                    d = dequant32(adc_int(qz["t"], cd), qz["delta32"], qz["B32"])
            ds.append(d)
            idl.append(index.ids[mem])
        if ds:
            ti, td = topk(np.concatenate(ds), np.concatenate(idl), kq, dt)
            out_i[i, :kq] = ti
            out_d[i, :kq] = td
    if return_probes:
        return out_i, out_d, probes, pd
    return out_i, out_d


def knn_bruteforce(base: np.ndarray, Q: np.ndarray, k: int, ids=None):
    """Exact kNN in FP64 by direct differences, ties by ascending id."""
    base = np.asarray(base, dtype=F64)
    ids = np.arange(base.shape[0], dtype=np.int64) if ids is None else np.asarray(ids)
    out_i = np.empty((len(Q), k), dtype=np.int64)
    out_d = np.empty((len(Q), k), dtype=F64)
    for i, q in enumerate(np.asarray(Q, dtype=F64)):
        diff = base - q[None, :]
        d = np.einsum("nd,nd->n", diff, diff)
        out_i[i], out_d[i] = topk(d, ids, k, F64)
    return out_i, out_d
