"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against an
independent definition (a reconstruction, a brute-force search, Python's own
sort, finite differences, hand-worked values) or an invariant.
"""
import os

import numpy as np
import pytest

from oracle import ivfpq, predictor
from tests.conftest import int_dataset

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _index(ix, ids=None):
    return ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], ids)


# ---------------------------------------------------------------- P1: ADC identity

def test_adc_equals_distance_to_reconstruction(small_a):
    """sum_m T[m][code_m(x)] = ||q - (c_l + decode(x))||^2: the M sub-spaces are
    disjoint blocks of dimensions (Section 2.1), so the LUT sum is the distance
    to the PQ reconstruction."""
    d, ix = small_a
    I = _index(ix)
    for qi in range(4):
        q = d["queries"][qi]
        for l in range(0, I.nlist, 3):
            mem = I.members[l]
            T = ivfpq.lut_fp64(q, I.centroids[l], I.books)
            got = ivfpq.adc_fp64(T, I.codes[mem])
            xh = I.reconstruct(mem)
            want = ((xh - q.astype(np.float64)) ** 2).sum(1)
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_decomposed_table_identity(small_a):
    """D2 + sum_m T'[m][code_m] = ||q - x_hat||^2 in FP64, where T' is the
    table shifted by ||r_m||^2 (the form the FP32 rule evaluates)."""
    d, ix = small_a
    I = _index(ix)
    for qi in range(3):
        q = d["queries"][qi]
        for l in range(0, I.nlist, 4):
            mem = I.members[l]
            D2 = float(((q.astype(np.float64) - I.centroids[l].astype(np.float64)) ** 2).sum())
            got = D2 + ivfpq.adc_fp64(ivfpq.lut_shift_fp64(q, I.centroids[l], I.books), I.codes[mem])
            want = ((I.reconstruct(mem) - q.astype(np.float64)) ** 2).sum(1)
            np.testing.assert_allclose(got, want, rtol=1e-10)


# ------------------------------------------------------- P2: brute-force equivalence

@pytest.mark.parametrize("fp64", [True, False])
def test_full_probe_exact_codebook_equals_bruteforce(fp64):
    """nprobe = nlist, M = D and codebooks holding every residual value make the
    PQ reconstruction exact, so the search is exact kNN (ties by id)."""
    base, ix = int_dataset()
    I = _index(ix)
    r = np.random.Generator(np.random.PCG64(11))
    Q = r.integers(0, 16, size=(20, base.shape[1])).astype(np.float32)
    ids, dists = ivfpq.search(I, Q, nprobe=I.nlist, k=7, fp64=fp64)
    bi, bd = ivfpq.knn_bruteforce(base, Q, 7)
    np.testing.assert_array_equal(ids, bi)
    np.testing.assert_array_equal(np.asarray(dists, np.float64), bd)


def test_exact_operand_mode_fp32_rules_equal_fp64():
    """On small-integer operands every FP32 operation is exact, so the FP32
    rules must give the FP64 definitions exactly (catches a wrong formula in
    either family)."""
    base, ix = int_dataset(dim=16, nlist=6)
    I = _index(ix)
    r = np.random.Generator(np.random.PCG64(3))
    Q = r.integers(0, 16, size=(10, 16)).astype(np.float32)
    D32 = ivfpq.coarse_d2_fp32(Q, I.centroids)
    np.testing.assert_array_equal(D32, ivfpq.coarse_d2_fp64(Q, I.centroids))
    for l in range(I.nlist):
        T32 = ivfpq.lut_fp32(Q[0], I.centroids[l], I.books)
        np.testing.assert_array_equal(T32.astype(np.float64),
                                      ivfpq.lut_shift_fp64(Q[0], I.centroids[l], I.books))
        T64 = ivfpq.lut_fp64(Q[0], I.centroids[l], I.books)
        cd = I.codes[I.members[l]]
        np.testing.assert_array_equal(ivfpq.adc_fp32(T32, cd, D32[0, l]).astype(np.float64),
                                      ivfpq.adc_fp64(T64, cd))


def test_fp32_rules_within_rounding_bound(small_a):
    """On general float data the FP32 rules stay within their forward error
    bound of the FP64 definitions: |fl32 sum - sum| <= n u sum + O(u^2) for n
    non-negative terms (u = 2^-24), plus the rounding of the inputs."""
    d, ix = small_a
    I = _index(ix)
    Q = d["queries"][:6]
    u = 2.0 ** -24
    D32 = ivfpq.coarse_d2_fp32(Q, I.centroids).astype(np.float64)
    D64 = ivfpq.coarse_d2_fp64(Q, I.centroids)
    assert np.all(np.abs(D32 - D64) <= (I.dim + 2) * u * D64 * 1.01)
    for qi in range(3):
        q, c = Q[qi].astype(np.float64), I.centroids[qi].astype(np.float64)
        T32 = ivfpq.lut_fp32(Q[qi], I.centroids[qi], I.books).astype(np.float64)
        T64 = ivfpq.lut_shift_fp64(Q[qi], I.centroids[qi], I.books)
        # each inner product of the decomposed rule is within (dsub+1) u of its
        # absolute sum; the final sum and subtraction add two more roundings
        y = I.books.astype(np.float64)
        qm, cm = q.reshape(I.M, 1, I.dsub), c.reshape(I.M, 1, I.dsub)
        s_abs = (y * y).sum(-1) + 2 * np.abs(cm * y).sum(-1) + 2 * np.abs(qm * y).sum(-1)
        assert np.all(np.abs(T32 - T64) <= (I.dsub + 3) * u * s_abs * 1.01)


@pytest.mark.parametrize("key,M", [("A", 16), ("B", 32), ("C", 48)])
def test_fp32_lut_per_element_tolerance(key, M):
    """Each entry of the FP32 table (the decomposed rule) is within
    1e-5 (T64 + mean T64) of the FP64 definition, T64 the unshifted entry
    ||r_m - y||^2 and mean T64 the pair table's mean entry: relative 1e-5 with
    an absolute floor of 1e-5 of the table's scale, per element, on data
    shaped like the Gaussian-mixture, SIFT-shaped (integer, uncentred) and
    Deep-shaped (normalised) workloads."""
    from workloads import make_dataset, train_ivfpq
    d = make_dataset(key, n=6000, nq=3, ncomp=32)
    I = _index(train_ivfpq(d["base"], 12, M, seed=1, device="cpu"))
    worst = 0.0
    for q in d["queries"]:
        for l in range(I.nlist):
            T32 = ivfpq.lut_fp32(q, I.centroids[l], I.books).astype(np.float64)
            Ts = ivfpq.lut_shift_fp64(q, I.centroids[l], I.books)
            T64 = ivfpq.lut_fp64(q, I.centroids[l], I.books)
            worst = max(worst, float((np.abs(T32 - Ts) / (T64 + T64.mean())).max()))
    assert worst <= 1e-5


# ------------------------------------------------------------ P3: integer exactness

def test_quantiser_hand_worked():
    """A hand-worked case of the quantiser reading: T = [[1,2,4],[3,3,5]], b = 4
    gives bias [1,3], range 3, step 0.2, multiplier 5, t = [[0,5,15],[0,0,10]],
    offset 4; codes (2,2) give S = 25 and 0.2*25 + 4 = 9 = 4 + 5."""
    T = np.array([[1, 2, 4], [3, 3, 5]], dtype=np.float32)
    qz = ivfpq.quantize_lut(T, 4)
    np.testing.assert_array_equal(qz["bias"], [1, 3])
    assert qz["range"] == 3 and qz["delta64"] == 0.2 and qz["s32"] == 5
    np.testing.assert_array_equal(qz["t"], [[0, 5, 15], [0, 0, 10]])
    assert qz["B64"] == 4.0
    S = ivfpq.adc_int(qz["t"], np.array([[2, 2]]))
    assert S[0] == 25
    assert ivfpq.dequant32(S, qz["delta32"], qz["B32"])[0] == np.float32(9.0)


def test_nearest_f32_is_ieee_rounding():
    """nearest_f32 of a value that FP64 holds exactly equals numpy's IEEE
    FP64 -> FP32 conversion (one round-to-nearest-even), over random values of
    every magnitude, halfway cases and the overflow threshold."""
    from fractions import Fraction
    r = np.random.Generator(np.random.PCG64(12))
    x = r.standard_normal(3000) * 2.0 ** r.integers(-140, 120, size=3000)
    for v in x:
        assert ivfpq.nearest_f32(Fraction(float(v))).tobytes() == np.float32(v).tobytes()
    one = Fraction(1)
    assert ivfpq.nearest_f32(one + Fraction(1, 2 ** 24)) == np.float32(1.0)           # tie -> even
    assert ivfpq.nearest_f32(one + Fraction(3, 2 ** 24)) == np.float32(1 + 2.0 ** -22)  # tie -> even
    fmax = Fraction(float(np.finfo(np.float32).max))
    assert ivfpq.nearest_f32(fmax + Fraction(2) ** 103 - 1) == np.finfo(np.float32).max
    assert ivfpq.nearest_f32(fmax + Fraction(2) ** 103) == np.float32(np.inf)


def test_offset_is_the_exact_sum_rounded_once():
    """The offset is the exact sum of the coarse distance and the biases,
    rounded once to FP32 (ties to even), whatever the order of the terms:
    1 + 2^-24 is a tie (-> 1); adding 2^-60 puts it above the tie (-> 1 + 2^-23),
    which a sum first rounded to FP64 would miss (double rounding);
    1e30 + 1 - 1e30 = 1, which any running FP32 or FP64 sum gets wrong;
    two smallest subnormals sum to the next one."""
    import math
    f = np.float32
    assert ivfpq.exact_sum_f32([f(1), f(2.0 ** -24)]) == f(1)
    assert ivfpq.exact_sum_f32([f(1), f(2.0 ** -24), f(2.0 ** -60)]) == f(1 + 2.0 ** -23)
    assert f(math.fsum([1.0, 2.0 ** -24, 2.0 ** -60])) == f(1)     # the double-rounding trap
    assert ivfpq.exact_sum_f32([f(1e30), f(1), f(-1e30)]) == f(1)
    assert ivfpq.exact_sum_f32([f(2.0 ** -149), f(2.0 ** -149)]) == f(2.0 ** -148)
    assert ivfpq.exact_sum_f32([f(-3), f(3)]) == 0
    r = np.random.Generator(np.random.PCG64(14))
    for _ in range(20):
        v = (r.standard_normal(129) * 10.0 ** r.integers(-30, 30, size=129)).astype(np.float32)
        want = ivfpq.exact_sum_f32(v)
        assert ivfpq.exact_sum_f32(v[r.permutation(len(v))]).tobytes() == want.tobytes()
        # dyadic values of 2^-20 resolution below 2^30: math.fsum is exact in
        # FP64, so one conversion to FP32 is the single rounding
        w = (r.integers(-2 ** 30, 2 ** 30, size=129) * 2.0 ** -20).astype(np.float32)
        assert ivfpq.exact_sum_f32(w) == np.float32(math.fsum(float(x) for x in w))
    qz = ivfpq.quantize_lut(np.array([[1, 2], [2.0 ** -24, 3]], dtype=np.float32), 8, d2=0.0)
    assert qz["B32"] == f(1) and qz["B_exact"] == 1 + __import__("fractions").Fraction(1, 2 ** 24)


def test_single_rounding_of_fp32_scale():
    """s = fl32(fl64(L) / fl64(range)) equals the correctly rounded FP32
    quotient (double rounding through FP64 is innocuous for division since
    53 >= 2*24 + 2); checked against exact rational arithmetic."""
    from fractions import Fraction
    r = np.random.Generator(np.random.PCG64(13))
    for rng in r.uniform(1e-3, 1e6, size=2000).astype(np.float32):
        for L in (15, 63, 255, 4095, 65535):
            s = np.float32(np.float64(L) / np.float64(rng))
            q = Fraction(L) / Fraction(float(rng))
            lo = Fraction(float(np.nextafter(s, np.float32(0))))
            hi = Fraction(float(np.nextafter(s, np.float32(np.inf))))
            sv = Fraction(float(s))
            assert abs(sv - q) <= abs(lo - q) and abs(sv - q) <= abs(hi - q)


def test_quantiser_range_zero():
    """A constant table has range 0: every level is 0, step 0, estimate = offset."""
    T = np.full((4, 256), 2.5, dtype=np.float32)
    qz = ivfpq.quantize_lut(T, 8)
    assert np.all(qz["t"] == 0) and qz["delta64"] == 0 and qz["B64"] == 10.0
    assert ivfpq.dequant32(np.array([0]), qz["delta32"], qz["B32"])[0] == np.float32(10.0)


@pytest.mark.parametrize("b", ivfpq.BITS)
def test_quantised_distance_error_bound(small_a, b):
    """S is an exact integer sum of levels in [0, 2^b-1]; the FP64 estimate
    Delta*S + B is within M*Delta/2 (+ the FP32 rounding of T - bias and of the
    product) of sum_m T[m][code_m]; each sub-table has level 0 at its minimum
    and the table's largest entry maps to 2^b-1."""
    d, ix = small_a
    I = _index(ix)
    q = d["queries"][1]
    u = 2.0 ** -24
    for l in (0, 5, 9):
        T32 = ivfpq.lut_fp32(q, I.centroids[l], I.books)
        qz = ivfpq.quantize_lut(T32, b)
        t = qz["t"]
        assert t.min() == 0 and t.max() == qz["L"] and np.all(t.min(axis=1) == 0)
        cd = I.codes[I.members[l]]
        S = ivfpq.adc_int(t, cd)
        # brute force: Python ints
        for row in range(0, len(cd), 37):
            assert int(S[row]) == sum(int(t[m][int(cd[row, m])]) for m in range(I.M))
        exact = ivfpq.adc_fp64(T32.astype(np.float64), cd)
        est = qz["delta64"] * S.astype(np.float64) + qz["B64"]
        rng = float(qz["range"])
        bound = I.M * qz["delta64"] / 2 + I.M * rng * 4 * u + I.M * np.abs(T32).max() * u
        assert np.all(np.abs(est - exact) <= bound)


# ------------------------------------------------- P4: 16 bits ~ plain FP32 recall

def test_sixteen_bits_differs_only_near_the_boundary(small_a):
    """At 16 bits the estimate is within M*Delta/2 (+ rounding) of the FP32 ADC
    distance, so the top-k may change only among candidates whose FP32
    distance is within twice that bound of the k-th; recall stays within one
    point of the plain search."""
    d, ix = small_a
    I = _index(ix)
    Q = d["queries"]
    k, npb = 10, 4
    gt, _ = ivfpq.knn_bruteforce(d["base"], Q, k)
    i32, d32, probes, _ = ivfpq.search(I, Q, npb, k + 40, return_probes=True)
    i16, _ = ivfpq.search(I, Q, npb, k, bits=16)
    for qi in range(len(Q)):
        a, b = set(i32[qi, :k].tolist()), set(i16[qi].tolist())
        if a == b:
            continue
        bound = 0.0
        for l in probes[qi]:
            qz = ivfpq.quantize_lut(ivfpq.lut_fp32(Q[qi], I.centroids[l], I.books), 16)
            bound = max(bound, I.M * qz["delta64"] / 2 * 1.01 + 1e-6 * float(d32[qi, k - 1]))
        dk = float(d32[qi, k - 1])
        pos = {int(x): float(v) for x, v in zip(i32[qi], d32[qi])}
        for x in a ^ b:
            assert abs(pos[int(x)] - dk) <= 2 * bound + 1e-9

    def rec(f):
        return np.mean([len(set(x) & set(y)) / k for x, y in zip(f[:, :k], gt)])

    assert abs(rec(i32) - rec(i16)) <= 0.01


# --------------------------------------------------- P5: CL and TS are a stable sort

def test_locate_and_topk_equal_python_sort():
    r = np.random.Generator(np.random.PCG64(5))
    d = r.integers(0, 6, size=(3, 40)).astype(np.float32)     # many ties
    probes, pd = ivfpq.locate(d, 9)
    for i in range(3):
        want = sorted(range(40), key=lambda l: (float(d[i, l]), l))[:9]
        assert list(probes[i]) == want
    ids = r.permutation(1000)[:40].astype(np.int64)
    ti, td = ivfpq.topk(d[0], ids, 50)
    want = sorted(zip(d[0].tolist(), ids.tolist()))
    assert [int(x) for x in ti[:40]] == [w[1] for w in want]
    assert np.all(ti[40:] == -1) and np.all(np.isinf(td[40:]))


# ------------------------------------------------------------ P6: label invariant

def test_label_bits_keep_the_topk_set(small_a):
    """Quantising every probed list at its label keeps the FP32 top-k set."""
    d, ix = small_a
    I = _index(ix)
    Q = d["queries"][:8]
    k, npb = 10, 4
    lab = predictor.labels(I, Q, npb, k)
    assert lab.shape == (8, npb)
    i32, _ = ivfpq.search(I, Q, npb, k)
    bits = np.where(lab == 0, 0, lab)
    iq, _ = ivfpq.search(I, Q, npb, k, bits=bits)
    for a, b in zip(i32, iq):
        assert set(a.tolist()) == set(b.tolist())
    assert np.any(lab > 0)


def test_label_is_minimal(small_a):
    """The label is the fewest bits whose worst error beats the margin."""
    d, ix = small_a
    I = _index(ix)
    q = d["queries"][3]
    probes, _ = ivfpq.locate(ivfpq.coarse_d2_fp32(q[None], I.centroids), 4)
    lab, tau, margins, errs = predictor.labels_for_query(I, q, probes[0], 10)
    for j in range(4):
        ok = [b for bi, b in enumerate(ivfpq.BITS) if errs[j, bi] < margins[j]]
        assert lab[j] == (ok[0] if ok else 0)


# ------------------------------------------------------------ P7: MLP backward

def test_mlp_backward_finite_differences():
    p = predictor.init_mlp(3)
    p = {k: v.astype(np.float64) + 0.01 for k, v in p.items()}
    r = np.random.Generator(np.random.PCG64(9))
    X = r.standard_normal((17, 5))
    y = r.integers(0, 5, size=17)
    _, g = predictor.loss_and_grad64(p, X, y)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = predictor.loss_and_grad64(p, X, y)
            flat[idx] = old - h
            lm, _ = predictor.loss_and_grad64(p, X, y)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            ana = g[name].reshape(-1)[idx]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)) + 1e-8, (name, idx, num, ana)


def test_fp16_inference_rule_close_to_fp64():
    p = predictor.init_mlp(1)
    r = np.random.Generator(np.random.PCG64(2))
    X = r.standard_normal((200, 5)).astype(np.float32)
    z16 = predictor.mlp_logits16(predictor.to_fp16(p), X)
    p16 = {k: v.astype(np.float16).astype(np.float64) for k, v in p.items()}
    z64 = predictor.mlp_forward64(p16, X.astype(np.float16).astype(np.float64))["z"]
    # hidden activations are rounded to FP16 (u = 2^-11) twice
    assert np.max(np.abs(z16 - z64)) <= 4 * 2.0 ** -11 * (np.abs(z64).max() + 1)


def test_decide_bits_round_up_and_ties():
    z = np.array([[1, 3, 3, 0, 0], [5, 0, 0, 0, 0], [0, 0, 0, 2.0, 1.9]], dtype=np.float32)
    np.testing.assert_array_equal(predictor.decide_bits(z, 0.0), [6, 4, 12])
    np.testing.assert_array_equal(predictor.decide_bits(z, 0.5), [8, 4, 16])
    # a negative tau rounds down: a width within -tau of the wider ones' best logit
    np.testing.assert_array_equal(predictor.decide_bits(z, -1.5), [6, 4, 12])
    np.testing.assert_array_equal(predictor.decide_bits(z, -2.0), [4, 4, 4])
    np.testing.assert_array_equal(predictor.gpu_width(predictor.decide_bits(z, 0.0)), [8, 4, 0])
    np.testing.assert_array_equal(predictor.gpu_width([4, 6, 8, 12, 16, 0]), [4, 8, 8, 0, 0, 0])


def test_decide_bits_against_brute_force():
    """tau = 0 is the argmax (ties to the narrower width); in general the
    chosen width is the fewest c such that every wider logit is beaten by
    tau by some logit at or below c (checked pair by pair); the width never
    shrinks as tau grows."""
    r = np.random.Generator(np.random.PCG64(5))
    z = r.integers(-3, 4, size=(400, 5)).astype(np.float32) * np.float32(0.5)
    z[:200] += r.standard_normal((200, 5)).astype(np.float32)
    am = np.argmax(z, axis=1)
    np.testing.assert_array_equal(predictor.decide_bits(z, 0.0), np.asarray(predictor.BITS)[am])
    prev = None
    for tau in (-np.inf, -3.0, -1.0, -0.25, 0.0, 0.25, 0.5, 1.0, 3.0, np.inf):
        got = predictor.decide_bits(z, tau)
        want = []
        for row in z:
            pick = 16
            for c in range(4):
                if all(any(np.float32(row[i2] - row[i]) >= np.float32(tau) for i2 in range(c + 1))
                       for i in range(c + 1, 5)):
                    pick = predictor.BITS[c]
                    break
            want.append(pick)
        np.testing.assert_array_equal(got, want)
        if prev is not None:
            assert np.all(got >= prev)
        prev = got
    assert np.all(prev == 16)


# ------------------------------------------------------- P8: Eq. 1 / Eq. 2 features

def test_eq1_eq2_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "eq2_worked.txt"))
    d, r1, r2, f, holds = rows.T
    np.testing.assert_array_equal(predictor.eq2(d, r1, r2), f)
    np.testing.assert_array_equal(predictor.eq1_bound_holds(d, r1, r2), holds.astype(bool))
    np.testing.assert_array_equal(predictor.eq2_fp32(d, r1, r2), f.astype(np.float32))
    same = r1 == r2
    np.testing.assert_array_equal((d[same] / r1[same]) > 4, holds[same].astype(bool))


def test_features_from_definitions(small_a):
    d, ix = small_a
    I = _index(ix)
    Q = d["queries"][:3]
    D2 = ivfpq.coarse_d2_fp32(Q, I.centroids)
    probes, pd = ivfpq.locate(D2, 5)
    F = predictor.features(pd, probes, I.radius, I.sizes)
    for i in range(3):
        for j in range(5):
            l0, lj = probes[i, 0], probes[i, j]
            assert F[i, j, 0] == np.float32(np.sqrt(np.float32(D2[i, lj])) - np.sqrt(np.float32(D2[i, l0])))
            assert F[i, j, 1] == np.float32(I.radius[l0]) and F[i, j, 2] == np.float32(I.radius[lj])
            assert F[i, j, 3] == np.float32(np.sqrt(np.float32(I.sizes[lj])))
            assert F[i, j, 4] == np.float32(j / 5)
    assert np.all(F[:, 0, 0] == 0) and np.all(F[:, 1:, 0] >= 0)


def test_radius_is_covering_radius(small_a):
    d, ix = small_a
    I = _index(ix)
    for l in range(I.nlist):
        xh = I.reconstruct(I.members[l])
        r = np.sqrt(((xh - I.centroids[l].astype(np.float64)) ** 2).sum(1)).max()
        assert abs(r - I.radius[l]) <= 1e-12 * max(1.0, r)


def test_eq2_bits_monotone():
    F = np.zeros((1, 6, 5), dtype=np.float32)
    F[0, :, 0] = [0, 1, 3, 4, 8, 16]   # f = [-2.5, -1.5, 0.5, 1.5, 5.5, 13.5]
    F[0, :, 1] = 0.5
    F[0, :, 2] = 1.0
    b = predictor.eq2_bits(F, (8.0, 4.0, 1.0, 0.0))
    np.testing.assert_array_equal(b[0], [16, 16, 12, 8, 6, 4])


# ------------------------------------------- planted mistakes must fail a pin

def test_planted_mistakes_are_caught(small_a, monkeypatch):
    """Plant plausible mistakes in the oracle and check that a pin catches each."""
    d, ix = small_a
    I = _index(ix)
    q = d["queries"][0]
    l = 2
    mem = I.members[l]
    xh = I.reconstruct(mem)
    want = ((xh - q.astype(np.float64)) ** 2).sum(1)

    # (a) residual sign flipped
    T = ivfpq.lut_fp64(-q + 2 * I.centroids[l], I.centroids[l], I.books)
    assert not np.allclose(ivfpq.adc_fp64(T, I.codes[mem]), want, rtol=1e-9)
    # (b) sub-tables transposed (code of sub-space m looked up in table m+1)
    T = ivfpq.lut_fp64(q, I.centroids[l], I.books)
    assert not np.allclose(ivfpq.adc_fp64(np.roll(T, 1, axis=0), I.codes[mem]), want, rtol=1e-9)
    # (c) quantiser that drops the bias
    T32 = ivfpq.lut_fp32(q, I.centroids[l], I.books)
    qz = ivfpq.quantize_lut(T32, 8)
    cd = I.codes[mem]
    est_bad = qz["delta64"] * ivfpq.adc_int(qz["t"], cd)
    assert np.max(np.abs(est_bad - ivfpq.adc_fp64(T32, cd))) > I.M * qz["delta64"] / 2
    # (d) floor instead of round-to-nearest breaks the M*Delta/2 bound somewhere
    Tp = (T32 - qz["bias"][:, None]).astype(np.float32)
    t_floor = np.floor((Tp * qz["s32"]).astype(np.float32)).astype(np.int64)
    S = ivfpq.adc_int(t_floor, cd)
    err = np.abs(qz["delta64"] * S + qz["B64"] - ivfpq.adc_fp64(T32, cd))
    assert np.max(err) > I.M * qz["delta64"] / 2
