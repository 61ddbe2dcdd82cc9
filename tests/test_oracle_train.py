"""Pins of the index-training oracle (oracle/train.py) against what the
generator's publication, the definition of k-means and brute force fix."""
import os

import numpy as np

from oracle import ivfpq, train

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_values():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = [train.splitmix64((i + 1) * train.GOLDEN) for i in range(len(want))]
    assert got == want


def test_sample_rows_rate_order_and_determinism():
    n, target = 20000, 3000
    rows = train.sample_rows(n, target, seed=7)
    assert np.all(np.diff(rows) > 0)
    # Bernoulli(p = target / n): within 5 standard deviations
    sd = np.sqrt(n * (target / n) * (1 - target / n))
    assert abs(len(rows) - target) < 5 * sd
    np.testing.assert_array_equal(rows, train.sample_rows(n, target, seed=7))
    assert not np.array_equal(rows, train.sample_rows(n, target, seed=8))
    np.testing.assert_array_equal(train.sample_rows(50, 60, seed=1), np.arange(50))


def test_exact_mean_is_one_rounding_of_the_sum_then_one_division():
    from fractions import Fraction
    r = np.random.Generator(np.random.PCG64(3))
    for _ in range(50):
        v = (r.standard_normal(int(r.integers(1, 40))) * 10.0 ** r.integers(-5, 5)).astype(np.float32)
        s = ivfpq.nearest_f32(sum((Fraction(float(x)) for x in v), Fraction(0)))
        assert train._exact_mean(v) == np.float32(s / np.float32(len(v)))
    # a cancellation that any running FP32 sum would lose
    v = np.array([1e8, 1.0, -1e8, 3.0], np.float32)
    assert train._exact_mean(v) == np.float32(1.0)


def _blobs(k=6, per=40, dim=4, seed=5):
    r = np.random.Generator(np.random.PCG64(seed))
    centres = r.uniform(-50, 50, size=(k, dim))
    # blob-contiguous rows: the initial centroids (rows j * S / k) fall one per blob
    X = np.concatenate([c + r.standard_normal((per, dim)) * 0.1 for c in centres]).astype(np.float32)
    return X, centres


def test_kmeans_recovers_separated_blobs_as_exact_means():
    X, centres = _blobs()
    C = train.kmeans(X, 6, 8)
    a, _ = train.assign(X, C)
    for j in range(6):
        mem = X[a == j]
        assert len(mem) == 40                               # every blob is one cluster
        want = mem.astype(np.float64).mean(0)
        assert np.all(np.abs(C[j] - want) <= 2 * np.abs(want) * 2.0 ** -23 + 1e-30)


def test_kmeans_objective_never_increases():
    r = np.random.Generator(np.random.PCG64(9))
    X = r.standard_normal((300, 6)).astype(np.float32)
    prev = np.inf
    for it in range(1, 7):
        C = train.kmeans(X, 12, it)
        _, d = train.assign(X, C)
        obj = float(np.sum(d, dtype=np.float64))
        assert obj <= prev * (1 + 1e-5)
        prev = obj


def test_assignment_is_the_brute_force_nearest():
    r = np.random.Generator(np.random.PCG64(4))
    X = r.standard_normal((200, 5)).astype(np.float32)
    C = r.standard_normal((17, 5)).astype(np.float32)
    a, d = train.assign(X, C)
    D64 = ((X[:, None, :].astype(np.float64) - C[None].astype(np.float64)) ** 2).sum(-1)
    srt = np.sort(D64, axis=1)
    clear = srt[:, 1] - srt[:, 0] > 1e-4 * srt[:, 1]
    np.testing.assert_array_equal(a[clear], np.argmin(D64, axis=1)[clear])
    # exact ties go to the lower index
    a2, _ = train.assign(np.zeros((1, 5), np.float32), np.ones((3, 5), np.float32))
    assert a2[0] == 0


def test_empty_cluster_takes_the_farthest_point():
    # two identical initial rows: the second centroid gets no member in the
    # first assignment and is re-seeded with the point farthest from its centroid
    X = np.array([[0, 0], [0, 0], [1, 0], [10, 0]], np.float32)
    C = train.kmeans(X, 2, 1)
    # init rows 0 and 2 -> (0,0), (1,0); both have members; use a case that empties
    X2 = np.array([[0, 0], [5, 5], [0, 0], [0, 0.5], [9, 9]], np.float32)
    C2 = train.kmeans(X2, 3, 1)            # init rows 0, 1, 3 -> (0,0), (5,5), (0,0.5)
    assert C.shape == (2, 2) and C2.shape == (3, 2)
    X3 = np.array([[0, 0], [0, 0], [0, 0], [4, 0], [7, 0], [1, 0]], np.float32)
    C3 = train.kmeans(X3, 2, 1)            # init rows 0 and 3 are (0,0) and (4,0)
    a, _ = train.assign(X3, np.array([[0, 0], [4, 0]], np.float32))
    assert set(a.tolist()) == {0, 1}
    X4 = np.array([[0, 0], [3, 0], [0, 0], [0, 0]], np.float32)
    C4 = train.kmeans(X4, 2, 1)            # init rows 0 and 2: both (0,0); cluster 1 is empty
    # cluster 0 = mean of all four = (0.75, 0); cluster 1 = farthest point from its centroid: (3, 0)
    np.testing.assert_array_equal(C4, np.array([[0.75, 0], [3, 0]], np.float32))


def test_encode_is_the_brute_force_nearest_codeword():
    r = np.random.Generator(np.random.PCG64(6))
    base = r.standard_normal((150, 8)).astype(np.float32)
    cent = r.standard_normal((3, 8)).astype(np.float32)
    books = r.standard_normal((4, 256, 2)).astype(np.float32)
    out = train.encode(base, cent, books)
    lst = out["list_of"]
    res = base.astype(np.float64) - cent[lst].astype(np.float64)
    for m in range(4):
        D = ((res[:, None, 2 * m:2 * m + 2] - books[m][None].astype(np.float64)) ** 2).sum(-1)
        srt = np.sort(D, axis=1)
        clear = srt[:, 1] - srt[:, 0] > 1e-4 * (srt[:, 1] + 1e-6)
        np.testing.assert_array_equal(out["codes"][clear, m], np.argmin(D, axis=1)[clear])


def test_train_end_to_end_small():
    from workloads import make_dataset
    d = make_dataset("A", n=3000, nq=1)
    ix = train.train(d["base"], 8, 16, iters=3, pq_iters=2, seed=2, per_centroid=64, pq_sample=2000, ksub=256)
    assert ix["centroids"].shape == (8, 128) and ix["codebooks"].shape == (16, 256, 8)
    assert ix["codes"].shape == (3000, 16) and ix["list_of"].max() < 8
    # the PQ reconstruction is closer than the centroid alone
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    xh = o.reconstruct(np.arange(3000))
    e_pq = ((xh - d["base"]) ** 2).sum(1).mean()
    e_c = ((ix["centroids"][ix["list_of"]] - d["base"]) ** 2).sum(1).mean()
    assert e_pq < 0.5 * e_c
