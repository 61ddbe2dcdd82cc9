"""Pins of the sub-space precision oracle (oracle/subspace.py): the uint8
map and the bit truncation by hand, Eq. 2 at the sub-space level by hand,
covering radii, and the integer distances against brute force."""
import numpy as np
import pytest

from oracle import ivfpq, subspace

INF3 = (np.inf, np.inf, np.inf)


def test_uint8_map_and_truncation_by_hand():
    lo, inv = subspace.fixed_point(0.0, 255.0)
    assert lo == 0 and inv == 1
    np.testing.assert_array_equal(subspace.to_u8(np.array([-3, 0.5, 1.5, 2.5, 254.6, 300], np.float32), lo, inv),
                                  [0, 0, 2, 2, 255, 255])                  # half to even, clamped
    assert subspace.keep_bits(np.array([0b10110111]), 4)[0] == 0b10110000
    assert subspace.keep_bits(np.array([0b10110111]), 2)[0] == 0b10000000
    assert subspace.keep_bits(np.array([201]), 8)[0] == 201
    lo, inv = subspace.fixed_point(-1.0, 1.0)
    assert inv == np.float32(127.5)
    assert subspace.to_u8(np.array([0.0], np.float32), lo, inv)[0] == 128   # rint(127.5) -> 128 (even)


def test_sub_bits_eq2_by_hand():
    """Three centres on a line at 0, 10, 40 with radii 1, 2, 3 and the query at 0:
    d = (0, 10, 40); g = (d - d1 - 3 r1 - r_k) / r_k = (-4, (10 - 3 - 2)/2 = 2.5,
    (40 - 3 - 3)/3 = 11.33); with thresholds (10, 2, 1): bits (8, 4, 2)."""
    part = dict(centres=np.array([[0.0], [10.0], [40.0]], np.float32),
                radius=np.array([1.0, 2.0, 3.0], np.float32))
    np.testing.assert_array_equal(subspace.sub_bits(np.array([0.0], np.float32), part, (10, 2, 1)), [8, 4, 2])
    np.testing.assert_array_equal(subspace.sub_bits(np.array([0.0], np.float32), part, (12, 3, 2.4)), [8, 6, 4])
    np.testing.assert_array_equal(subspace.sub_bits(np.array([0.0], np.float32), part, INF3), [8, 8, 8])


def test_partition_radius_and_sizes():
    r = np.random.Generator(np.random.PCG64(3))
    X = r.standard_normal((200, 4)).astype(np.float32)
    p = subspace.partition(X, 9, 3)
    assert p["size"].sum() == 200
    for k in range(9):
        mem = X[p["assign"] == k].astype(np.float64)
        want = np.sqrt(((mem - p["centres"][k]) ** 2).sum(1)).max() if len(mem) else 0.0
        assert p["radius"][k] == np.float32(want)


def _int_case():
    """Integer data in 0..255 (D 16, 16 lists, M 8 of dsub 2) with integer codebooks."""
    r = np.random.Generator(np.random.PCG64(8))
    base = r.integers(0, 256, size=(800, 16)).astype(np.float32)
    cent = base[r.permutation(800)[:16]] + np.float32(0.25)
    list_of = np.argmin(((base[:, None, :] - cent[None]) ** 2).sum(-1), axis=1).astype(np.int32)
    books = np.round(r.uniform(-60, 60, size=(8, 256, 2))).astype(np.float32)
    codes = r.integers(0, 256, size=(800, 8)).astype(np.uint8)
    o = ivfpq.Index(cent, books, codes, list_of)
    Q = r.integers(0, 256, size=(10, 16)).astype(np.float32)
    return o, Q


def test_full_precision_cl_is_the_integer_distance():
    """With every sub-space at 8 bits and integer data in 0..255 (the map is
    the identity on centroids rounded to integers), CL's integer distances
    rank lists exactly as sum (q - rint(c))^2 does."""
    o, Q = _int_case()
    ss = subspace.build(o, 4, 4, 8, 2)
    lo, inv = ss["cl_map"]
    probes, pd, low = subspace.locate(o, ss, Q, 5, INF3)
    assert low == 0.0
    c8 = subspace.to_u8(o.centroids, lo, inv)
    q8 = subspace.to_u8(Q, lo, inv)
    for i in range(len(Q)):
        D = ((q8[i][None, :] - c8) ** 2).sum(1)
        sel = np.lexsort((np.arange(o.nlist), D))[:5]
        assert set(probes[i].tolist()) == set(sel.tolist())
        np.testing.assert_array_equal(pd[i], ivfpq.coarse_d2_fp32(Q[i:i + 1], o.centroids[probes[i]])[0])
        assert np.all(np.diff(pd[i]) >= 0)


def test_full_precision_lc_is_the_uint8_distance_to_the_reconstruction():
    """At 8 bits, S(x) = sum_m ||r8_m - y8_code_m||^2: the vector's distance in the
    uint8 map, summed over sub-spaces (brute force per vector)."""
    o, Q = _int_case()
    ss = subspace.build(o, 4, 4, 8, 2)
    ids, dists, sh = subspace.search(o, ss, Q, 4, 6, INF3, INF3, cl=False, lc=True)
    assert sh["lc_low"] == 0.0
    lo, inv = ss["lc_map"]
    probes, _ = ivfpq.locate(ivfpq.coarse_d2_fp32(Q, o.centroids), 4)
    for i in range(len(Q)):
        keys, allid = [], []
        for l in probes[i]:
            r8 = subspace.to_u8((Q[i] - o.centroids[l]).astype(np.float32), lo, inv).reshape(8, 2)
            for x in o.members[l]:
                y8 = ss["y8"][np.arange(8), o.codes[x].astype(np.int64)]          # [8, 2]
                keys.append(int(((r8 - y8) ** 2).sum()))
                allid.append(int(o.ids[x]))
        sel = np.lexsort((np.array(allid), np.array(keys)))[:6]
        np.testing.assert_array_equal(ids[i], np.array(allid)[sel])
        scale = np.float32(np.float32(1.0) / np.float32(inv * inv))
        np.testing.assert_array_equal(dists[i], (np.array(keys)[sel].astype(np.float32) * scale).astype(np.float32))


def test_truncation_error_bound_and_shares():
    """Keeping b bits moves each coordinate by less than 2^(8-b), so a
    partial distance over w dimensions moves by less than
    w (2 * 255 * 2^(8-b) + 2^(2(8-b))); lower thresholds put more sub-spaces
    below 8 bits."""
    o, Q = _int_case()
    ss = subspace.build(o, 4, 4, 8, 2)
    q8 = subspace.to_u8(Q, *ss["cl_map"])
    for b in (2, 4, 6):
        t = 8 - b
        for l in range(o.nlist):
            full = ((q8[0] - ss["c8"][l]) ** 2).sum()
            cut = ((subspace.keep_bits(q8[0], b) - subspace.keep_bits(ss["c8"][l], b)) ** 2).sum()
            assert abs(int(cut) - int(full)) < 16 * (2 * 255 * 2 ** t + 2 ** (2 * t))
    shares = [subspace.locate(o, ss, Q, 5, th)[2] for th in (INF3, (8, 4, 2), (2, 1, 0.5), (0.5, 0.25, 0.1))]
    assert shares[0] == 0 and all(a <= b for a, b in zip(shares, shares[1:])) and shares[-1] > 0
