"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Integer results (probed lists, LUT levels, integer sums, returned ids) must be
identical; FP32 results follow the oracle's FP32 rules and must be identical
too; FP32 results are also checked against the FP64 definitions within the
rounding tolerance.
"""
import numpy as np
import pytest

from oracle import ivfpq, predictor
from tests.conftest import int_dataset

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as m
    return m


def _pair(amp, ix, ids=None):
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], ids=ids, device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], ids)
    return g, o


@pytest.fixture(scope="module", params=["basic", "lists", "grouped", "split"])
def case_a(amp, small_a, request):
    """Config A shape, searched by each of the three search kernels."""
    d, ix = small_a
    g, o = _pair(amp, ix)
    g.set_kernel(request.param)
    g.kernel_name = request.param
    yield d, ix, g, o
    g.close()




def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


# ------------------------------------------------------------------ index

def test_index_tables_match(case_a):
    d, ix, g, o = case_a
    np.testing.assert_array_equal(g.list_sizes(), o.sizes)
    np.testing.assert_array_equal(g.list_radius(), o.radius.astype(np.float32))
    want = np.concatenate([o.ids[m] for m in o.members])
    np.testing.assert_array_equal(g.packed_ids(), want)


# ------------------------------------------------------------------ CL

@pytest.mark.parametrize("nprobe", [1, 5, 16])
def test_coarse_probes_bit_exact(amp, case_a, nprobe):
    d, ix, g, o = case_a
    Q = d["queries"]
    g.search(cuda(Q), nprobe, 10)
    torch.cuda.synchronize()
    probes = g.tap(amp.abi.TAP_PROBES, (len(Q), nprobe), np.int32)
    pd = g.tap(amp.abi.TAP_PROBE_D2, (len(Q), nprobe), np.float32)
    D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
    rp, rd = ivfpq.locate(D2, nprobe)
    np.testing.assert_array_equal(probes, rp)
    np.testing.assert_array_equal(pd, rd)
    D64 = ivfpq.coarse_d2_fp64(Q, o.centroids)
    ref = np.take_along_axis(D64, rp.astype(np.int64), axis=1)
    assert np.all(np.abs(pd - ref) <= 1e-5 * ref + 1e-30)


# ------------------------------------------------------------------ LC + quantiser

@pytest.mark.parametrize("bits", [0, 4, 6, 8, 12, 16])
def test_luts_bit_exact(case_a, bits):
    d, ix, g, o = case_a
    Q = d["queries"]
    pq = np.array([0, 1, 2, 3, 5, 7], dtype=np.int32)
    pl = np.array([0, 3, 7, 11, 15, 2], dtype=np.int32)
    pb = np.full(len(pq), bits, dtype=np.uint8)
    T, t, sc = g.compute_luts(cuda(Q), cuda(pq), cuda(pl), cuda(pb))
    T, t, sc = T.cpu().numpy(), t.cpu().numpy().view(np.uint16), sc.cpu().numpy()
    D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
    for p in range(len(pq)):
        T32 = ivfpq.lut_fp32(Q[pq[p]], o.centroids[pl[p]], o.books)
        np.testing.assert_array_equal(T[p], T32)
        # per element: relative 1e-5 with a floor of 1e-5 of the table's mean entry
        Ts = ivfpq.lut_shift_fp64(Q[pq[p]], o.centroids[pl[p]], o.books)
        T64 = ivfpq.lut_fp64(Q[pq[p]], o.centroids[pl[p]], o.books)
        assert np.all(np.abs(T[p] - Ts) <= 1e-5 * (T64 + T64.mean()))
        if bits:
            qz = ivfpq.quantize_lut(T32, bits, D2[pq[p], pl[p]])
            np.testing.assert_array_equal(t[p].astype(np.int64), qz["t"])
            assert sc[p, 0] == qz["delta64"] and sc[p, 1] == float(qz["B32"])
            assert sc[p, 2] == float(qz["range"]) and sc[p, 3] == float(qz["s32"])


# ------------------------------------------------------------------ DC

@pytest.mark.parametrize("bits", [0, 4, 8, 16])
def test_scan_distances_bit_exact(case_a, bits):
    d, ix, g, o = case_a
    Q = d["queries"]
    pq = np.arange(8, dtype=np.int32) % len(Q)
    pl = (np.arange(8, dtype=np.int32) * 5) % o.nlist
    pb = np.full(8, bits, dtype=np.uint8)
    dist, S, off, n_each = g.scan_pairs(cuda(Q), cuda(pq), cuda(pl), cuda(pb))
    dist, S = dist.cpu().numpy(), S.cpu().numpy()
    D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
    for p in range(8):
        cd = o.codes[o.members[pl[p]]]
        T32 = ivfpq.lut_fp32(Q[pq[p]], o.centroids[pl[p]], o.books)
        d2 = D2[pq[p], pl[p]]
        seg = slice(off[p], off[p] + n_each[p])
        if bits == 0:
            np.testing.assert_array_equal(dist[seg], ivfpq.adc_fp32(T32, cd, d2))
        else:
            qz = ivfpq.quantize_lut(T32, bits, d2)
            Sref = ivfpq.adc_int(qz["t"], cd)
            np.testing.assert_array_equal(S[seg].astype(np.int64), Sref)
            np.testing.assert_array_equal(dist[seg], ivfpq.dequant32(Sref, qz["delta32"], qz["B32"]))


# ------------------------------------------------------------------ full search

@pytest.mark.parametrize("bits", [0, 4, 6, 8, 12, 16])
@pytest.mark.parametrize("k", [1, 10, 40])
def test_search_bit_exact(amp, case_a, bits, k):
    d, ix, g, o = case_a
    Q = d["queries"]
    pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
    ids, dists = g.search(cuda(Q), 6, k, pol)
    ri, rd = ivfpq.search(o, Q, 6, k, bits=bits)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)


def test_search_plain_within_fp32_tolerance_of_fp64(case_a):
    d, ix, g, o = case_a
    Q = d["queries"]
    ids, dists = g.search(cuda(Q), 6, 10)
    r64i, r64d = ivfpq.search(o, Q, 6, 10, fp64=True)
    dists = dists.cpu().numpy().astype(np.float64)
    # same candidates up to near-ties; compare each returned id's FP64 distance
    for i in range(len(Q)):
        m = {int(a): b for a, b in zip(r64i[i], r64d[i])}
        for a, b in zip(ids[i].cpu().numpy(), dists[i]):
            if int(a) in m:
                assert abs(b - m[int(a)]) <= 1e-5 * m[int(a)]


def test_search_explicit_mixed_bits(amp, case_a):
    """Per-pair bits mixing FP32 and every width in one batch."""
    d, ix, g, o = case_a
    Q = d["queries"]
    r = np.random.Generator(np.random.PCG64(4))
    bits = r.choice(np.array([0, 4, 6, 8, 12, 16], dtype=np.uint8), size=(len(Q), 7))
    pb = cuda(bits)
    ids, dists = g.search(cuda(Q), 7, 10, amp.policy("explicit", pair_bits=pb))
    ri, rd = ivfpq.search(o, Q, 7, 10, bits=bits)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    np.testing.assert_array_equal(g.tap(amp.abi.TAP_BITS, (len(Q), 7), np.uint8), bits)


def test_search_eq2_policy(amp, case_a):
    d, ix, g, o = case_a
    Q = d["queries"]
    th = (2.0, 1.0, 0.0, -1.0)
    ids, dists = g.search(cuda(Q), 6, 10, amp.policy("eq2", thresholds=th))
    torch.cuda.synchronize()
    D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
    probes, pd = ivfpq.locate(D2, 6)
    F = predictor.features(pd, probes, o.radius, o.sizes)
    np.testing.assert_array_equal(g.tap(amp.abi.TAP_FEATURES, (len(Q), 6, 5), np.float32), F)
    bits = predictor.eq2_bits(F, th)
    np.testing.assert_array_equal(g.tap(amp.abi.TAP_BITS, (len(Q), 6), np.uint8), bits)
    ri, rd = ivfpq.search(o, Q, 6, 10, bits=bits)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)


def test_search_eq2_policy_width_map(amp, case_a):
    d, ix, g, o = case_a
    Q = d["queries"]
    th = (2.0, 1.0, 0.0, -1.0)
    ids, dists = g.search(cuda(Q), 6, 10, amp.policy("eq2", thresholds=th, width_map=True))
    torch.cuda.synchronize()
    D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
    probes, pd = ivfpq.locate(D2, 6)
    bits = predictor.gpu_width(predictor.eq2_bits(predictor.features(pd, probes, o.radius, o.sizes), th))
    np.testing.assert_array_equal(g.tap(amp.abi.TAP_BITS, (len(Q), 6), np.uint8), bits)
    ri, rd = ivfpq.search(o, Q, 6, 10, bits=bits)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)


def test_per_query_nprobe_and_k(amp, case_a):
    d, ix, g, o = case_a
    Q = d["queries"]
    r = np.random.Generator(np.random.PCG64(8))
    npq = r.integers(0, 9, size=len(Q)).astype(np.int32)
    kpq = r.choice(np.array([0, 1, 10, 33], dtype=np.int32), size=len(Q))
    kmax = 33
    ids, dists = g.search(cuda(Q), 8, kmax, amp.policy("fixed", bits=6), nprobe_per_q=cuda(npq),
                          k_per_q=cuda(kpq))
    ri, rd = ivfpq.search(o, Q, 8, kmax, bits=6, nprobe_per_q=npq, k_per_q=kpq)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)


def test_host_buffers_equal_device(amp, case_a):
    d, ix, g, o = case_a
    Q = d["queries"]
    pol = amp.policy("fixed", bits=8)
    di, dd = g.search(cuda(Q), 5, 10, pol)
    hi, hd = g.search_host(torch.from_numpy(Q).pin_memory(), 5, 10, pol)
    np.testing.assert_array_equal(di.cpu().numpy(), hi)
    np.testing.assert_array_equal(dd.cpu().numpy(), hd)


def test_empty_batch(amp, case_a):
    d, ix, g, o = case_a
    ids, dists = g.search(cuda(d["queries"][:0]), 4, 10)
    assert ids.shape == (0, 10)


# ------------------------------------------------------------------ edge cases

def test_ties_broken_by_user_id_and_padding(amp):
    """Integer data: many exactly equal distances; scrambled user ids decide the order.
    Four lists, some tiny, k larger than the candidates of a 1-probe search."""
    base, ix = int_dataset(n=300, dim=8, nlist=4, hi=3)
    r = np.random.Generator(np.random.PCG64(1))
    uids = r.permutation(10_000_000)[:300].astype(np.int64) * 7 + 3
    g, o = _pair(amp, ix, ids=uids)
    Q = r.integers(0, 4, size=(30, 8)).astype(np.float32)
    for kern, npb, k, bits in ((kn, *c) for kn in ("basic", "lists")
                               for c in ((4, 20, 0), (1, 128, 0), (2, 50, 4), (4, 7, 16))):
        g.set_kernel(kern)
        pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
        ids, dists = g.search(cuda(Q), npb, k, pol)
        ri, rd = ivfpq.search(o, Q, npb, k, bits=bits)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    # brute-force equivalence through the GPU (exact codebook, every list probed)
    ids, dists = g.search(cuda(Q), 4, 9)
    bi, bd = ivfpq.knn_bruteforce(base, Q, 9, ids=uids)
    np.testing.assert_array_equal(ids.cpu().numpy(), bi)
    np.testing.assert_array_equal(dists.cpu().numpy().astype(np.float64), bd)
    g.close()


@pytest.mark.parametrize("M,dim", [(24, 96), (120, 120), (8, 64), (48, 96)])
def test_odd_subspace_counts(amp, M, dim):
    """M not a multiple of 16 (padded code rows), M = 120 (8 chunks), dsub 1..8,
    empty lists and ragged last tiles."""
    from workloads.index_train import train_ivfpq
    r = np.random.Generator(np.random.PCG64(M))
    base = r.standard_normal((1500, dim)).astype(np.float32)
    ix = train_ivfpq(base, 12, M, seed=2, device="cpu", iters=3)
    ix["list_of"][ix["list_of"] == 5] = 6                     # list 5 becomes empty
    g, o = _pair(amp, ix)
    Q = r.standard_normal((12, dim)).astype(np.float32)
    for kern in ("basic", "lists"):
        g.set_kernel(kern)
        for bits in (0, 8, 12):
            pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
            ids, dists = g.search(cuda(Q), 7, 12, pol)
            ri, rd = ivfpq.search(o, Q, 7, 12, bits=bits)
            np.testing.assert_array_equal(ids.cpu().numpy(), ri)
            np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    g.close()


def test_invalid_arguments(amp, case_a):
    d, ix, g, o = case_a
    q = cuda(d["queries"])
    with pytest.raises(amp.AnnsError):
        g.search(q, 0, 10)
    with pytest.raises(amp.AnnsError):
        g.search(q, o.nlist + 1, 10)
    with pytest.raises(amp.AnnsError):
        g.search(q, 4, 129)
    with pytest.raises(amp.AnnsError):
        g.search(q, 4, 10, amp.policy("fixed", bits=5))
    with pytest.raises(amp.AnnsError, match="predictor"):
        g.search(q, 4, 10, amp.policy("mlp"))


# ------------------------------------------------------------------ offset rule

def test_exact_sum_rule_matches_oracle(amp):
    """The device rule for the quantiser's offset (exact sum, one rounding)
    equals the oracle's on sets built to break a wrong implementation: ties
    to even, a sum just above a tie that a rounded partial sum would miss,
    cancellation, subnormals, overflow, random magnitudes and bit patterns."""
    f = np.float32
    r = np.random.Generator(np.random.PCG64(21))
    sets = [[f(1), f(2.0 ** -24)], [f(1), f(2.0 ** -24), f(2.0 ** -60)], [f(1 + 2.0 ** -23), f(2.0 ** -24)],
            [f(1e30), f(1), f(-1e30)], [f(2.0 ** -149)] * 2, [f(-3), f(3)], [f(-1), f(2.0 ** -30)],
            [np.finfo(f).max] * 2, [f(-2.0 ** -149)] * 5, []]
    for _ in range(2000):
        n = int(r.integers(1, 130))
        kind = r.integers(0, 3)
        if kind == 0:
            v = (r.standard_normal(n) * 10.0 ** r.integers(-30, 30, size=n)).astype(f)
        elif kind == 1:
            v = r.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32).view(f).copy()
            v[~np.isfinite(v)] = 1
        else:
            b = (r.standard_normal(n) * 1e3).astype(f)
            v = np.concatenate([b, -b[: n // 2]])
            r.shuffle(v)
        sets.append(list(v))
    n = max(len(x) for x in sets)
    vals = np.zeros((len(sets), n), dtype=f)           # zero padding leaves every sum unchanged
    for i, x in enumerate(sets):
        vals[i, :len(x)] = x
    out = torch.empty(len(sets), dtype=torch.float32, device="cuda:0")
    dv = cuda(vals)
    amp.abi.anns_debug_exact_sum(dv.data_ptr(), len(sets), n, out.data_ptr())
    got = out.cpu().numpy()
    want = np.array([ivfpq.exact_sum_f32(x) if x else f(0) for x in sets], dtype=f)
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
