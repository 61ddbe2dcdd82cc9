"""The CUDA path against the oracle at the list sizes of the SIFT-shaped
benchmark (about 1000 vectors per list, nprobe 64, hundreds of queries), and
the FP32 tables against their FP64 definition per element on SIFT-shaped and
Deep-shaped data.

At these sizes the grouped kernel runs the way the benchmark runs it: many
groups of four pairs per list, limits that tighten during the scan, a work
order chunked by query, and a query-major pass for the rank-0 and wide pairs.
"""
import numpy as np
import pytest

from oracle import ivfpq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.fixture(scope="module")
def sift_case(amp):
    """SIFT-shaped data (integer 0..255, D 128) with B's list sizes: 128k
    vectors in 128 lists, M 32."""
    from workloads import make_dataset, train_ivfpq
    d = make_dataset("B", n=131072, nq=192, ncomp=256)
    ix = train_ivfpq(d["base"], 128, 32, iters=6, seed=2, device="cuda:0")
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    yield d, ix, g, o
    g.close()


@pytest.mark.parametrize("mode", ["fixed8", "plain", "mixed", "fixed8_qchunk37", "fixed8_k100"])
def test_bench_size_search_bit_exact(amp, sift_case, mode):
    d, ix, g, o = sift_case
    Q = d["queries"]
    nq, nprobe, k = len(Q), 64, (100 if mode.endswith("k100") else 10)
    assert 700 <= np.median(o.sizes) <= 1300
    bits = 8 if mode.startswith("fixed8") else 0
    pol = amp.policy("fixed", bits=8) if bits else amp.policy("plain")
    if mode == "mixed":
        r = np.random.Generator(np.random.PCG64(31))
        bits = r.choice(np.array([8, 8, 8, 6, 4, 0, 12], np.uint8), size=(nq, nprobe))
        pol = amp.policy("explicit", pair_bits=cuda(bits))
    if mode.endswith("qchunk37"):
        g.set_qchunk(37)
    try:
        ids, dists = g.search(cuda(Q), nprobe, k, pol)
    finally:
        g.set_qchunk(0)
    ri, rd = ivfpq.search(o, Q, nprobe, k, bits=bits)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)


@pytest.mark.parametrize("key,M,n", [("B", 32, 20000), ("C", 48, 20000)])
def test_fp32_tables_per_element_against_fp64(amp, key, M, n):
    """Each entry of the GPU's FP32 table is within 1e-5 (T64 + mean T64) of
    the FP64 definition, and the distances of the plain FP32 scan are within
    1e-5 relative of the FP64 ADC distance (plus the coarse distance)."""
    from workloads import make_dataset, train_ivfpq
    d = make_dataset(key, n=n, nq=12, ncomp=64)
    ix = train_ivfpq(d["base"], 24, M, iters=4, seed=1, device="cuda:0")
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    try:
        Q = d["queries"]
        pq = np.repeat(np.arange(len(Q), dtype=np.int32), 4)
        pl = (np.arange(len(pq), dtype=np.int32) * 7) % o.nlist
        pb = np.zeros(len(pq), dtype=np.uint8)
        T, _, _ = g.compute_luts(cuda(Q), cuda(pq), cuda(pl), cuda(pb))
        T = T.cpu().numpy().astype(np.float64)
        for p in range(len(pq)):
            Ts = ivfpq.lut_shift_fp64(Q[pq[p]], o.centroids[pl[p]], o.books)
            T64 = ivfpq.lut_fp64(Q[pq[p]], o.centroids[pl[p]], o.books)
            assert np.all(np.abs(T[p] - Ts) <= 1e-5 * (T64 + T64.mean())), p
        dist, _, off, n_each = g.scan_pairs(cuda(Q), cuda(pq), cuda(pl), cuda(pb))
        dist = dist.cpu().numpy().astype(np.float64)
        for p in range(len(pq)):
            cd = o.codes[o.members[pl[p]]]
            want = ivfpq.adc_fp64(ivfpq.lut_fp64(Q[pq[p]], o.centroids[pl[p]], o.books), cd)
            got = dist[off[p]:off[p] + n_each[p]]
            assert np.all(np.abs(got - want) <= 1e-5 * want), p
    finally:
        g.close()
