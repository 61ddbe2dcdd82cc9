"""Index training on the GPU against the training oracle (centroids,
codebooks, every vector's list and codes, bit for bit), and the save/load
round trip (the loaded index searches exactly like the saved one, with its
MLP predictor and SVR model)."""
import numpy as np
import pytest

from oracle import ivfpq, svr, train

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


@pytest.mark.parametrize("key,n,nlist,M,on_device", [("A", 3000, 8, 16, False), ("B", 2500, 12, 32, True),
                                                     ("C", 2000, 6, 48, False)])
def test_training_equals_the_oracle(amp, key, n, nlist, M, on_device):
    from workloads import make_dataset
    base = make_dataset(key, n=n, nq=1, ncomp=8)["base"]
    kw = dict(iters=3, pq_iters=2, seed=11, per_centroid=40, pq_sample=1500)
    want = train.train(base, nlist, M, **kw)
    g = amp.Index.train(cuda(base) if on_device else base, nlist, M, **kw)
    try:
        ex = g.export()
        np.testing.assert_array_equal(ex["centroids"], want["centroids"])
        np.testing.assert_array_equal(ex["codebooks"], want["codebooks"])
        rows = ex["ids"]                                  # ids are the row indices
        lst = np.repeat(np.arange(nlist), ex["list_len"])
        np.testing.assert_array_equal(np.sort(rows), np.arange(n))
        np.testing.assert_array_equal(lst, want["list_of"][rows])
        np.testing.assert_array_equal(ex["codes"], want["codes"][rows])
        # and the trained index searches like the oracle over the same arrays
        o = ivfpq.Index(want["centroids"], want["codebooks"], want["codes"], want["list_of"])
        Q = make_dataset(key, n=n, nq=12, ncomp=8)["queries"]
        ids, dists = g.search(cuda(Q), 3, 10, amp.policy("fixed", bits=8))
        ri, rd = ivfpq.search(o, Q, 3, 10, bits=8)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        g.close()


def test_training_with_empty_clusters(amp):
    """Duplicate rows make clusters empty: both sides re-seed them the same way."""
    r = np.random.Generator(np.random.PCG64(2))
    base = np.repeat(r.standard_normal((40, 16)).astype(np.float32), 20, axis=0)   # 800 rows, 40 distinct
    base = base[r.permutation(len(base))]
    kw = dict(iters=4, pq_iters=2, seed=5, per_centroid=30, pq_sample=800)
    want = train.train(base, 60, 8, **kw)                  # more clusters than distinct points
    g = amp.Index.train(base, 60, 8, **kw)
    try:
        ex = g.export()
        np.testing.assert_array_equal(ex["centroids"], want["centroids"])
        np.testing.assert_array_equal(ex["codebooks"], want["codebooks"])
    finally:
        g.close()


def test_save_load_round_trip(amp, small_a, tmp_path):
    d, ix = small_a
    r = np.random.Generator(np.random.PCG64(4))
    uid = r.permutation(len(ix["codes"])).astype(np.int64) * 3 + 7
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], ids=uid, device=0)
    Q = cuda(d["queries"])
    try:
        g.train_predictor(Q, 6, 10, amp.train_cfg(epochs=2, batch=64, seed=1))
        sv = r.standard_normal((30, 5)).astype(np.float32)
        g.set_svr(sv, r.standard_normal(30).astype(np.float32), 0.7, np.zeros(5), np.ones(5), 256,
                  1.0 - 2.0 ** -5, np.float32(1.0 / -np.log(1.0 - 2.0 ** -5)))
        path = str(tmp_path / "index.anns")
        g.save(path)
        h = amp.Index.load(path)
        try:
            a, b = g.export(), h.export()
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
            for pol in (amp.policy("plain"), amp.policy("fixed", bits=6), amp.policy("mlp", margin=0.3),
                        amp.policy("svr", margin=0.2, width_map=True)):
                i1, d1 = g.search(Q, 6, 10, pol)
                i2, d2 = h.search(Q, 6, 10, pol)
                np.testing.assert_array_equal(i1.cpu().numpy(), i2.cpu().numpy())
                np.testing.assert_array_equal(d1.cpu().numpy(), d2.cpu().numpy())
            for k, v in g.get_predictor().items():
                np.testing.assert_array_equal(v, h.get_predictor()[k])
        finally:
            h.close()
    finally:
        g.close()
