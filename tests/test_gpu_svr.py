"""The SVR-RBF policy (Section 3.4) on the GPU against the oracle: the widths
each (query, probe) pair receives from the table-exponential FP32 rule, and
the search results those widths give, bit for bit."""
import numpy as np
import pytest

from oracle import ivfpq, predictor, svr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO = 1.0 - 2.0 ** -5


@pytest.fixture(scope="module")
def amp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("margin,wmap,table_n", [(0.0, False, 1024), (0.6, True, 1024), (-0.4, False, 96)])
def test_svr_policy_bit_exact(amp, small_a, margin, wmap, table_n):
    d, ix = small_a
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    try:
        Q = d["queries"]
        nprobe = 9
        D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
        probes, pd = ivfpq.locate(D2, nprobe)
        F = predictor.features(pd, probes, o.radius, o.sizes).reshape(-1, 5)
        mean = F.mean(0).astype(np.float32)
        inv_std = (1.0 / (F.std(0) + 1e-3)).astype(np.float32)
        Xn = svr.normalise32(F, mean, inv_std)
        # a regression target that depends on the features (distance beyond the
        # nearest list and rank), in the width-index range 0..5
        y = np.clip(1.0 + 3.0 * Xn[:, 0] + 0.5 * Xn[:, 4], 0, 5).astype(np.float64)
        r = np.random.Generator(np.random.PCG64(5))
        take = r.permutation(len(y))[:160]
        m = svr.fit(Xn[take].astype(np.float64), y[take], 1.0, 1.0, 0.1, max_sweeps=50)
        sv, beta = Xn[take], m["beta"].astype(np.float32)
        inv_step = np.float32(1.0 / -np.log(RHO))
        g.set_svr(sv, beta, 1.0, mean, inv_std, table_n, RHO, inv_step)
        ids, dists = g.search(cuda(Q), nprobe, 10, amp.policy("svr", margin=margin, width_map=wmap))
        torch.cuda.synchronize()
        tab = svr.exp_table_geometric(table_n, RHO)
        f = svr.predict32(sv, beta, 1.0, inv_step, tab, Xn)
        bits = svr.widths32(f, margin).reshape(len(Q), nprobe)
        if wmap:
            bits = predictor.gpu_width(bits)
        got = g.tap(amp.abi.TAP_BITS, bits.shape, np.uint8)
        np.testing.assert_array_equal(got, bits)
        assert len(np.unique(bits)) >= 2
        ri, rd = ivfpq.search(o, Q, nprobe, 10, bits=bits)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        g.close()


def test_svr_policy_needs_a_model_and_checks_it(amp, small_a):
    d, ix = small_a
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    try:
        with pytest.raises(amp.AnnsError, match="SVR policy needs"):
            g.search(cuda(d["queries"]), 4, 10, amp.policy("svr"))
        sv = np.zeros((3, 5), np.float32)
        with pytest.raises(amp.AnnsError, match="table_ratio"):
            g.set_svr(sv, np.ones(3), 1.0, np.zeros(5), np.ones(5), 64, 1.5, 1.0)
        with pytest.raises(amp.AnnsError, match="non-finite"):
            g.set_svr(sv, np.array([1.0, np.nan, 0.0]), 1.0, np.zeros(5), np.ones(5), 64, 0.5, 1.0)
    finally:
        g.close()
