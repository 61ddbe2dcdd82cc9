"""CL on the tensor cores (tcgen05 BF16 GEMM + exact re-rank) vs the oracle.

The probed lists and their coarse distances must be identical to the FP32
rule (the re-rank makes the fast path exact); the BF16 distances themselves
must lie within the error bound the re-rank relies on.
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


def _case(key, n, nlist, M, nq, ncomp=16):
    from workloads import make_dataset, train_ivfpq
    d = make_dataset(key, n=n, nq=nq, ncomp=ncomp)
    ix = train_ivfpq(d["base"], nlist, M, iters=4, seed=1, device="cpu")
    return d, ix


@pytest.fixture(scope="module", params=[("A", 4000, 150, 16), ("B", 6000, 300, 32), ("C", 3000, 200, 48),
                                        ("D", 2500, 140, 120)])
def geo(amp, request):
    key, n, nlist, M = request.param
    d, ix = _case(key, n, nlist, M, 200)
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    yield key, d, ix, g, o
    g.close()


def _bound(Q, C, dt):
    """The kernel's per-pair bound, evaluated in FP64 from the same inputs."""
    mu = C.astype(np.float64).mean(axis=0).astype(np.float32)
    qh_ = (Q - mu).astype(np.float32)
    ch_ = (C - mu).astype(np.float32)
    qb = torch.from_numpy(qh_).to(torch.bfloat16).float().numpy().astype(np.float64)
    cb = torch.from_numpy(ch_).to(torch.bfloat16).float().numpy().astype(np.float64)
    qn, cn = (qb ** 2).sum(1), (cb ** 2).sum(1)
    qh = np.linalg.norm(qh_.astype(np.float64), axis=1)
    ch = np.linalg.norm(ch_.astype(np.float64), axis=1)
    qe = np.linalg.norm(qb - qh_, axis=1)
    ce = np.linalg.norm(cb - ch_, axis=1)
    dim = Q.shape[1]
    Dp = (dim + 63) // 64 * 64
    ef = (2 * Dp + 8) * 2.0 ** -24 * (qn[:, None] + cn[None, :])
    dn = qe[:, None] + ce[None, :] + 2.0 ** -23 * (qh[:, None] + ch[None, :])
    sup = np.maximum(dt, 0) + ef
    E = dn * (2 * np.sqrt(sup) + dn)
    return ef + E + (dim + 2) * 2.0 ** -24 * (sup + E)


@pytest.mark.parametrize("nprobe", [1, 7, 40])
def test_bf16_probes_identical_to_fp32_rule(amp, geo, nprobe):
    key, d, ix, g, o = geo
    Q = d["queries"]
    pol = amp.policy("fixed", bits=8, cl="bf16")
    ids, dists = g.search(cuda(Q), nprobe, 10, pol)
    torch.cuda.synchronize()
    probes = g.tap(amp.abi.TAP_PROBES, (len(Q), nprobe), np.int32)
    pd = g.tap(amp.abi.TAP_PROBE_D2, (len(Q), nprobe), np.float32)
    D2 = ivfpq.coarse_d2_fp32(Q, o.centroids)
    rp, rd = ivfpq.locate(D2, nprobe)
    np.testing.assert_array_equal(probes, rp)
    np.testing.assert_array_equal(pd, rd)
    ncand = g.tap(amp.abi.TAP_COARSE_CANDIDATES, (len(Q),), np.int32)
    assert np.all(ncand >= nprobe) and np.all(ncand <= o.nlist)
    # the BF16 tensor-core distances lie within the bound the re-rank uses
    dt = g.tap(amp.abi.TAP_COARSE_APPROX, (len(Q), o.nlist), np.float32).astype(np.float64)
    err = np.abs(dt - D2.astype(np.float64))
    bound = _bound(Q, o.centroids, dt)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and they are BF16-accurate, not merely bounded: relative to the norms
    scale = (np.linalg.norm(Q - o.centroids.mean(0), axis=1)[:, None] +
             np.linalg.norm(o.centroids - o.centroids.mean(0), axis=1)[None, :]) ** 2
    assert np.median(err / scale) < 2.0 ** -8
    ri, rd = ivfpq.search(o, Q, nprobe, 10, bits=8)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    st = np.zeros(1, np.int32)
    amp.abi.anns_debug_tap(g.handle, amp.abi.TAP_STATUS, st.ctypes.data, 4)
    assert st[0] == 0


def test_bf16_uneven_batch_and_graph(amp, geo):
    key, d, ix, g, o = geo
    from workloads import zipf_nprobe
    Q = d["queries"]
    npq = zipf_nprobe(len(Q), 2, lo=1, hi=30)
    npq[::7] = 0
    pol = amp.policy("plain", cl="bf16")
    ids, dists = g.search(cuda(Q), 30, 5, pol, nprobe_per_q=cuda(npq))
    ri, rd = ivfpq.search(o, Q, 30, 5, bits=0, nprobe_per_q=npq)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    graph, gi, gd = g.capture_graph(cuda(Q), 30, 5, pol, nprobe_per_q=cuda(npq))
    try:
        gi.zero_()
        graph.launch()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(gi.cpu().numpy(), ri)
    finally:
        graph.close()


def test_bf16_rejects_bf16_lut(amp, geo):
    key, d, ix, g, o = geo
    p = amp.policy("plain", cl="bf16")
    p.lc_prec = amp.abi.PREC_BF16
    with pytest.raises(amp.abi.AnnsError):
        g.search(cuda(d["queries"][:4]), 4, 5, p)


def test_locate_entry_point(amp, geo):
    key, d, ix, g, o = geo
    Q = d["queries"]
    rp, rd = ivfpq.locate(ivfpq.coarse_d2_fp32(Q, o.centroids), 9)
    for cl in ("fp32", "bf16"):
        p, pd = g.locate(cuda(Q), 9, cl=cl)
        np.testing.assert_array_equal(p.cpu().numpy(), rp)
        np.testing.assert_array_equal(pd.cpu().numpy(), rd)
