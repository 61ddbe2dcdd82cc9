"""CL on the tensor cores (tcgen05 GEMM with BF16, FP16 or FP8 E4M3 operands,
FP32 accumulation, + exact re-rank) vs the oracle.

The probed lists and their coarse distances must be identical to the FP32
rule (the re-rank makes the fast path exact); the tensor-core distances
themselves must lie within the error bound the re-rank relies on.
"""
import numpy as np
import pytest

from oracle import ivfpq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMATS = ("bf16", "fp16", "fp8")
# (torch dtype, top exponent of the per-row scale, K elements per 128-byte chunk, unit roundoff)
FMT = {"bf16": (torch.bfloat16, 14, 64, 2.0 ** -8), "fp16": (torch.float16, 14, 64, 2.0 ** -11),
       "fp8": (torch.float8_e4m3fn, 8, 128, 2.0 ** -4)}


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


def _operand(X, mu, cl):
    """Rows centred, scaled by 2^e (largest magnitude in [2^(top-1), 2^top)),
    rounded to the format by torch and scaled back (FP64), with the centred
    FP32 rows."""
    dtype, top, _, _ = FMT[cl]
    v = (X - mu).astype(np.float32)
    amax = np.abs(v).max(axis=1)
    _, ex = np.frexp(amax)                       # amax = m 2^ex, m in [0.5, 1)
    e = np.where(amax > 0, np.clip(top - ex, -126, 126), 0)
    w = (v * np.exp2(e)[:, None].astype(np.float32)).astype(np.float32)
    r = torch.from_numpy(w).to(dtype).float().numpy().astype(np.float64)
    return r * np.exp2(-e)[:, None], v


def _bound(Q, C, dt, cl):
    """The kernel's per-pair bound, evaluated in FP64 from the same inputs."""
    mu = C.astype(np.float64).mean(axis=0).astype(np.float32)
    qb, qh_ = _operand(Q, mu, cl)
    cb, ch_ = _operand(C, mu, cl)
    qn, cn = (qb ** 2).sum(1), (cb ** 2).sum(1)
    qh = np.linalg.norm(qh_.astype(np.float64), axis=1)
    ch = np.linalg.norm(ch_.astype(np.float64), axis=1)
    qe = np.linalg.norm(qb - qh_, axis=1)
    ce = np.linalg.norm(cb - ch_, axis=1)
    dim = Q.shape[1]
    per = FMT[cl][2]
    Dp = (dim + per - 1) // per * per
    ef = (2 * Dp + 8) * 2.0 ** -24 * (qn[:, None] + cn[None, :])
    dn = qe[:, None] + ce[None, :] + 2.0 ** -23 * (qh[:, None] + ch[None, :])
    sup = np.maximum(dt, 0) + ef
    E = dn * (2 * np.sqrt(sup) + dn)
    return ef + E + (dim + 2) * 2.0 ** -24 * (sup + E)


@pytest.mark.parametrize("cl", FORMATS)
@pytest.mark.parametrize("nprobe", [1, 7, 40])
def test_tc_probes_identical_to_fp32_rule(amp, geo, nprobe, cl):
    key, d, ix, g, o = geo
    Q = d["queries"]
    pol = amp.policy("fixed", bits=8, cl=cl)
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
    # the tensor-core distances lie within the bound the re-rank uses
    dt = g.tap(amp.abi.TAP_COARSE_APPROX, (len(Q), o.nlist), np.float32).astype(np.float64)
    err = np.abs(dt - D2.astype(np.float64))
    bound = _bound(Q, o.centroids, dt, cl)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and they are as accurate as the format, not merely bounded: relative to the norms
    scale = (np.linalg.norm(Q - o.centroids.mean(0), axis=1)[:, None] +
             np.linalg.norm(o.centroids - o.centroids.mean(0), axis=1)[None, :]) ** 2
    assert np.median(err / scale) < FMT[cl][3]
    ri, rd = ivfpq.search(o, Q, nprobe, 10, bits=8)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    st = np.zeros(1, np.int32)
    amp.abi.anns_debug_tap(g.handle, amp.abi.TAP_STATUS, st.ctypes.data, 4)
    assert st[0] == 0


@pytest.mark.parametrize("cl", FORMATS)
def test_tc_uneven_batch_and_graph(amp, geo, cl):
    key, d, ix, g, o = geo
    from workloads import zipf_nprobe
    Q = d["queries"]
    npq = zipf_nprobe(len(Q), 2, lo=1, hi=30)
    npq[::7] = 0
    pol = amp.policy("plain", cl=cl)
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
    for cl in ("fp32",) + FORMATS:
        p, pd = g.locate(cuda(Q), 9, cl=cl)
        np.testing.assert_array_equal(p.cpu().numpy(), rp)
        np.testing.assert_array_equal(pd.cpu().numpy(), rd)


def _random_index(amp, nlist, dim, seed):
    """An index whose centroids are clustered random draws (the coarse stage
    reads only the centroids): lists of one vector each."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(size=(max(nlist // 40, 1), dim)).astype(np.float32) * 3
    C = (centres[rng.integers(0, len(centres), nlist)] + rng.normal(size=(nlist, dim))).astype(np.float32)
    M = 2 if dim % 2 == 0 else 1
    books = rng.normal(size=(M, 256, dim // M)).astype(np.float32)
    codes = rng.integers(0, 256, size=(nlist, M)).astype(np.uint8)
    Q = (centres[rng.integers(0, len(centres), 300)] + rng.normal(size=(300, dim))).astype(np.float32)
    g = amp.Index(C, books, codes, np.arange(nlist, dtype=np.int32), device=0)
    return g, C, Q


@pytest.mark.parametrize("nlist,dim", [(30000, 24), (12000, 24), (700, 18), (900, 37)])
def test_tc_streaming_and_unaligned_rerank(amp, nlist, dim):
    """nlist 30000 leaves the re-rank's keys out of shared memory (the
    streaming re-rank); 12000 keeps them (the select kernel at one block per
    SM); dims 18 and 37 are not multiples of 4 (element-wise row staging).
    Probes and distances must still be the FP32 rule's."""
    g, C, Q = _random_index(amp, nlist, dim, nlist + dim)
    try:
        for nprobe in (1, 33, 100):
            rp, rd = ivfpq.locate(ivfpq.coarse_d2_fp32(Q, C), nprobe)
            for cl in FORMATS:
                p, pd = g.locate(cuda(Q), nprobe, cl=cl)
                np.testing.assert_array_equal(p.cpu().numpy(), rp)
                np.testing.assert_array_equal(pd.cpu().numpy(), rd)
                ncand = g.tap(amp.abi.TAP_COARSE_CANDIDATES, (len(Q),), np.int32)
                assert np.all(ncand >= nprobe) and np.all(ncand <= nlist)
    finally:
        g.close()


def test_tc_candidates_shrink_with_the_format(amp):
    """A finer operand format gives a tighter bound, hence fewer lists to
    re-rank: FP16 (11 significant bits) <= BF16 (8) <= FP8 E4M3 (4)."""
    g, C, Q = _random_index(amp, 4096, 64, 7)
    try:
        mean = {}
        for cl in FORMATS:
            g.locate(cuda(Q), 16, cl=cl)
            mean[cl] = float(g.tap(amp.abi.TAP_COARSE_CANDIDATES, (len(Q),), np.int32).mean())
        assert mean["fp16"] <= mean["bf16"] <= mean["fp8"], mean
    finally:
        g.close()


@pytest.mark.parametrize("nlist,dim,nq", [(333, 4, 1), (257, 8, 129), (1000, 12, 7)])
def test_tc_edge_geometries(amp, nlist, dim, nq):
    """One query, nq not a multiple of the 128-row tile, nlist odd and below one
    256-column tile, dims far below one K chunk (mostly zero padding), nprobe
    from 1 to 128: every format still gives the FP32 rule's probes."""
    g, C, Q = _random_index(amp, nlist, dim, 3 * nlist + dim)
    Q = Q[:nq] if nq <= len(Q) else np.concatenate([Q] * (nq // len(Q) + 1))[:nq]
    try:
        for nprobe in (1, min(nlist, 128)):
            rp, rd = ivfpq.locate(ivfpq.coarse_d2_fp32(Q, C), nprobe)
            for cl in FORMATS:
                p, pd = g.locate(cuda(Q), nprobe, cl=cl)
                np.testing.assert_array_equal(p.cpu().numpy(), rp, err_msg=f"{cl} {nprobe}")
                np.testing.assert_array_equal(pd.cpu().numpy(), rd, err_msg=f"{cl} {nprobe}")
    finally:
        g.close()
