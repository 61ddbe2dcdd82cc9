"""The paper's sub-space precision granularity on the GPU against the
oracle (oracle/subspace.py): partitions, the probes chosen by the truncated
integer CL, the integer LC + DC results, and the counts of computations below
8 bits, bit for bit."""
import numpy as np
import pytest

from oracle import ivfpq, subspace

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


@pytest.fixture(scope="module", params=[("B", 5000, 32, 32, 4, 8, 16), ("C", 4000, 24, 48, 6, 6, 12)])
def case(amp, request):
    from workloads import make_dataset, train_ivfpq
    key, n, nlist, M, S, K, Klc = request.param
    d = make_dataset(key, n=n, nq=20, ncomp=16)
    ix = train_ivfpq(d["base"], nlist, M, iters=4, seed=1, device="cpu")
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    g.build_subspaces(S, K, Klc, iters=3)
    ss = subspace.build(o, S, K, Klc, 3)
    yield d, g, o, ss
    g.close()


def test_partition_sizes_match(amp, case):
    d, g, o, ss = case
    cl = np.empty(ss["S"] * ss["K"], np.int64)
    lc = np.empty(o.M * ss["K_lc"], np.int64)
    amp.abi.anns_subspace_sizes(g.handle, cl.ctypes.data, lc.ctypes.data)
    np.testing.assert_array_equal(cl, np.concatenate([p["size"] for p in ss["cl"]]))
    np.testing.assert_array_equal(lc, np.concatenate([p["size"] for p in ss["lc"]]))


@pytest.mark.parametrize("cl,lc", [(1, 1), (1, 0), (0, 1)])
@pytest.mark.parametrize("th", [(4.0, 2.0, 1.0), (np.inf, np.inf, np.inf), (-1.0, -2.0, -3.0)])
def test_subspace_search_bit_exact(amp, case, cl, lc, th):
    d, g, o, ss = case
    Q = d["queries"]
    nprobe, k = 6, 10
    ids, dists, low = g.search_subspace(cuda(Q), nprobe, k, th, th, cl=bool(cl), lc=bool(lc))
    torch.cuda.synchronize()
    ri, rd, sh = subspace.search(o, ss, Q, nprobe, k, th, th, cl=bool(cl), lc=bool(lc))
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    low = low.cpu().numpy()
    assert low[0] == round(sh["cl_low"] * len(Q) * o.nlist * ss["S"])
    assert low[1] == round(sh["lc_low"] * len(Q) * nprobe * o.M * 256) or sh["lc_low"] == 0
    if th[0] == np.inf:
        assert low[0] == 0 and low[1] == 0
    elif th[0] == -1.0:
        # every sub-space but the nearest (g = -4) goes below 8 bits
        assert (low[0] > 0) == bool(cl) and (low[1] > 0) == bool(lc)
