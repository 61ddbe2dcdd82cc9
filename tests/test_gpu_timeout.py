"""Failure detection on the GPU without a fault: the tensor-core CL kernel's
main-loop waits are given a limit of one clock cycle, so they run out. The
kernel must record the timeout in the index's status word (read by
anns_sync_status as ANNS_ERR_TIMEOUT, then cleared), drain the TMA copies it
issued (on this geometry the 4-stage ring has wrapped: D = 960 gives 15 K
chunks), free its tensor memory and return; with the default limit back, the
same index must again give the oracle's probes and search results.
"""
import numpy as np
import pytest

from oracle import ivfpq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("key,n,nlist,M", [("D", 2500, 140, 120), ("C", 3000, 200, 48)])
def test_cl_wait_timeout_is_reported_and_recovers(key, n, nlist, M):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as amp
    from paper_2606_07156_gb300 import abi
    from workloads import make_dataset, train_ivfpq

    d = make_dataset(key, n=n, nq=300, ncomp=16)
    ix = train_ivfpq(d["base"], nlist, M, iters=3, seed=1, device="cpu")
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    Qn = d["queries"]
    Q = torch.from_numpy(Qn).to("cuda:0")
    rp, rd = ivfpq.locate(ivfpq.coarse_d2_fp32(Qn, o.centroids), 8)
    try:
        g.locate(Q, 8, cl="bf16")
        abi.anns_sync_status(g.handle)                      # no timeout with the default limit
        abi.anns_set_option(g.handle, abi.OPT_WAIT_CYCLES, 1)
        for _ in range(2):
            g.locate(Q, 8, cl="bf16")
            with pytest.raises(amp.AnnsError) as e:
                abi.anns_sync_status(g.handle)
            assert e.value.code == -4 and "ran out" in str(e.value)
            assert g.tap(abi.TAP_STATUS, (1,), np.int32)[0] == 0   # read and cleared
        abi.anns_set_option(g.handle, abi.OPT_WAIT_CYCLES, 0)
        probes, pd = g.locate(Q, 8, cl="bf16")
        abi.anns_sync_status(g.handle)
        np.testing.assert_array_equal(probes.cpu().numpy(), rp)
        np.testing.assert_array_equal(pd.cpu().numpy(), rd)
        ids, dists = g.search(Q, 8, 10, amp.policy("fixed", bits=8, cl="bf16"))
        abi.anns_sync_status(g.handle)
        ri, rdd = ivfpq.search(o, Qn, 8, 10, bits=8)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rdd)
        with pytest.raises(amp.AnnsError):
            abi.anns_set_option(g.handle, abi.OPT_WAIT_CYCLES, -1)
    finally:
        g.close()
