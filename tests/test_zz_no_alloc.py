"""The allocation-free coarse stage (anns_locate_static).

Some callers cannot allocate device memory: hosts that forbid allocation after
start-up (cudaMalloc and cudaFree take unbounded time and may synchronise the
device) and plugins whose host application owns every memory pool. This entry
point serves them from a fixed scratch array compiled into the library. Its
results must equal the oracle's probe selection and the probes anns_search
selects (the PROBES / PROBE_D2 taps), on two calls in a row: the second with a
different batch, so stale contents of the shared array would show. A second
index with 64 lists covers probe counts above one warp's width (nprobe 40).
"""
import numpy as np
import pytest

from oracle import ivfpq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check_index(amp, abi, ix, Qnp, cases):
    index = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    try:
        Q = torch.from_numpy(Qnp).to("cuda:0")
        D2 = ivfpq.coarse_d2_fp32(Qnp, ix["centroids"])
        for nq, nprobe in cases:
            q = Q[:nq].contiguous()
            index.search(q, nprobe, 10)
            torch.cuda.synchronize()
            want_p = index.tap(abi.TAP_PROBES, (nq, nprobe), np.int32)
            want_d = index.tap(abi.TAP_PROBE_D2, (nq, nprobe), np.float32)
            rp, rd = ivfpq.locate(D2[:nq], nprobe)
            probes = torch.full((nq, nprobe), -7, dtype=torch.int32, device="cuda:0")
            d2 = torch.full((nq, nprobe), -7.0, dtype=torch.float32, device="cuda:0")
            abi.anns_locate_static(index.handle, q.data_ptr(), nq, nprobe, probes.data_ptr(), d2.data_ptr())
            torch.cuda.synchronize()
            got_p, got_d = probes.cpu().numpy(), d2.cpu().numpy()
            np.testing.assert_array_equal(got_p, rp)
            np.testing.assert_array_equal(got_d, rd)
            np.testing.assert_array_equal(got_p, want_p)
            np.testing.assert_array_equal(got_d, want_d)
        with pytest.raises(amp.AnnsError, match="static scratch"):
            big = abi.STATIC_SCRATCH_FLOATS // index.nlist + 1
            abi.anns_locate_static(index.handle, Q.data_ptr(), big, 4, probes.data_ptr(), d2.data_ptr())
        with pytest.raises(amp.AnnsError, match="static scratch"):
            # nq * nlist would wrap a signed 64-bit product
            abi.anns_locate_static(index.handle, Q.data_ptr(), 2 ** 62, 4, probes.data_ptr(), d2.data_ptr())
    finally:
        index.close()


def test_locate_static_matches_oracle_and_search_probes(small_a):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as amp
    from paper_2606_07156_gb300 import abi
    from workloads import make_dataset, train_ivfpq

    d, ix = small_a
    nq = len(d["queries"])
    _check_index(amp, abi, ix, d["queries"], ((nq, 6), (nq // 2, 3)))
    d64 = make_dataset("A", n=6000, nq=40)
    ix64 = train_ivfpq(d64["base"], 64, 16, iters=3, seed=3, device="cpu")
    _check_index(amp, abi, ix64, d64["queries"], ((40, 40), (17, 33)))
