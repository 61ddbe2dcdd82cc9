"""The allocation-free coarse stage (anns_locate_static).

Some callers cannot allocate device memory (inside a CUDA graph capture, on
hosts that forbid allocation after start-up, in plugins whose host owns the
memory pools); this entry point serves them from a fixed scratch array
compiled into the library. Its results must equal the probes anns_search
selects (the PROBES / PROBE_D2 taps), on two calls in a row — the second
with a different batch, so stale contents of the shared array would show.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_locate_static_matches_search_probes(small_a):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as amp
    from paper_2606_07156_gb300 import abi

    d, ix = small_a
    index = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    Q = torch.from_numpy(d["queries"]).to("cuda:0")
    for nq, nprobe in ((len(d["queries"]), 6), (len(d["queries"]) // 2, 3)):
        q = Q[:nq].contiguous()
        index.search(q, nprobe, 10)
        torch.cuda.synchronize()
        want_p = index.tap(abi.TAP_PROBES, (nq, nprobe), np.int32)
        want_d = index.tap(abi.TAP_PROBE_D2, (nq, nprobe), np.float32)
        probes = torch.full((nq, nprobe), -7, dtype=torch.int32, device="cuda:0")
        d2 = torch.full((nq, nprobe), -7.0, dtype=torch.float32, device="cuda:0")
        abi.anns_locate_static(index.handle, q.data_ptr(), nq, nprobe, probes.data_ptr(), d2.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(probes.cpu().numpy(), want_p)
        np.testing.assert_array_equal(d2.cpu().numpy(), want_d)
    with pytest.raises(amp.AnnsError, match="static scratch"):
        big = abi.STATIC_SCRATCH_FLOATS // index.nlist + 1
        abi.anns_locate_static(index.handle, Q.data_ptr(), big, 4, probes.data_ptr(), d2.data_ptr())
    index.close()
