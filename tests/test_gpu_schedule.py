"""Scheduling and batching (LPT query order, CUDA graphs, autotuner) and the
Deep-, GIST- and embedding-shaped index geometries, CUDA path vs the oracle.

Every schedule, kernel and replay must return the oracle's results bit for
bit: the order in which queries run never changes what a query returns.
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
def pair_a(amp, small_a):
    d, ix = small_a
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    yield d, g, o
    g.close()


def _uneven(nq, seed, hi, kchoices):
    from workloads import mixed_k, zipf_nprobe
    return zipf_nprobe(nq, seed, lo=1, hi=hi), mixed_k(nq, seed, choices=kchoices)


@pytest.mark.parametrize("sched", ["natural", "lpt", "auto"])
def test_schedules_bit_exact(amp, pair_a, sched):
    d, g, o = pair_a
    Q = d["queries"]
    npq, kpq = _uneven(len(Q), 3, 12, (1, 10, 40))
    g.set_schedule(sched)
    try:
        for bits in (0, 8):
            pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
            ids, dists = g.search(cuda(Q), 12, 40, pol, nprobe_per_q=cuda(npq), k_per_q=cuda(kpq))
            ri, rd = ivfpq.search(o, Q, 12, 40, bits=bits, nprobe_per_q=npq, k_per_q=kpq)
            np.testing.assert_array_equal(ids.cpu().numpy(), ri)
            np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        g.set_schedule("auto")


def test_graph_replays_with_new_queries(amp, pair_a):
    d, g, o = pair_a
    Q = d["queries"]
    nq = len(Q)
    npq, kpq = _uneven(nq, 5, 10, (1, 10))
    qbuf, nbuf, kbuf = cuda(Q), cuda(npq), cuda(kpq)
    pol = amp.policy("fixed", bits=6)
    g.set_schedule("lpt")
    graph, ids, dists = g.capture_graph(qbuf, 10, 10, pol, nprobe_per_q=nbuf, k_per_q=kbuf)
    try:
        g.set_schedule("auto")
        ri, rd = ivfpq.search(o, Q, 10, 10, bits=6, nprobe_per_q=npq, k_per_q=kpq)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        # an unrelated search on the index (different shape) between replays
        g.search(cuda(Q[:3]), 4, 7)
        r = np.random.Generator(np.random.PCG64(9))
        for rep in range(3):
            Q2 = (Q[r.permutation(nq)] + r.normal(0, 0.01, Q.shape)).astype(np.float32)
            np2 = r.integers(0, 11, nq).astype(np.int32)
            qbuf.copy_(cuda(Q2))
            nbuf.copy_(cuda(np2))
            ids.fill_(-7)
            graph.launch()
            torch.cuda.synchronize()
            ri, rd = ivfpq.search(o, Q2, 10, 10, bits=6, nprobe_per_q=np2, k_per_q=kpq)
            np.testing.assert_array_equal(ids.cpu().numpy(), ri)
            np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        graph.close()


def test_graph_of_the_split_search(amp, pair_a):
    """The split query-major search (wide pairs into a partial top-k, then the
    1..8-bit pairs on byte tables only) captured as one CUDA graph, with mixed
    widths per pair (the explicit policy) and new queries and widths between
    replays: every replay equals the oracle."""
    d, g, o = pair_a
    Q = d["queries"]
    nq = len(Q)
    r = np.random.Generator(np.random.PCG64(21))
    widths = np.array([0, 4, 6, 8, 12, 16], np.uint8)
    qbuf = cuda(Q)
    bbuf = cuda(widths[r.integers(0, len(widths), nq * 9)])
    g.set_kernel("split")
    try:
        graph, ids, dists = g.capture_graph(qbuf, 9, 40, amp.policy("explicit", pair_bits=bbuf))
    finally:
        g.set_kernel("auto")
    try:
        for rep in range(3):
            Q2 = (Q[r.permutation(nq)] + r.normal(0, 0.01, Q.shape)).astype(np.float32)
            b2 = widths[r.integers(0, len(widths), nq * 9)]
            qbuf.copy_(cuda(Q2))
            bbuf.copy_(cuda(b2))
            ids.fill_(-7)
            graph.launch()
            torch.cuda.synchronize()
            ri, rd = ivfpq.search(o, Q2, 9, 40, bits=b2.reshape(nq, 9))
            np.testing.assert_array_equal(ids.cpu().numpy(), ri)
            np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        graph.close()


def test_graph_on_stream_and_list_major(amp, pair_a):
    d, g, o = pair_a
    Q = d["queries"]
    g.set_kernel("lists")
    try:
        graph, ids, dists = g.capture_graph(cuda(Q), 5, 10, amp.policy("plain"))
    finally:
        g.set_kernel("auto")
    try:
        st = torch.cuda.Stream()
        ids.zero_()
        graph.launch(st)
        st.synchronize()
        ri, rd = ivfpq.search(o, Q, 5, 10, bits=0)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        graph.close()


def test_autotune_installs_a_configuration(amp, pair_a):
    d, g, o = pair_a
    Q = d["queries"]
    res = g.autotune(cuda(Q), 8, 10, amp.policy("fixed", bits=8), reps=2)
    kinds = {(kk, s) for kk, s, *_ in res}
    assert (amp.abi.KERNEL_BASIC, amp.abi.SCHED_NATURAL) in kinds
    assert (amp.abi.KERNEL_BASIC, amp.abi.SCHED_LPT) in kinds
    assert all(r[2] > 0 for r in res)
    assert (amp.abi.KERNEL_GROUPED, amp.abi.SCHED_LPT) in kinds
    assert (amp.abi.KERNEL_SPLIT, amp.abi.SCHED_NATURAL) in kinds
    ids, dists = g.search(cuda(Q), 8, 10, amp.policy("fixed", bits=8))
    ri, rd = ivfpq.search(o, Q, 8, 10, bits=8)
    np.testing.assert_array_equal(ids.cpu().numpy(), ri)
    g.set_kernel("auto")
    g.set_schedule("auto")


def test_option_and_argument_errors(amp, pair_a):
    d, g, o = pair_a
    with pytest.raises(amp.abi.AnnsError):
        amp.abi.anns_set_option(g.handle, amp.abi.OPT_SCHEDULE, 7)
    with pytest.raises(amp.abi.AnnsError):
        g.autotune(cuda(d["queries"]), 4, 10, reps=0)
    with pytest.raises(amp.abi.AnnsError):
        g.capture_graph(cuda(d["queries"][:0]), 4, 10)


# ------------------------------------------- index geometries of the workloads

def _geometry_case(key, n, nlist, M, ncomp, nq):
    from workloads import make_dataset, train_ivfpq
    d = make_dataset(key, n=n, nq=nq, ncomp=ncomp)
    ix = train_ivfpq(d["base"], nlist, M, iters=4, seed=1, device="cpu")
    return d, ix


@pytest.mark.parametrize("key,M,nlist,bits_set", [
    ("C", 48, 24, (0, 4, 8, 12)),    # Deep-shaped: D = 96, dsub = 2 (query tables formed in place), Mp = 48
    ("D", 120, 16, (0, 4, 16)),      # GIST-shaped: D = 960, dsub = 8, Mp = 128
    ("E", 96, 16, (0, 6, 8)),        # embedding-shaped: D = 768, dsub = 8, Mp = 96
])
def test_workload_geometries_bit_exact(amp, key, M, nlist, bits_set):
    d, ix = _geometry_case(key, 2500, nlist, M, 16, 10)
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    Q = d["queries"]
    npq, kpq = _uneven(len(Q), 7, 8, (1, 10, 100))
    try:
        for bits in bits_set:
            pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
            for kern in ("auto", "lists", "grouped", "basic", "split"):
                g.set_kernel(kern)
                ids, dists = g.search(cuda(Q), 8, 100, pol, nprobe_per_q=cuda(npq), k_per_q=cuda(kpq))
                ri, rd = ivfpq.search(o, Q, 8, 100, bits=bits, nprobe_per_q=npq, k_per_q=kpq)
                np.testing.assert_array_equal(ids.cpu().numpy(), ri, err_msg=f"{key} {bits} {kern}")
                np.testing.assert_array_equal(dists.cpu().numpy(), rd, err_msg=f"{key} {bits} {kern}")
    finally:
        g.close()


def test_stage_profile_and_launch_count(amp, pair_a):
    """Stage timing splits the grouped search into its query-major pass, the
    grouped kernels and the merge; the library's launch counter sees every
    kernel of a search (5 query-major: CL distances, CL selection, precision
    choice, query tables, search; 11 grouped without nibble packing: the same
    four, pair regrouping (count, offsets, scatter, group table), query-major
    pass, grouped kernel, merge; 16 with it: a second regrouping for the 4-bit
    pairs and the nibble kernel)."""
    d, g, o = pair_a
    Q = cuda(d["queries"])
    abi = amp.abi
    cases = (("basic", "natural", amp.policy("plain"), 5, False, True),
             ("grouped", "auto", amp.policy("fixed", bits=8), 11, True, False),
             ("grouped", "auto", amp.policy("fixed", bits=8), 16, True, True))
    idle = {}
    try:
        for kern, sched, pol, n_launch, grouped, nib in cases:
            g.set_kernel(kern)
            g.set_schedule(sched)
            g.set_nibble(nib)
            g.search(Q, 8, 10, pol)
            torch.cuda.synchronize()
            abi.anns_profile(g.handle, 1)
            before = abi.anns_kernel_launches()
            g.search(Q, 8, 10, pol)
            g.search(Q, 8, 10, pol)
            after = abi.anns_kernel_launches()
            ms, cnt = abi.anns_profile(g.handle, 0)
            assert cnt == 2
            assert after - before == 2 * n_launch, (kern, after - before)
            assert len(ms) == abi.PROFILE_STAGES and all(v >= 0.0 for v in ms)
            assert ms[3] > 0.0
            idle[grouped] = ms[4]
        # stage 4 of the query-major search is two events recorded back to back
        assert idle[True] > 2.0 * idle[False], idle
    finally:
        g.set_kernel("auto")
        g.set_schedule("auto")
        g.set_nibble(True)


@pytest.mark.parametrize("nib", [True, False])
def test_nibble_packing_bit_exact(amp, pair_a, nib):
    """4-bit pairs eight to a word (or four, with the option off) return the
    oracle's results, mixed with 6-bit, 8-bit and wide pairs, uneven nprobe
    and k, and two query chunks."""
    d, g, o = pair_a
    Q = d["queries"]
    nq, nprobe = len(Q), 12
    npq, kpq = _uneven(nq, 17, nprobe, (1, 10, 32))
    r = np.random.Generator(np.random.PCG64(19))
    bits = r.choice(np.array([4, 4, 4, 4, 6, 8, 0, 12], np.uint8), size=(nq, nprobe))
    g.set_kernel("grouped")
    g.set_nibble(nib)
    g.set_qchunk(9)
    try:
        pol = amp.policy("explicit", pair_bits=cuda(bits))
        ids, dists = g.search(cuda(Q), nprobe, 32, pol, nprobe_per_q=cuda(npq), k_per_q=cuda(kpq))
        ri, rd = ivfpq.search(o, Q, nprobe, 32, bits=bits, nprobe_per_q=npq, k_per_q=kpq)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rd)
    finally:
        g.set_kernel("auto")
        g.set_nibble(True)
        g.set_qchunk(0)


@pytest.mark.parametrize("qchunk", [1, 7, 64, 0])
def test_grouped_query_chunks_bit_exact(amp, pair_a, qchunk):
    """The grouped kernel's work order by (query chunk, list): chunks of one
    query, a ragged chunk size, a chunk larger than the batch and the automatic
    choice all return the oracle's results, with uneven nprobe and k and a
    mix of 8-bit, 6-bit and wide tables."""
    d, g, o = pair_a
    Q = d["queries"]
    nq, nprobe = len(Q), 10
    npq, kpq = _uneven(nq, 11, nprobe, (1, 10, 32))
    r = np.random.Generator(np.random.PCG64(13))
    bits = r.choice(np.array([8, 8, 8, 6, 4, 0, 16], np.uint8), size=(nq, nprobe))
    g.set_kernel("grouped")
    g.set_qchunk(qchunk)
    try:
        pol = amp.policy("explicit", pair_bits=cuda(bits))
        ids, dists = g.search(cuda(Q), nprobe, 32, pol, nprobe_per_q=cuda(npq), k_per_q=cuda(kpq))
        ri, rd = ivfpq.search(o, Q, nprobe, 32, bits=bits, nprobe_per_q=npq, k_per_q=kpq)
        np.testing.assert_array_equal(ids.cpu().numpy(), ri)
        np.testing.assert_array_equal(dists.cpu().numpy(), rd)
        graph, gi, gd = g.capture_graph(cuda(Q), nprobe, 32, pol, nprobe_per_q=cuda(npq), k_per_q=cuda(kpq))
        try:
            gi.fill_(-3)
            graph.launch()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(gi.cpu().numpy(), ri)
        finally:
            graph.close()
    finally:
        g.set_kernel("auto")
        g.set_qchunk(0)


def test_qchunk_option_errors(amp, pair_a):
    d, g, o = pair_a
    with pytest.raises(amp.abi.AnnsError):
        amp.abi.anns_set_option(g.handle, amp.abi.OPT_QCHUNK, -1)


def test_wide_ids_with_128_entry_lists(amp, small_a):
    """Ids beyond 32 bits (not ascending in row order) keep the 128-entry
    lists (k > 32) on 64-bit ids; every search kernel still gives the
    oracle's ids and distances, ties broken by the 64-bit id."""
    d, ix = small_a
    n = len(ix["list_of"])
    r = np.random.Generator(np.random.PCG64(5))
    ids = (np.int64(1) << 40) + r.permutation(n).astype(np.int64) * 3
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], ids=ids, device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], ids=ids)
    Q = d["queries"]
    try:
        for bits in (0, 4, 8):
            pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
            ri, rd = ivfpq.search(o, Q, 6, 40, bits=bits)
            for kern in ("basic", "grouped", "split"):
                g.set_kernel(kern)
                gi, gd = g.search(cuda(Q), 6, 40, pol)
                np.testing.assert_array_equal(gi.cpu().numpy(), ri, err_msg=f"{bits} {kern}")
                np.testing.assert_array_equal(gd.cpu().numpy(), rd, err_msg=f"{bits} {kern}")
    finally:
        g.set_kernel("auto")
        g.close()


@pytest.mark.parametrize("M", [4, 8])
def test_split_narrow_pass_few_table_rows(amp, M):
    """The split search's narrow pass with fewer table rows than warps (M = 4:
    warps 4..7 stream no row and rows 4..15 pad the table) and with one row a
    warp (M = 8), under 128-entry and 32-entry warp lists, against the oracle."""
    from workloads import make_dataset, train_ivfpq
    d = make_dataset("A", n=3000, nq=12)
    ix = train_ivfpq(d["base"], 16, M, iters=3, seed=2, device="cpu")
    g = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=0)
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    Q = d["queries"]
    try:
        g.set_kernel("split")
        for bits in (0, 4, 8):
            pol = amp.policy("plain") if bits == 0 else amp.policy("fixed", bits=bits)
            for k in (10, 100):
                ids, dists = g.search(cuda(Q), 6, k, pol)
                ri, rd = ivfpq.search(o, Q, 6, k, bits=bits)
                np.testing.assert_array_equal(ids.cpu().numpy(), ri, err_msg=f"M {M} bits {bits} k {k}")
                np.testing.assert_array_equal(dists.cpu().numpy(), rd, err_msg=f"M {M} bits {bits} k {k}")
    finally:
        g.close()
