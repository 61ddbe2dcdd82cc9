"""Host logic of bench.py without a GPU: recall, the margin and Eq. 2
calibrations on the recall budget, and the roofline's algorithmic bytes.

The searches are fakes: each policy returns a fixed result table, so the test
checks which policy the calibration picks, not the library.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeAmp:
    """Stands in for the package: policy() returns its arguments."""

    @staticmethod
    def policy(mode, **kw):
        return (mode, tuple(sorted(kw.items())))


def _gt(nq=40, k=10):
    return np.arange(nq * k, dtype=np.int64).reshape(nq, k)


def _with_hits(gt, hits):
    """Result rows holding the first `hits` ground-truth ids (the rest misses)."""
    out = np.full_like(gt, -5)
    out[:, :hits] = gt[:, :hits]
    return out


def test_recall_counts_ground_truth_hits():
    gt = _gt()
    assert bench.recall(gt, gt, 10) == 1.0
    assert bench.recall(_with_hits(gt, 7), gt, 10) == 0.7
    assert bench.recall(np.full_like(gt, -1), gt, 10) == 0.0


def test_margin_calibration_takes_the_most_aggressive_margin_within_budget():
    gt = _gt()
    # plain recall 1.0; the recall the fake search reaches at each margin
    # (any other margin: 1.0)
    table = {-8.0: 0.97, -6.0: 0.996, -4.0: 0.998}

    def run(Qc, nprobe, pol):
        mode, kw = pol
        if mode == "plain":
            return gt
        keep = table.get(dict(kw)["margin"], 1.0)
        # turn the first (1 - keep) of all result entries into misses
        out = gt.copy()
        nbad = int(round((1.0 - keep) * gt.size))
        out.reshape(-1)[:nbad] = -5
        return out

    m, tried = bench.calibrate_margin(FakeAmp, None, gt, 64, 10, run, budget=0.5)
    # -8 loses 3 points, -6 loses 0.4 (within 0.5): -6 is the most aggressive within budget
    assert m == -6.0
    assert tried[-8.0] > 0.5 >= tried[-6.0]
    # with a budget no margin meets, the calibration gives up (infinite margin: all wide)
    m2, _ = bench.calibrate_margin(FakeAmp, None, gt, 64, 10,
                                   lambda Qc, n, pol: run(Qc, n, pol) if pol[0] == "plain"
                                   else _with_hits(gt, 8), budget=0.5)
    assert m2 == float("inf")


def test_eq2_calibration_on_the_budget():
    gt = _gt()

    def run(Qc, nprobe, pol):
        mode, kw = pol
        if mode == "plain":
            return gt
        t = dict(kw)["thresholds"][3]
        return gt if t >= -4.0 else _with_hits(gt, 5)

    th, tried = bench.calibrate_eq2(FakeAmp, None, gt, 64, 10, run, budget=0.5)
    assert th == (-2.5, -3.0, -3.5, -4.0)
    assert tried[-5.0] == 50.0 and tried[-4.0] == 0.0


def test_pair_bytes_counts_list_sizes_of_probed_pairs():
    class FakeIndex:
        @staticmethod
        def list_sizes():
            return np.array([10, 0, 7, 3], dtype=np.int32)

    probes = np.array([[0, 2, -1], [3, 3, 1]], dtype=np.int32)
    pb = bench.pair_bytes(FakeIndex, probes, 32)
    np.testing.assert_array_equal(pb, [[320, 224, 0], [96, 96, 0]])


def test_oracle_all_cores_equals_in_process_oracle(small_a, tmp_path, monkeypatch):
    """The all-core oracle leg (spawned workers over memory-mapped arrays,
    widths from the oracle's own MLP inference) returns exactly what the
    oracle returns in this process, rows in order."""
    from oracle import ivfpq, predictor
    monkeypatch.setattr(bench, "CACHE", str(tmp_path))
    d, ix = small_a
    W = dict(ix, queries=d["queries"])
    cfg = {"k": 10, "name": "tiny"}
    o = ivfpq.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"])
    D2 = ivfpq.coarse_d2_fp32(d["queries"], o.centroids)
    pr, pd = ivfpq.locate(D2, 6)
    F = predictor.features(pd, pr, o.radius, o.sizes).reshape(-1, 5)
    pred = predictor.init_mlp(4)
    pred["mean"] = F.mean(0).astype(np.float32)
    pred["inv_std"] = (1.0 / (F.std(0) + 1e-3)).astype(np.float32)
    pred["W3"] = (pred["W3"] * 4).astype(np.float32)
    ids, dists, secs = bench.oracle_all_cores(W, cfg, 6, 3, 9, pred, 0.25, 2)
    bits = bench.oracle_mlp_bits(o, d["queries"][3:12], 6, pred, 0.25)
    assert len(np.unique(bits)) >= 2
    ri, rd = ivfpq.search(o, d["queries"][3:12], 6, 10, bits=bits)
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(dists, rd)
    assert secs > 0


def test_search_stages_name_the_kernel_that_ran():
    """The split search's passes, the grouped search's kernels and the other
    searches' single stage each get their own stage names and roofline
    candidates, with every pair's code bytes counted where that pair ran."""
    bits = np.array([[4, 4, 0, 8], [8, 0, 4, 4]], dtype=np.uint8)
    pb = np.array([[10, 20, 30, 40], [50, 60, 70, 80]], dtype=np.int64)
    names, c = bench.search_stages("split", [0.0, 0.1, 0.2, 1.0, 5.0, 0.0, 0.0], bits, pb)
    assert len(names) == 5 and names[3].startswith("split_wide") and names[4].startswith("split_narrow")
    assert [x[3] for x in c] == [30 + 60, 10 + 20 + 40 + 50 + 70 + 80]   # the narrow pass takes rank 0 too
    assert max(c, key=lambda x: x[2])[0].startswith("search_kernel (split search, narrow pass")
    names, c = bench.search_stages("grouped", [0.0, 0.1, 0.2, 1.0, 0.5, 4.0, 0.1], bits, pb)
    assert len(names) == 7 and names[5] == "grouped_kernel_4bit_nibble"
    # query-major pass: rank 0 and the FP32 pairs; byte tables: the 8-bit pair of
    # rank >= 1; nibbles: the 4-bit pairs of rank >= 1
    assert [x[3] for x in c] == [10 + 30 + 50 + 60, 40, 20 + 70 + 80]
    assert max(c, key=lambda x: x[2])[0].startswith("nibble_kernel")
    names, c = bench.search_stages(None, [0.0, 0.1, 0.2, 2.0, 0.0, 0.0, 0.0], bits, pb)
    assert len(c) == 1 and c[0][3] == int(pb.sum()) and c[0][0].startswith("search_kernel (LUT build")
