"""Benchmark: QPS of adaptive-precision vs plain-FP32 IVF-PQ search on one GB300.

A step is one batched search (CL -> precision choice -> RC + LC + quantise +
DC + TS) of the whole query batch, queries resident in HBM. The default
workload is the Deep-shaped one (N = 10M, D = 96, nlist = 4096, M = 48, 10k
queries, nprobe 32, k = 10): its codes (480 MB) exceed the 129 MB L2, and L2
is flushed (a 512 MB write) between timed steps as well. ``--config B`` runs
the SIFT-shaped workload (1M, D = 128, nlist = 1024, M = 32, nprobe 64),
whose codes fit in L2.

The headline policy is the learned predictor: trained on the GPU (labels,
features, MLP training) from separate training queries, its round-up margin
calibrated on 2000 held-out calibration queries (exact ground truth) as the
most aggressive margin whose recall@10 stays within half the 1-point loss
budget of plain FP32's. Plain FP32, uniform widths and the Eq. 2 heuristic
(calibrated the same way) are timed beside it; the evaluation queries are
used for neither training nor calibration.

Recall. recall@10 is read as 10-recall@10 (|top-10 found ∩ exact top-10| /
10). On these workloads IVF-PQ's codes bound it below 0.9 at every nprobe of
the sweep, which the line states (``recall_condition``); it also reports a
second operating point at the smallest nprobe whose plain 1-recall@10 (the
exact nearest neighbour among the 10 returned) reaches 0.9.

The CPU oracle leg (rank 0, one GPU) times the oracle single-threaded and on
every host core, compares its sampled results with the GPU's bit for bit
(fixed 8 bits, and the learned policy with the oracle's own inference), and
states the measured error of every float output against FP64.

Default: python bench.py [--gpus 1 --steps K --warmup W]
Reference arm: python bench.py --impl reference (the CPU oracle, a bounded sample).
Under torchrun each rank searches its own replica of the workload (weak
scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

# the CPU oracle runs one BLAS thread per process (single-threaded leg; the
# all-core leg runs one process per core)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CACHE = os.environ.get("ANNS_BENCH_CACHE", os.path.join(tempfile.gettempdir(), "anns_amp_cache"))
METRIC = "QPS at recall@10 >= 0.9 on 1 GB300: adaptive-precision vs plain FP32; scan HBM GB/s % peak"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ workload

NCAL = 2000  # calibration queries (seed offset 300), disjoint from the evaluation queries


def workload(key: str, nq: int | None = None, device=None):
    """Dataset, index arrays, exact ground truth of the evaluation and the
    calibration queries (cached on disk)."""
    from workloads import CONFIGS, exact_knn, make_dataset, make_queries, train_ivfpq
    cfg = CONFIGS[key]
    nq = nq or cfg["nq"]
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, f"{key}_{cfg['n']}_{nq}_cal{NCAL}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return cfg, {k: z[k] for k in z.files}
    t = time.time()
    d = make_dataset(key, nq=nq)
    ix = train_ivfpq(d["base"], cfg["nlist"], cfg["M"], seed=cfg["seed"], device=device)
    gt, _ = exact_knn(d["base"], d["queries"], 100, device=device)
    cal = make_queries(key, NCAL, stream=300)
    cal_gt, _ = exact_knn(d["base"], cal, 100, device=device)
    out = dict(queries=d["queries"], gt=gt, cal_queries=cal, cal_gt=cal_gt, **ix)
    np.savez(path, **out)
    log(f"workload {key}: generated in {time.time() - t:.1f}s")
    return cfg, out


def nn_in_top(found: np.ndarray, gt: np.ndarray, k: int) -> float:
    """Fraction of queries whose exact nearest neighbour is among the first k results."""
    return float(np.mean([g[0] in f[:k] for f, g in zip(found, gt)]))


def recall(found: np.ndarray, gt: np.ndarray, k: int) -> float:
    hits = 0
    for f, g in zip(found[:, :k], gt[:, :k]):
        hits += len(np.intersect1d(f[f >= 0], g))
    return hits / (k * len(found))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.path = gpu, None, None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ------------------------------------------------------------------ GPU arm

def time_steps(fn, steps: int, warmup: int, stream, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 255)
        evs[i][0].record(stream)
        fn()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def max_over_ranks(totals: dict, world: int, device) -> dict:
    """Each timed total (seconds) replaced by its maximum over the ranks (the
    job is as slow as its slowest replica). World 1: unchanged."""
    if world <= 1:
        return dict(totals)
    import torch
    import torch.distributed as dist
    names = sorted(totals)
    tt = torch.tensor([float(totals[n]) for n in names], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return dict(zip(names, tt.tolist()))


def weak_scaling_qps(totals: dict, world: int, nq: int, steps: int) -> dict:
    """Whole-job queries/s: every rank searched nq queries per step."""
    return {name: world * nq * steps / t for name, t in totals.items()}


def nvtx_push(name: str):
    """Marks the timed region for profilers (a no-op where NVTX is unavailable)."""
    import torch
    try:
        torch.cuda.nvtx.range_push(name)
    except (RuntimeError, AttributeError):
        pass


def nvtx_pop():
    import torch
    try:
        torch.cuda.nvtx.range_pop()
    except (RuntimeError, AttributeError):
        pass


def pair_bytes(index, probes: np.ndarray, M: int) -> np.ndarray:
    """Algorithmic bytes per probed (query, list): n_l * M code bytes, one per
    LUT lookup (0 for unused probe slots)."""
    sizes = index.list_sizes().astype(np.int64)
    return np.where(probes >= 0, sizes[np.maximum(probes, 0)], 0) * M


def overlap(a: np.ndarray, b: np.ndarray, k: int) -> float:
    """Mean fraction of the first k ids of b also found in the first k of a."""
    return float(np.mean([len(np.intersect1d(x[:k], y[:k])) / k for x, y in zip(a, b)]))


LOSS_BUDGET = 0.5  # recall@10 points allowed on the calibration queries (half the 1-point target)


SVR_RATIO = 1.0 - 2.0 ** -5   # ratio of the SVR's geometric exponential table (a dyadic number)
SVR_TABLE = 1024              # entries: exp(-t) tabulated up to t = 32.5
WIDTH_INDEX = {4: 0, 6: 1, 8: 2, 12: 3, 16: 4, 0: 5}  # regression target of a label width (0 = FP32)


def fit_svr(amp, abi, index, Qt, nprobe: int, k: int, nsamp: int = 1280, seed: int = 3) -> dict:
    """The SVR-RBF comparator of Section 3.4, fitted as the paper does: at most
    1280 (feature, label) samples drawn from the GPU's training labels, gamma
    = C = 1 (its LC setting), at most 50 sweeps of the library's solver;
    targets = the label width's index in (4, 6, 8, 12, 16, FP32)."""
    import torch
    feat, lab = index.make_training_set(Qt, nprobe, k)
    torch.cuda.synchronize()
    F = feat.reshape(-1, 5).cpu().numpy().astype(np.float32)
    L = lab.reshape(-1).cpu().numpy()
    mean = F.mean(0).astype(np.float32)
    inv_std = (1.0 / np.maximum(F.std(0), 1e-6)).astype(np.float32)
    Xn = ((F - mean).astype(np.float32) * inv_std).astype(np.float32)
    take = np.random.Generator(np.random.PCG64(seed)).permutation(len(L))[:nsamp]
    y = np.array([WIDTH_INDEX[int(b)] for b in L[take]], dtype=np.float64)
    t0 = time.perf_counter()
    beta, sweeps = abi.anns_svr_fit(Xn[take].astype(np.float64), y, 1.0, 1.0, 0.1, 1e-10, 50)
    fit_s = time.perf_counter() - t0
    inv_step = np.float32(1.0 / -np.log(SVR_RATIO))
    # only the support vectors (beta != 0) enter the model: a zero term adds exactly 0
    sv = beta != 0.0
    index.set_svr(Xn[take][sv], beta[sv].astype(np.float32), 1.0, mean, inv_std, SVR_TABLE, SVR_RATIO, inv_step)
    return {"samples": int(len(take)), "gamma": 1.0, "C": 1.0, "eps": 0.1, "sweeps": int(sweeps),
            "fit_s": round(fit_s, 3), "support_vectors": int(np.count_nonzero(beta)),
            "table": f"{SVR_TABLE} entries, ratio 1 - 2^-5"}


def calibrate_svr(amp, Qc, gt_c, nprobe: int, run, budget: float = LOSS_BUDGET):
    """Most aggressive SVR width margin (widths mapped to this GPU's tables)
    within the recall budget on the calibration queries."""
    base = 100.0 * recall(run(Qc, nprobe, amp.policy("plain")), gt_c, 10)
    tried = {}
    for m in (3.0, 2.0, 1.5, 1.0, 0.75, 0.5, 0.25, 0.0, -0.25, -0.5, -1.0, -2.0):
        loss = base - 100.0 * recall(run(Qc, nprobe, amp.policy("svr", margin=m, width_map=True)), gt_c, 10)
        tried[m] = round(loss, 3)
        if loss <= budget:
            return m, tried
    return -8.0, tried


def calibrate_margin(amp, Qc, gt_c, nprobe: int, k: int, run, budget: float = LOSS_BUDGET):
    """Most aggressive MLP round-up margin (widths mapped to this GPU's
    tables) whose recall@10 on the calibration queries is at most `budget`
    points below plain FP32's: the plain search judges the recall loss, on
    queries used neither for training nor for the timed evaluation. Margins
    below 0 favour the narrower width; the grid ends at 16 (nearly all wide)."""
    base = 100.0 * recall(run(Qc, nprobe, amp.policy("plain")), gt_c, 10)
    tried = {}
    for m in (-8.0, -6.0, -4.0, -3.0, -2.0, -1.5, -1.0, -0.75, -0.5, -0.25, 0.0, 0.1, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0,
              3.0, 4.0, 8.0, 16.0):
        loss = base - 100.0 * recall(run(Qc, nprobe, amp.policy("mlp", margin=m, width_map=True)), gt_c, 10)
        tried[m] = round(loss, 3)
        if loss <= budget:
            return m, tried
    return float("inf"), tried


def calibrate_eq2(amp, Qc, gt_c, nprobe: int, k: int, run, budget: float = LOSS_BUDGET):
    """Most aggressive Eq. 2 threshold set th = (t + 1.5, t + 1, t + 0.5, t) for
    4, 6, 8, 12 bits (widths mapped to this GPU's tables) within the same
    recall budget on the calibration queries."""
    base = 100.0 * recall(run(Qc, nprobe, amp.policy("plain")), gt_c, 10)
    best, tried = None, {}
    for t in (-24.0, -16.0, -12.0, -10.0, -8.0, -7.0, -6.0, -5.0, -4.0, -3.5, -3.0, -2.5, -2.0, -1.5, -1.0,
              -0.5, 0.0, 0.5, 1.0, 2.0, 4.0):
        th = (t + 1.5, t + 1.0, t + 0.5, t)
        loss = base - 100.0 * recall(run(Qc, nprobe, amp.policy("eq2", thresholds=th, width_map=True)), gt_c, 10)
        tried[t] = round(loss, 3)
        if loss <= budget:
            best = th
            break
    return best, tried


def bits_mix(index, abi, nq: int, nprobe: int, npq=None) -> dict:
    """Share of the probed pairs on each table width (with per-query nprobe,
    only the pairs each query actually probes)."""
    b = index.tap(abi.TAP_BITS, (nq, nprobe), np.uint8)
    if npq is not None:
        b = b[np.arange(nprobe)[None, :] < np.asarray(npq)[:, None]]
    b = b.reshape(-1)
    return {("fp32" if v == 0 else f"{v}bit"): round(float(np.mean(b == v)), 4) for v in (0, 4, 6, 8, 12, 16)}


def cl_tensor_bench(amp, dev, steps: int, warmup: int, flush) -> dict:
    """The coarse stage alone at the embedding-shaped CL size (20000 queries x
    8192 centroids x D = 768, nprobe 64): the FP32 CUDA-core path vs the
    tcgen05 GEMM with BF16, FP16 or FP8 E4M3 operands + the exact re-rank.
    Centroids are draws of the same mixture as the queries (stand-ins for
    trained centroids; the stage's cost does not depend on the lists'
    contents)."""
    import torch
    from workloads import make_queries
    nq, nlist, dim, M, nprobe = 20000, 8192, 768, 96, 64
    C = make_queries("E", nlist, stream=500)
    Q = torch.from_numpy(make_queries("E", nq, stream=100)).to(dev)
    books = np.zeros((M, 256, dim // M), np.float32)
    codes = np.zeros((nlist, M), np.uint8)
    ix = amp.Index(C, books, codes, np.arange(nlist, dtype=np.int32), device=dev.index)
    st = torch.cuda.current_stream(dev)
    out = {"workload": f"embedding-shaped CL: {nq} queries x {nlist} centroids x D={dim}, nprobe={nprobe}"}
    ref = None
    for cl in ("fp32", "bf16", "fp16", "fp8"):
        res = ix.locate(Q, nprobe, cl=cl, stream=st)
        ms = float(np.median(time_steps(lambda: ix.locate(Q, nprobe, cl=cl, stream=st), steps, warmup, st, flush)))
        torch.cuda.synchronize()
        rec = {"ms": round(ms, 4)}
        if cl == "fp32":
            ref = res
        else:
            rec["identical_probes"] = bool(torch.equal(ref[0], res[0]) and torch.equal(ref[1], res[1]))
            rec["rerank_candidates_mean"] = round(float(ix.tap(amp.abi.TAP_COARSE_CANDIDATES, (nq,),
                                                               np.int32).mean()), 1)
            rec["speedup_vs_fp32"] = round(out["fp32"]["ms"] / ms, 2)
            per = 128 if cl == "fp8" else 64
            rec["gemm_flop"] = 2.0 * nq * nlist * ((dim + per - 1) // per * per)
        out[cl] = rec
    ix.close()
    return out


def pick_cl(index, Q, nprobe: int, stream, reps: int = 5):
    """The faster CL of the adaptive policies on this workload's queries: the
    FP32 CUDA-core rule or the FP16 tensor-core GEMM + exact re-rank (both
    give the same probes and distances, which is checked here). Returns the
    choice and the median times (ms)."""
    import torch
    ref = index.locate(Q, nprobe, cl="fp32", stream=stream)
    got = index.locate(Q, nprobe, cl="fp16", stream=stream)
    torch.cuda.synchronize()
    if not (torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])):
        raise RuntimeError("tensor-core CL differs from the FP32 rule")
    ms = {}
    for cl in ("fp32", "fp16"):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            index.locate(Q, nprobe, cl=cl, stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms[cl] = round(float(np.median(ts)), 4)
    return min(ms, key=ms.get), ms


def calibrate_margin_nn(amp, Qc, gt_c, nprobe: int, run, budget: float = LOSS_BUDGET):
    """calibrate_margin with 1-recall@10 (exact nearest neighbour among the 10
    returned) as the judged recall: the reading of the second operating point."""
    base = 100.0 * nn_in_top(run(Qc, nprobe, amp.policy("plain")), gt_c, 10)
    tried = {}
    for m in (-8.0, -6.0, -4.0, -3.0, -2.0, -1.5, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0):
        loss = base - 100.0 * nn_in_top(run(Qc, nprobe, amp.policy("mlp", margin=m, width_map=True)), gt_c, 10)
        tried[m] = round(loss, 3)
        if loss <= budget:
            return m, tried
    return float("inf"), tried


def roofline_profile(kernel_src: str, workload_name: str, kernel: str):
    """The committed ncu record (profiles/traffic.json) for this kernel, its
    source and the workload: DRAM bytes per launch and the binding unit, or
    None (no record, or the source changed since it was taken)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    recs = json.load(open(path))
    for rec in recs if isinstance(recs, list) else [recs]:
        if (rec.get("source_sha") == sha and rec.get("workload") == workload_name
                and rec.get("kernel", "").split("<")[0] == kernel):
            return rec
    return None


def index_build_bench(amp, dev, key: str, n: int = 1_000_000, nlist: int = 1024) -> dict:
    """Index training on the GPU (anns_train_index: k-means, PQ codebooks,
    encoding, packing) against the PyTorch trainer that builds the
    benchmark's workloads, on n vectors of the workload's distribution; both
    indexes are judged by the recall@10 of a plain search (nprobe 16, 1000
    queries) against exact ground truth."""
    import torch
    from workloads import CONFIGS, exact_knn, make_dataset, train_ivfpq
    cfg = CONFIGS[key]
    d = make_dataset(key, n=n, nq=1000)
    gt, _ = exact_knn(d["base"], d["queries"], 10, device=dev)
    Xd = torch.from_numpy(d["base"]).to(dev)
    Q = torch.from_numpy(d["queries"]).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = amp.Index.train(Xd, nlist, cfg["M"], iters=10, pq_iters=10, seed=1, per_centroid=256, pq_sample=65536,
                        device=dev.index)
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    ids, _ = g.search(Q, 16, 10, amp.policy("plain"))
    rec_gpu = recall(ids.cpu().numpy(), gt, 10)
    g.close()
    t0 = time.perf_counter()
    ix = train_ivfpq(d["base"], nlist, cfg["M"], seed=1, device=dev)
    t_ref = time.perf_counter() - t0
    h = amp.Index(ix["centroids"], ix["codebooks"], ix["codes"], ix["list_of"], device=dev.index)
    ids, _ = h.search(Q, 16, 10, amp.policy("plain"))
    rec_ref = recall(ids.cpu().numpy(), gt, 10)
    h.close()
    return {"workload": f"{cfg['name']} distribution, n={n}, nlist={nlist}, M={cfg['M']}, 10 + 10 iterations",
            "anns_train_index_s": round(t_gpu, 3), "recall_at_10_nprobe16": round(rec_gpu, 4),
            "torch_trainer_s": round(t_ref, 3), "torch_trainer_recall_at_10_nprobe16": round(rec_ref, 4)}


SUBSPACE_TH = (4.0, 2.0, 1.0)   # Eq. 2 thresholds of g for 2, 4 and 6 bits at the sub-space level


def subspace_sweep(amp, index, W, cfg, nprobe: int, k: int, dev, nq: int = 2000) -> dict:
    """The paper's sub-space granularity (Section 5.3, Fig. 13): for a sweep
    of dimension slices S and sub-spaces per slice K, the share of CL partial
    distances computed below 8 bits and the recall@10 of the search whose CL
    runs at sub-space precision (FP32 LUT after it); then LC at sub-space
    precision (codebook-entry groups, integer tables) on the FP32 probes.
    Judged against plain FP32 on the same queries."""
    import torch
    Q = torch.from_numpy(W["queries"][:nq]).to(dev)
    gt = W["gt"][:nq]
    dim, nlist = cfg["dim"], cfg["nlist"]
    ids, _ = index.search(Q, nprobe, k, amp.policy("plain"))
    base = recall(ids.cpu().numpy(), gt, 10)
    slices = [s for s in (1, 2, 4, 8, 16, 32) if dim % s == 0]
    Ks = [kk for kk in (64, 128, 256, 512) if kk <= nlist]
    rows = []

    def one(S, K):
        index.build_subspaces(S, K, 16, iters=10)
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        ids, _, low = index.search_subspace(Q, nprobe, k, SUBSPACE_TH, SUBSPACE_TH, cl=True, lc=False)
        ev[1].record()
        torch.cuda.synchronize()
        low = low.cpu().numpy()
        return {"slices": S, "K": K, "cl_low_share": round(float(low[0]) / (nq * nlist * S), 4),
                "recall_at_10": round(recall(ids.cpu().numpy(), gt, 10), 4),
                "recall_loss_pts": round(100.0 * (base - recall(ids.cpu().numpy(), gt, 10)), 3),
                "ms": round(ev[0].elapsed_time(ev[1]), 3)}

    for S in slices:
        rows.append(one(S, 256 if 256 <= nlist else Ks[-1]))
    S16 = 16 if dim % 16 == 0 else slices[-1]
    for K in Ks:
        if K != 256:
            rows.append(one(S16, K))
    index.build_subspaces(S16, 256 if 256 <= nlist else Ks[-1], 16, iters=10)
    ids, _, low = index.search_subspace(Q, nprobe, k, SUBSPACE_TH, SUBSPACE_TH, cl=False, lc=True)
    torch.cuda.synchronize()
    low = low.cpu().numpy()
    lc_rec = recall(ids.cpu().numpy(), gt, 10)
    ids, _, _ = index.search_subspace(Q, nprobe, k, (np.inf,) * 3, (np.inf,) * 3, cl=False, lc=True)
    lc8_rec = recall(ids.cpu().numpy(), gt, 10)
    return {"queries": nq, "nprobe": nprobe, "thresholds_2_4_6_bits": list(SUBSPACE_TH),
            "plain_fp32_recall_at_10": round(base, 4), "cl": rows,
            "lc": {"K_lc": 16, "low_share": round(float(low[1]) / (nq * nprobe * cfg["M"] * 256), 4),
                   "recall_at_10": round(lc_rec, 4), "recall_at_10_all_8bit": round(lc8_rec, 4),
                   "note": "integer tables of uint8 operands (the codebook's map); all-8-bit is the map's own loss"}}


STAGES_CL = ("cl_distances", "cl_select (the whole tensor-core CL)", "precision_choice+query_tables")


def search_stages(kernel, st_ms, bits: np.ndarray, pb: np.ndarray):
    """Names of the profile stages (anns_profile) for the search that ran, and
    the candidates for the roofline's dominant kernel: (label, source file, ms
    per step, algorithmic code bytes). `kernel` is the autotuner's choice
    ("split", "grouped", ...; None: the automatic one), `st_ms` the stage
    times, `bits` and `pb` the pairs' table widths and code bytes [nq, nprobe].
    The split search runs its wide pairs (stage 3) and then every 1..8-bit pair
    (stage 4); the grouped search runs every rank-0 pair and the wide pairs in
    its query-major pass (stage 3), the other 1..8-bit pairs in the byte-table
    (stage 4) and nibble (stage 5) kernels; the other searches have stage 3
    alone."""
    narrow = (bits >= 1) & (bits <= 8)
    if kernel == "split":
        names = STAGES_CL + ("split_wide_pass (query-major, FP32 tables)",
                             "split_narrow_pass (query-major, 1..8-bit byte tables)")
        return names, [
            ("search_kernel (split search, wide pass: FP32 tables; LUT + scan + top-k)", "search.cu",
             st_ms[3], int(pb[~narrow].sum())),
            ("search_kernel (split search, narrow pass: 1..8-bit byte tables; two-pass build + scan + top-k)",
             "search.cu", st_ms[4], int(pb[narrow].sum()))]
    names = STAGES_CL + ("search_before_grouped (invert + query-major)", "grouped_kernel_5to8bit",
                         "grouped_kernel_4bit_nibble", "grouped_merge")
    if not (st_ms[4] > 0.0 or st_ms[5] > 0.0):
        return names, [("search_kernel (LUT build + quantise + ADC scan + top-k)", "search.cu", st_ms[3],
                        int(pb.sum()))]
    narrow[:, 0] = False
    nib = narrow & (bits <= 4) if st_ms[5] > 0.0 else np.zeros_like(narrow)
    return names, [
        ("search_kernel (query-major pass of the grouped search: rank 0 + wide pairs)", "search.cu",
         st_ms[3], int(pb[~narrow].sum())),
        ("packed_kernel (grouped: four queries' 5..8-bit tables per gather; build + scan + top-k)",
         "search_grouped.cu", st_ms[4], int(pb[narrow & ~nib].sum())),
        ("nibble_kernel (grouped: eight queries' 4-bit tables per gather; build + scan + top-k)",
         "search_grouped.cu", st_ms[5], int(pb[nib].sum()))]


def run_gpu(args, rank: int, world: int, local_rank: int):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as amp
    from paper_2606_07156_gb300 import abi
    from workloads import make_queries

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg, W = workload(args.config, device=dev)
    if args.nq:
        W = dict(W, queries=W["queries"][:args.nq], gt=W["gt"][:args.nq])
    index = amp.Index(W["centroids"], W["codebooks"], W["codes"], W["list_of"], device=local_rank)
    if args.no_nibble:
        index.set_nibble(False)
    if args.qchunk:
        index.set_qchunk(args.qchunk)
    Q = torch.from_numpy(W["queries"]).to(dev)
    nq, k = Q.shape[0], cfg["k"]
    stream = torch.cuda.current_stream(dev)
    out = (torch.empty((nq, k), dtype=torch.int64, device=dev), torch.empty((nq, k), dtype=torch.float32, device=dev))

    def run_q(Qd, nprobe, pol):
        ids, _ = index.search(Qd, nprobe, k, pol, stream=stream)
        torch.cuda.synchronize()
        return ids.cpu().numpy()

    def run(nprobe, pol):
        return run_q(Q, nprobe, pol)

    def run_full(nprobe, pol):
        ids, dists = index.search(Q, nprobe, k, pol, stream=stream)
        torch.cuda.synchronize()
        return ids.cpu().numpy(), dists.cpu().numpy()

    # the workload's nprobe (SIFT-shaped: the smallest of its sweep reaching
    # recall@10 >= 0.9, else the largest); plain FP32 recall over a sweep
    plain = amp.policy("plain")
    if args.nprobe is not None:
        nprobe, sweep = args.nprobe, (args.nprobe,)
    elif "nprobe_sweep" in cfg:
        sweep = cfg["nprobe_sweep"]
        nprobe = None
    else:
        nprobe = cfg["nprobe"]
        sweep = tuple(sorted({max(1, nprobe // 2), nprobe, min(cfg["nlist"], 2 * nprobe, 128)}))
    rec_plain, nn_plain = {}, {}
    for npb in sweep:
        ids = run(npb, plain)
        rec_plain[npb], nn_plain[npb] = recall(ids, W["gt"], 10), nn_in_top(ids, W["gt"], 10)
    if nprobe is None:
        ok = [npb for npb in sweep if rec_plain[npb] >= 0.9]
        nprobe = ok[0] if ok else max(sweep)
    ref_ids = run(nprobe, plain)
    cl_pick = None
    if args.cl == "auto":
        args.cl, cl_pick = pick_cl(index, Q, nprobe, stream)

    # learned predictor: labels, features and training on the GPU from training queries
    ntrain = cfg.get("ntrain", args.ntrain)
    Qt = torch.from_numpy(make_queries(args.config, ntrain, stream=200)).to(dev)

    def train(npb):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # trained on the two tables of the GB300 width map, wide pairs weighted up
        # (a wide pair put on a narrow table costs recall, the reverse only speed)
        index.train_predictor(Qt, npb, k, amp.train_cfg(epochs=args.epochs, batch=1024, lr=3e-3, seed=1,
                                                        gpu_classes=True, high_weight=args.high_weight,
                                                        nibble_classes=not args.two_classes))
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    Qc = torch.from_numpy(W["cal_queries"]).to(dev)

    def cal_ms(pol):
        """Mean time of a search of the calibration queries (3 runs after one)."""
        run_q(Qc, nprobe, pol)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        for _ in range(3):
            index.search(Qc, nprobe, k, pol, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 3

    # the predictor's classes chosen on the calibration queries: trained on
    # the three GB300 tables (4-bit / 8-bit / wide) and on two (8-bit / wide),
    # each calibrated on the recall budget; the faster one is kept
    class_maps = [False] if args.two_classes else [True, False]
    choice = {}
    for nib in class_maps:
        args.two_classes = not nib
        t_s = train(nprobe)
        m, tr = calibrate_margin(amp, Qc, W["cal_gt"], nprobe, k, run_q)
        pol = amp.policy("mlp", margin=m if np.isfinite(m) else 3.0e38, width_map=True)
        choice[nib] = dict(margin=m, tried=tr, train_s=t_s, cal_ms=cal_ms(pol), weights=index.get_predictor())
    best_nib = min(choice, key=lambda c: choice[c]["cal_ms"])
    args.two_classes = not best_nib
    index.set_predictor(choice[best_nib]["weights"])
    margin, tried, train_s = choice[best_nib]["margin"], choice[best_nib]["tried"], choice[best_nib]["train_s"]
    eq2_th, eq2_tried = calibrate_eq2(amp, Qc, W["cal_gt"], nprobe, k, run_q)
    # the adaptive policies' CL: args.cl (the FP32 rule, or the tensor cores
    # with an exact FP32 re-rank: the same probes either way)
    adaptive = amp.policy("mlp", margin=margin if np.isfinite(margin) else 3.0e38, width_map=True, cl=args.cl)
    predictor_w = index.get_predictor()
    policies = {"mlp": adaptive, "plain": plain}
    svr_info = None
    if not args.no_svr:
        svr_info = fit_svr(amp, abi, index, Qt, nprobe, k)
        svr_margin, svr_tried = calibrate_svr(amp, Qc, W["cal_gt"], nprobe, run_q)
        svr_info.update({"margin": svr_margin, "margin_calibration_recall_loss_pts": {str(a): b for a, b in
                                                                                     svr_tried.items()}})
        policies["svr"] = amp.policy("svr", margin=svr_margin, width_map=True, cl=args.cl)
    if eq2_th is not None:
        policies["eq2"] = amp.policy("eq2", thresholds=eq2_th, width_map=True)
    for b in (4, 6, 8, 12, 16):
        policies[f"fixed{b}"] = amp.policy("fixed", bits=b)
    # the adaptive policies run in the configuration the library's autotuner
    # picks on this batch (kernel, query order, grouped work-order chunk);
    # the others in the automatic one
    KN = {abi.KERNEL_BASIC: "query-major", abi.KERNEL_LIST_MAJOR: "list-major", abi.KERNEL_GROUPED: "grouped",
          abi.KERNEL_SPLIT: "split"}
    SN = {abi.SCHED_NATURAL: "natural", abi.SCHED_LPT: "longest-first"}
    tuned = None
    if not args.no_autotune:
        trials = index.autotune(Q, nprobe, k, adaptive, reps=2)
        best_t = min(trials, key=lambda r: r[2])
        tuned = {"kernel": KN.get(best_t[0], str(best_t[0])), "schedule": SN.get(best_t[1], str(best_t[1])),
                 "qchunk": int(best_t[3]),
                 "trials_ms": {f"{KN.get(t[0], t[0])}/{SN.get(t[1], t[1])}/q{t[3]}": round(t[2], 3) for t in trials}}
        cfg_tuned = (best_t[0], best_t[1], best_t[3])

    def use(name):
        """The adaptive policies in the tuned configuration, the rest automatic."""
        if tuned is not None and name in ("mlp", "svr"):
            abi.anns_set_option(index.handle, abi.OPT_KERNEL, cfg_tuned[0])
            abi.anns_set_option(index.handle, abi.OPT_SCHEDULE, cfg_tuned[1])
            abi.anns_set_option(index.handle, abi.OPT_QCHUNK, cfg_tuned[2])
        else:
            index.set_kernel("auto")
            index.set_schedule("auto")
            index.set_qchunk(args.qchunk)

    recs, mixes, full = {}, {}, {}
    for name, pol in policies.items():
        use(name)
        ids, dists = run_full(nprobe, pol)
        if name in ("mlp", "fixed8", "plain"):
            full[name] = (ids, dists)
        recs[name] = (recall(ids, W["gt"], 10), overlap(ids, ref_ids, k), nn_in_top(ids, W["gt"], 10))
        mixes[name] = bits_mix(index, abi, nq, nprobe)
    log(f"nprobe {nprobe}; margin {margin} {tried}; eq2 {eq2_th} {eq2_tried}; recalls {recs}")

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    use("mlp")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    abi.anns_profile(index.handle, 1)
    launches0 = abi.anns_kernel_launches()
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        nvtx_push("anns_timed")
        ms_ad = time_steps(lambda: index.search(Q, nprobe, k, adaptive, stream=stream, out=out),
                           args.steps, args.warmup, stream, flush)
        nvtx_pop()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    stage_ms, cnt = abi.anns_profile(index.handle, 0)
    launches_per_step = (abi.anns_kernel_launches() - launches0) / max(cnt, 1)
    # stage view of the adaptive step (the last search before the taps below)
    probes_ad = index.tap(abi.TAP_PROBES, (nq, nprobe), np.int32)
    bits_ad = index.tap(abi.TAP_BITS, (nq, nprobe), np.uint8)
    ms_pol = {"mlp": ms_ad}
    for name, pol in policies.items():
        if name != "mlp":
            use(name)
            ms_pol[name] = time_steps(lambda: index.search(Q, nprobe, k, pol, stream=stream, out=out),
                                      args.steps, args.warmup, stream, flush)
    use("mlp")
    # end to end through the host-buffer entry point (pinned in, pinned out)
    Qh = torch.from_numpy(W["queries"]).pin_memory()
    ih = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    dh = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    for _ in range(args.warmup):
        index.search_host(Qh, nprobe, k, adaptive, stream=stream, out=(ih, dh))
    e2e_t = []
    for i in range(args.steps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        t = time.perf_counter()
        index.search_host(Qh, nprobe, k, adaptive, stream=stream, out=(ih, dh))
        e2e_t.append(time.perf_counter() - t)
    rec_e2e = recall(ih.numpy(), W["gt"], 10)

    # second operating point: the smallest nprobe whose plain 1-recall@10
    # reaches 0.9 (the predictor retrained and its margin recalibrated there,
    # on the 1-recall@10 reading)
    op2 = None
    use("plain")
    if not args.no_second_point:
        cands = [p for p in (1, 2, 4, 8, 16, 32, 64) if p <= min(cfg["nlist"], 128)]
        nn_sweep, np2 = {}, None
        for npb in cands:
            nn_sweep[npb] = nn_in_top(run(npb, plain), W["gt"], 10)
            if nn_sweep[npb] >= 0.9:
                np2 = npb
                break
        if np2 is not None:
            train(np2)
            m2, tried2 = calibrate_margin_nn(amp, Qc, W["cal_gt"], np2, run_q)
            pols2 = {"plain": plain, "mlp": amp.policy("mlp", margin=m2 if np.isfinite(m2) else 3.0e38,
                                                       width_map=True, cl=args.cl),
                     "fixed8": amp.policy("fixed", bits=8)}
            # the learned policy in the configuration the autotuner picks at
            # this nprobe (one probe per query leaves nothing to group)
            tuned2 = None
            if not args.no_autotune:
                t2 = min(index.autotune(Q, np2, k, pols2["mlp"], reps=2), key=lambda r: r[2])
                tuned2 = (t2[0], t2[1], t2[3])
            blk = {}
            for name, pol in pols2.items():
                if name == "mlp" and tuned2 is not None:
                    abi.anns_set_option(index.handle, abi.OPT_KERNEL, tuned2[0])
                    abi.anns_set_option(index.handle, abi.OPT_SCHEDULE, tuned2[1])
                    abi.anns_set_option(index.handle, abi.OPT_QCHUNK, tuned2[2])
                else:
                    use("plain")
                ids = run(np2, pol)
                ms = time_steps(lambda: index.search(Q, np2, k, pol, stream=stream, out=out), args.steps,
                                args.warmup, stream, flush)
                blk[name] = {"ms_per_step": round(float(np.mean(ms)), 4), "qps_per_gpu": round(nq / (np.mean(ms) / 1e3), 1),
                             "nn_in_top10": round(nn_in_top(ids, W["gt"], 10), 4),
                             "recall_at_10": round(recall(ids, W["gt"], 10), 4)}
            op2 = {"reading": "1-recall@10: the exact nearest neighbour among the 10 returned", "nprobe": np2,
                   "plain_nn_in_top10_sweep": {str(a): round(b, 4) for a, b in nn_sweep.items()},
                   "mlp_margin": m2, "margin_calibration_loss_pts": {str(a): b for a, b in tried2.items()},
                   "policies": blk, "mlp_config": None if tuned2 is None else
                   f"{KN.get(tuned2[0], tuned2[0])}/{SN.get(tuned2[1], tuned2[1])}/q{tuned2[2]}",
                   "speedup_mlp_vs_plain": round(blk["plain"]["ms_per_step"] / blk["mlp"]["ms_per_step"], 3)}
            use("plain")
        else:
            op2 = {"reading": "1-recall@10", "reached": False,
                   "plain_nn_in_top10_sweep": {str(a): round(b, 4) for a, b in nn_sweep.items()}}
        index.set_predictor(predictor_w)  # the headline predictor back
    del Qc, Qt

    totals = {name: sum(v) / 1e3 for name, v in ms_pol.items()}
    totals["_e2e"] = sum(e2e_t)
    totals = max_over_ranks(totals, world, dev)
    total_e2e = totals.pop("_e2e")
    if rank != 0:
        index.close()
        return None
    qps = weak_scaling_qps(totals, world, nq, args.steps)
    qps_e2e = world * nq * args.steps / total_e2e
    # roofline of the dominant kernel of the adaptive step (search_stages)
    pb = pair_bytes(index, probes_ad, cfg["M"])
    st_ms = [v / max(cnt, 1) for v in stage_ms]
    stage_names, cands = search_stages(tuned["kernel"] if tuned is not None else None, st_ms, bits_ad, pb)
    kname, kfile, kms, nbytes = max(cands, key=lambda c: c[2])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = nbytes / (kms / 1e3) / 1e9
    src = os.path.join(ROOT, "paper_2606_07156_gb300", "csrc", kfile)
    wl = f"{cfg['name']} nq={nq} nprobe={nprobe} k={k}"
    prof = roofline_profile(src, wl, kname.split(" ")[0])
    roof = {"bound": prof["bound"] if prof else "hbm", "kernel": kname,
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": "measured" if peaks else "fallback",
            "traffic": prof["dram_bytes_per_launch"] if prof else None,
            "algorithmic_bytes_per_launch": nbytes, "kernel_ms": round(kms, 4),
            "lookups_per_s": round(nbytes / (kms / 1e3), 1),
            "achieved_is": "algorithmic bytes (one code byte per LUT lookup, query-major) / kernel time"}
    if prof:
        dram_gbs = prof["dram_bytes_per_launch"] / (kms / 1e3) / 1e9
        roof.update({"dram_gbs": round(dram_gbs, 1), "dram_frac": round(dram_gbs / peak, 4),
                     "profile": prof.get("summary"), "binding_unit_pct": prof.get("binding_unit_pct")})
    nn_best = max(rec_plain, key=lambda a: rec_plain[a])
    line = {
        "metric": METRIC, "value": round(qps["mlp"], 1), "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(totals["mlp"] * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16-lut,i32-acc|f32",
        "data": f"synthetic (seeded {cfg['name']} mixture; no public dataset)",
        "config": {"workload": wl, "n": int(W["codes"].shape[0]), "dim": cfg["dim"], "nlist": cfg["nlist"],
                   "M": cfg["M"], "nprobe": nprobe, "k": k, "nq": nq,
                   "cl": f"{args.cl} (adaptive policies; plain FP32 uses the FP32 rule)"
                         + (f"; picked by timing the CL alone: {cl_pick} ms" if cl_pick else ""),
                   "policy": f"learned MLP per (query, list) trained on GB300 table classes, round-up "
                             f"margin {margin} (recall-loss budget {LOSS_BUDGET} pt on calibration queries), widths 6->8 bits "
                             f"and 12/16->FP32; 4-bit tables eight queries per gather",
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "recall_at_10": round(recs["mlp"][0], 4),
        "top10_kept_vs_plain": round(recs["mlp"][1], 4),
        "nn_in_top10": round(recs["mlp"][2], 4),
        "recall_condition": {
            "reading": "10-recall@10 = |top-10 found ∩ exact top-10| / 10", "threshold": 0.9,
            "reached": bool(rec_plain[nn_best] >= 0.9), "plain_recall_sweep": {str(a): round(b, 4) for a, b in
                                                                                 rec_plain.items()},
            "note": "not reachable on this workload by IVF-PQ with these codes at any nprobe of the sweep (the PQ "
                    "reconstruction error bounds it); the headline compares the policies at equal nprobe, loss "
                    "<= 1 point" if rec_plain[nn_best] < 0.9 else "reached"},
        "second_operating_point": op2,
        "bits_mix": mixes["mlp"],
        "plain_fp32": {"qps": round(qps["plain"], 1), "recall_at_10": round(recs["plain"][0], 4),
                       "ms_per_step": round(totals["plain"] * 1e3 / args.steps, 4)},
        "speedup_vs_plain_fp32": round(qps["mlp"] / qps["plain"], 3),
        "recall_loss_vs_plain_pts": round(100.0 * (recs["plain"][0] - recs["mlp"][0]), 3),
        "policies": {name: {"qps": round(qps[name], 1), "recall_at_10": round(recs[name][0], 4),
                            "top10_kept_vs_plain": round(recs[name][1], 4),
                            "nn_in_top10": round(recs[name][2], 4),
                            "ms_per_step": round(totals[name] * 1e3 / args.steps, 4)} for name in qps},
        "autotuned": tuned,
        "eq2_thresholds": list(eq2_th) if eq2_th is not None else None,
        "svr_comparator": None if svr_info is None else dict(
            svr_info, bits_mix=mixes["svr"], speedup_vs_plain=round(qps["svr"] / qps["plain"], 3),
            recall_at_10=round(recs["svr"][0], 4), mlp_speedup_vs_plain=round(qps["mlp"] / qps["plain"], 3),
            mlp_recall_at_10=round(recs["mlp"][0], 4)),
        "predictor": {"class_map_choice": {("3 tables (4/8/wide)" if c else "2 tables (8/wide)"): {
                          "margin": choice[c]["margin"], "calibration_ms": round(choice[c]["cal_ms"], 4)}
                          for c in choice},
                      "train_queries": ntrain, "train_s": round(train_s, 2), "epochs": args.epochs,
                      "classes": "GB300 tables (8-bit / wide)" if args.two_classes else "GB300 tables (4-bit / 8-bit / wide)", "high_weight": args.high_weight,
                      "margin_calibration_recall_loss_pts": {str(a): b for a, b in tried.items()},
                      "recall_loss_budget_pts": LOSS_BUDGET},
        "plain_nn_in_top10_sweep": {str(a): round(b, 4) for a, b in nn_plain.items()},
        "stage_ms_per_step": {n: round(v, 4) for n, v in zip(stage_names, st_ms)},
        "roofline": roof,
        "e2e": {"value": round(qps_e2e, 1), "unit": "queries/s", "h2d_bytes_per_step": int(Qh.numel() * 4),
                "d2h_bytes_per_step": int(ih.numel() * 8 + dh.numel() * 4), "recall_at_10": round(rec_e2e, 4)},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk.summary(),
        "wall_s_timed": round(wall, 3),
    }
    # the same step replayed as one CUDA graph
    use("mlp")
    graph, _, _ = index.capture_graph(Q, nprobe, k, adaptive, out=out)
    ms_graph = time_steps(lambda: graph.launch(stream), args.steps, args.warmup, stream, flush)
    graph.close()
    line["graph_ms_per_step"] = round(float(np.mean(ms_graph)), 4)
    if not args.no_cl_bench:
        line["cl_fastpath"] = cl_tensor_bench(amp, dev, max(3, args.steps // 4), args.warmup, flush)
    if not args.no_subspace and world == 1:
        line["subspace_granularity"] = subspace_sweep(amp, index, W, cfg, nprobe, k, dev)
    if not args.no_build_bench and world == 1:
        line["index_build"] = index_build_bench(amp, dev, args.config)
    if not args.no_cpu_baseline and world == 1:
        ctx = dict(amp=amp, abi=abi, index=index, Q=Q, stream=stream, margin=margin, predictor=predictor_w)
        line.update(oracle_leg(W, cfg, nprobe, args.cpu_seconds, full, ctx))
    index.close()
    return line


def recall_mixed_k(ids: np.ndarray, gt: np.ndarray, kpq: np.ndarray) -> dict:
    """Recall of an uneven batch: recall@10 over the queries with k >= 10 and
    the exact nearest neighbour's hit rate over the queries with k = 1."""
    big, one = kpq >= 10, kpq == 1
    return {"recall_at_10_k_ge_10": round(recall(ids[big], gt[big], 10), 4) if big.any() else None,
            "nn_hit_k1": round(float(np.mean(ids[one, 0] == gt[one, 0])), 4) if one.any() else None}


def run_uneven(args, rank: int, world: int, local_rank: int):
    """The uneven batch of the GIST-shaped workload: per-query nprobe ~
    Zipf(1.1) on [1, 128] and k uniform on {1, 10, 100}, Zipf list sizes.
    Times plain FP32, fixed 8 bits and the learned policy under the natural
    query order and the longest-first (LPT) order; the grouped kernel's work
    queue runs largest list first in both."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_07156_gb300 as amp
    from paper_2606_07156_gb300 import abi
    from workloads import make_queries, mixed_k, zipf_nprobe

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg, W = workload(args.config, device=dev)
    index = amp.Index(W["centroids"], W["codebooks"], W["codes"], W["list_of"], device=local_rank)
    nq = len(W["queries"])
    Q = torch.from_numpy(W["queries"]).to(dev)
    npq = zipf_nprobe(nq, cfg["seed"])
    kpq = mixed_k(nq, cfg["seed"])
    NP, K = 128, 100
    npq_d, kpq_d = torch.from_numpy(npq).to(dev), torch.from_numpy(kpq).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = (torch.empty((nq, K), dtype=torch.int64, device=dev), torch.empty((nq, K), dtype=torch.float32, device=dev))

    def run(pol, Qd=Q, npd=npq_d, kpd=kpq_d):
        ids, dists = index.search(Qd, NP, K, pol, nprobe_per_q=npd, k_per_q=kpd, stream=stream)
        torch.cuda.synchronize()
        return ids.cpu().numpy(), dists.cpu().numpy()

    # predictor trained at the batch's mean nprobe, on the three GB300 tables
    # (4-bit / 8-bit / wide) and on two (8-bit / wide); each margin calibrated
    # on calibration queries drawn with the same nprobe distribution (k = 10),
    # and the class map whose calibrated policy searches them faster is kept
    Qt = torch.from_numpy(make_queries(args.config, args.ntrain, stream=200)).to(dev)
    Qc = torch.from_numpy(W["cal_queries"]).to(dev)
    ncal = len(Qc)
    npc = torch.from_numpy(zipf_nprobe(ncal, cfg["seed"] + 7)).to(dev)
    k10 = torch.full((ncal,), 10, dtype=torch.int32, device=dev)

    def cal_recall(pol):
        return 100.0 * recall(run(pol, Qc, npc, k10)[0], W["cal_gt"], 10)

    def cal_ms(pol):
        run(pol, Qc, npc, k10)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        for _ in range(3):
            index.search(Qc, NP, K, pol, nprobe_per_q=npc, k_per_q=k10, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 3

    base = cal_recall(amp.policy("plain"))
    choice = {}
    for nib in ([False] if args.two_classes else [True, False]):
        t0 = time.perf_counter()
        index.train_predictor(Qt, 20, 10, amp.train_cfg(epochs=args.epochs, batch=1024, lr=3e-3, seed=1,
                                                        gpu_classes=True, high_weight=args.high_weight,
                                                        nibble_classes=nib))
        torch.cuda.synchronize()
        t_s = time.perf_counter() - t0
        m_ok, tr = float("inf"), {}
        for m in (-8.0, -6.0, -4.0, -3.0, -2.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0):
            tr[m] = round(base - cal_recall(amp.policy("mlp", margin=m, width_map=True)), 3)
            if tr[m] <= LOSS_BUDGET:
                m_ok = m
                break
        pol = amp.policy("mlp", margin=m_ok if np.isfinite(m_ok) else 3.0e38, width_map=True)
        choice[nib] = dict(margin=m_ok, tried=tr, train_s=t_s, cal_ms=cal_ms(pol), weights=index.get_predictor())
    best_nib = min(choice, key=lambda c: choice[c]["cal_ms"])
    index.set_predictor(choice[best_nib]["weights"])
    margin, tried, train_s = choice[best_nib]["margin"], choice[best_nib]["tried"], choice[best_nib]["train_s"]
    del Qt, Qc
    cl, cl_ms = pick_cl(index, Q, NP, stream) if args.cl == "auto" else (args.cl, None)
    policies = {"plain": amp.policy("plain"), "fixed8": amp.policy("fixed", bits=8, cl=cl),
                "mlp": amp.policy("mlp", margin=margin if np.isfinite(margin) else 3.0e38, width_map=True, cl=cl)}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    res, full = {}, {}
    with ClockSampler(local_rank) as clk:
        for name, pol in policies.items():
            ids, dists = run(pol)
            full[name] = (ids, dists)
            mix = bits_mix(index, abi, nq, NP, npq)
            # the automatic kernel (grouped for the adaptive policies) and, for
            # them, the split query-major search, each under both query orders
            for kern in (("auto", "split") if name != "plain" else ("auto",)):
                index.set_kernel(kern)
                for sched in ("natural", "lpt"):
                    index.set_schedule(sched)
                    abi.anns_profile(index.handle, 1)
                    ms = time_steps(lambda: index.search(Q, NP, K, pol, nprobe_per_q=npq_d, k_per_q=kpq_d,
                                                         stream=stream, out=out), args.steps, args.warmup, stream,
                                    flush)
                    st, cnt = abi.anns_profile(index.handle, 0)
                    res[(name, sched if kern == "auto" else f"split/{sched}")] = {
                        "ms_per_step": round(float(np.mean(ms)), 4), "qps": round(nq / (np.mean(ms) / 1e3), 1),
                        "stage_ms": [round(v / max(cnt, 1), 4) for v in st]}
            index.set_kernel("auto")
            res[(name, "recall")] = recall_mixed_k(ids, W["gt"], kpq)
            res[(name, "mix")] = mix
    index.set_schedule("auto")
    runs = {n: {c: res[(n, c)] for c in ("natural", "lpt", "split/natural", "split/lpt") if (n, c) in res}
            for n in policies}
    best = {n: min(r["ms_per_step"] for r in runs[n].values()) for n in policies}
    best_cfg = {n: min(runs[n], key=lambda c: runs[n][c]["ms_per_step"]) for n in policies}
    line = {
        "metric": METRIC, "value": round(nq / (best["mlp"] / 1e3), 1), "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["mlp"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16-lut,i32-acc|f32",
        "data": f"synthetic (seeded {cfg['name']} mixture; no public dataset)",
        "config": {"workload": f"{cfg['name']} nq={nq} nprobe~Zipf(1.1) on [1,128] (mean {npq.mean():.2f}) "
                               f"k in {{1,10,100}}", "n": int(W["codes"].shape[0]), "dim": cfg["dim"],
                   "nlist": cfg["nlist"], "M": cfg["M"], "largest_list": int(np.bincount(W["list_of"]).max()),
                   "l2": "flushed between steps (512 MB write)",
                   "cl": f"{cl} (adaptive policies; plain FP32 uses the FP32 rule)"
                         + (f"; picked by timing the CL alone at nprobe {NP}: {cl_ms} ms" if cl_ms else "")},
        "policies": {n: {**runs[n], "best": best_cfg[n], **res[(n, "recall")], "bits_mix": res[(n, "mix")]}
                     for n in policies},
        "speedup_mlp_vs_plain": round(best["plain"] / best["mlp"], 3),
        "lpt_vs_natural": {n: round(res[(n, "natural")]["ms_per_step"] / res[(n, "lpt")]["ms_per_step"], 3)
                           for n in policies},
        "predictor": {"train_s": round(train_s, 2), "margin": margin,
                      "classes": "GB300 tables (4-bit / 8-bit / wide)" if best_nib else "GB300 tables (8-bit / wide)",
                      "class_map_choice": {("3 tables (4/8/wide)" if c else "2 tables (8/wide)"): {
                          "margin": choice[c]["margin"], "calibration_ms": round(choice[c]["cal_ms"], 4)}
                          for c in choice},
                      "margin_calibration_recall_loss_pts": {str(a): b for a, b in tried.items()}},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and world == 1:
        from oracle import ivfpq
        ref = ivfpq.Index(W["centroids"], W["codebooks"], W["codes"], W["list_of"])
        done, t0 = 0, time.perf_counter()
        ok_i = ok_d = True
        while time.perf_counter() - t0 < args.cpu_seconds and done < nq:
            sl = slice(done, done + 4)
            oi, od = ivfpq.search(ref, W["queries"][sl], NP, K, bits=8, nprobe_per_q=npq[sl], k_per_q=kpq[sl])
            ok_i &= bool(np.array_equal(oi, full["fixed8"][0][sl]))
            ok_d &= bool(np.array_equal(od, full["fixed8"][1][sl]))
            done += len(oi)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(done / el, 2), "unit": "queries/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {done} queries of the uneven batch, fixed 8-bit tables"}
        line["parity_at_bench_size"] = {"fixed8": {"queries": done, "ids_equal": ok_i, "dists_equal": ok_d}}
    index.close()
    return line


# ------------------------------------------------------------------ CPU oracle leg

_REF = None


def _oracle_init(paths: dict, ready):
    """Worker set-up: the oracle's index over the memory-mapped arrays; counts
    itself in `ready` when done."""
    global _REF
    from oracle import ivfpq
    a = {k: np.load(p, mmap_mode="r") for k, p in paths.items()}
    _REF = ivfpq.Index(a["centroids"], a["codebooks"], a["codes"], a["list_of"])
    with ready.get_lock():
        ready.value += 1


def oracle_mlp_bits(ref, Qs: np.ndarray, nprobe: int, pred: dict, margin: float) -> np.ndarray:
    """The oracle's own widths for the learned policy: features, FP16-operand
    MLP inference, the round-up rule and the GB300 width map."""
    from oracle import ivfpq, predictor
    D2 = ivfpq.coarse_d2_fp32(Qs, ref.centroids)
    probes, pd = ivfpq.locate(D2, nprobe)
    F = predictor.features(pd, probes, ref.radius, ref.sizes)
    Xn = predictor.normalise(F.reshape(-1, 5), pred["mean"], pred["inv_std"])
    z = predictor.mlp_logits16(predictor.to_fp16({k: pred[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3")}), Xn)
    return predictor.gpu_width(predictor.decide_bits(z, np.float32(margin)).reshape(len(Qs), nprobe))


def _oracle_job(job):
    """One chunk of the oracle's search in a worker: (first row, ids, dists)."""
    from oracle import ivfpq
    row0, Qs, nprobe, k, mode, pred, margin = job
    bits = oracle_mlp_bits(_REF, Qs, nprobe, pred, margin) if mode == "mlp" else 8
    ids, dists = ivfpq.search(_REF, Qs, nprobe, k, bits=bits)
    return row0, ids, dists


def _margin32(margin: float) -> float:
    return float(np.float32(margin if np.isfinite(margin) else 3.0e38))


def oracle_all_cores(W, cfg, nprobe: int, row0: int, nrows: int, pred: dict, margin: float, cores: int):
    """The oracle's search of queries row0 .. row0 + nrows - 1 under the learned
    policy (widths from the oracle's own inference), one spawned process per
    core over memory-mapped index arrays. Returns (ids, dists, seconds), the
    seconds counted from the moment every worker has built its index."""
    import multiprocessing as mp
    k = cfg["k"]
    Qs = W["queries"]
    paths = {}
    os.makedirs(CACHE, exist_ok=True)
    for key in ("centroids", "codebooks", "codes", "list_of"):
        a = np.ascontiguousarray(W[key])
        p = os.path.join(CACHE, f"oracle_{cfg['name']}_{a.shape[0]}_{key}.npy")
        if not os.path.exists(p):
            np.save(p, a)
        paths[key] = p
    margin = _margin32(margin)
    jobs = [(row0 + s, Qs[row0 + s:row0 + min(s + 2, nrows)], nprobe, k, "mlp", pred, margin)
            for s in range(0, nrows, 2)]
    sp = mp.get_context("spawn")
    ready = sp.Value("i", 0)
    with sp.Pool(cores, initializer=_oracle_init, initargs=(paths, ready)) as pool:
        t_set = time.perf_counter()
        while ready.value < cores and time.perf_counter() - t_set < 600:
            time.sleep(0.05)  # every worker's index is built before the clock starts
        t0 = time.perf_counter()
        res = pool.map(_oracle_job, jobs, chunksize=1)
        elc = time.perf_counter() - t0
    res.sort(key=lambda r: r[0])
    mi = np.concatenate([r[1] for r in res]) if res else np.zeros((0, k), np.int64)
    md = np.concatenate([r[2] for r in res]) if res else np.zeros((0, k), np.float32)
    return mi, md, elc


def oracle_leg(W, cfg, nprobe: int, seconds: float, gpu_full: dict, ctx: dict) -> dict:
    """The oracle as it stands on a bounded sample of the same queries:
    single-threaded (fixed 8 bits) and one process per host core (the learned
    policy, widths from the oracle's own inference), each compared with the
    GPU's results bit for bit; then the error of every float output of the
    GPU path against FP64 on a few queries."""
    from oracle import ivfpq
    k = cfg["k"]
    Qs = W["queries"]
    ref = ivfpq.Index(W["centroids"], W["codebooks"], W["codes"], W["list_of"])
    # single thread, fixed 8 bits
    done, t0, chunk = 0, time.perf_counter(), 4
    o_ids, o_d = [], []
    while time.perf_counter() - t0 < seconds and done < len(Qs):
        i, d = ivfpq.search(ref, Qs[done:done + chunk], nprobe, k, bits=8)
        o_ids.append(i)
        o_d.append(d)
        done += len(i)
    el1 = time.perf_counter() - t0
    n1 = done
    oi, od = np.concatenate(o_ids), np.concatenate(o_d)
    par8 = {"queries": n1, "ids_equal": bool(np.array_equal(oi, gpu_full["fixed8"][0][:n1])),
            "dists_equal": bool(np.array_equal(od, gpu_full["fixed8"][1][:n1]))}
    # every core, the learned policy (rows after the single-threaded sample)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    rate1 = n1 / el1
    n_all = int(min(len(Qs) - n1, max(cores * 2, rate1 * cores * seconds * 0.8)))
    mi, md, elc = oracle_all_cores(W, cfg, nprobe, n1, n_all, ctx["predictor"], ctx["margin"], cores)
    g_i, g_d = gpu_full["mlp"]
    parm = {"queries": len(mi), "ids_equal": bool(np.array_equal(mi, g_i[n1:n1 + len(mi)])),
            "dists_equal": bool(np.array_equal(md, g_d[n1:n1 + len(md)])),
            "widths": "the oracle's own features, FP16-operand MLP inference, round-up rule and width map"}
    out = {
        "cpu_baseline": {"value": round(len(mi) / elc, 2), "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"queries {n1}..{n1 + len(mi) - 1} of {len(Qs)}, nprobe={nprobe}, learned "
                                   f"policy (the oracle's own inference), one numpy process per core",
                         "seconds": round(elc, 2),
                         "single_thread": {"value": round(n1 / el1, 2), "unit": "queries/s", "cores": 1,
                                           "sample": f"first {n1} queries, fixed 8-bit tables",
                                           "seconds": round(el1, 2)}},
        "parity_at_bench_size": {"fixed8": par8, "mlp": parm,
                                 "all_equal": bool(par8["ids_equal"] and par8["dists_equal"] and parm["ids_equal"]
                                                   and parm["dists_equal"])},
    }
    out["fp64_error"] = fp64_errors(ref, W, cfg, nprobe, ctx)
    return out


def fp64_errors(ref, W, cfg, nprobe: int, ctx: dict, nq_s: int = 16) -> dict:
    """Measured error against FP64 of every float output of the GPU path, on
    the first nq_s queries: the FP32 coarse distances, the BF16 tensor-core
    coarse distances D~, the FP32 table entries, the plain FP32 ADC distances
    and the quantised (8-bit) distances against their M Delta / 2 bound."""
    import torch

    from oracle import ivfpq
    amp, abi, index, stream = ctx["amp"], ctx["abi"], ctx["index"], ctx["stream"]
    k, M = cfg["k"], cfg["M"]
    Qs = W["queries"][:nq_s]
    Qd = ctx["Q"][:nq_s].contiguous()
    D64 = ivfpq.coarse_d2_fp64(Qs, ref.centroids)
    out = {"queries": nq_s}
    # FP32 coarse distances of the probed lists
    ids_p, d_p = index.search(Qd, nprobe, k, amp.policy("plain"), stream=stream)
    torch.cuda.synchronize()
    probes = index.tap(abi.TAP_PROBES, (nq_s, nprobe), np.int32)
    pd = index.tap(abi.TAP_PROBE_D2, (nq_s, nprobe), np.float32).astype(np.float64)
    want = np.take_along_axis(D64, probes.astype(np.int64), axis=1)
    out["cl_d2_fp32_max_rel"] = float((np.abs(pd - want) / want).max())
    # plain FP32 ADC distances of the returned vectors vs FP64 ||q - x_hat||^2
    ids_p, d_p = ids_p.cpu().numpy(), d_p.cpu().numpy().astype(np.float64)

    def d64_of(ids):
        o = np.zeros(ids.shape)
        for i in range(ids.shape[0]):
            v = ids[i] >= 0
            xh = ref.reconstruct(ids[i][v])
            o[i][v] = ((xh - Qs[i].astype(np.float64)) ** 2).sum(1)
        return o

    w = d64_of(ids_p)
    v = ids_p >= 0
    out["adc_fp32_max_rel"] = float((np.abs(d_p - w)[v] / w[v]).max())
    # quantised 8-bit distances vs FP64, relative to the pair's M Delta / 2 bound
    ids8, d8 = index.search(Qd, nprobe, k, amp.policy("fixed", bits=8), stream=stream)
    torch.cuda.synchronize()
    ids8, d8 = ids8.cpu().numpy(), d8.cpu().numpy().astype(np.float64)
    w8 = d64_of(ids8)
    D32 = ivfpq.coarse_d2_fp32(Qs, ref.centroids)
    worst_rel, worst_ratio = 0.0, 0.0
    for i in range(nq_s):
        for j in range(k):
            if ids8[i, j] < 0:
                continue
            l = int(W["list_of"][ids8[i, j]])
            T32 = ivfpq.lut_fp32(Qs[i], ref.centroids[l], ref.books)
            qz = ivfpq.quantize_lut(T32, 8, D32[i, l])
            err = abs(d8[i, j] - w8[i, j])
            worst_rel = max(worst_rel, err / w8[i, j])
            # M Delta / 2 plus the FP32 table's own error (the FP32 rule's distance vs FP64)
            t64 = ivfpq.lut_fp64(Qs[i], ref.centroids[l], ref.books)
            bound = M * qz["delta64"] / 2 + 1e-5 * (t64.sum() / 256 + w8[i, j])
            worst_ratio = max(worst_ratio, err / bound)
    out["adc_q8_max_rel"] = worst_rel
    out["adc_q8_err_over_bound_max"] = worst_ratio
    # FP32 table entries (pairs: each sample query with its first, middle and last probe)
    pq = np.repeat(np.arange(nq_s, dtype=np.int32), 3)
    pl = probes[:, [0, nprobe // 2, nprobe - 1]].reshape(-1).astype(np.int32)
    T, _, _ = index.compute_luts(Qd, torch.from_numpy(pq).to(Qd.device), torch.from_numpy(pl).to(Qd.device),
                                 torch.zeros(len(pq), dtype=torch.uint8, device=Qd.device))
    T = T.cpu().numpy().astype(np.float64)
    rel, mixed = 0.0, 0.0
    for p in range(len(pq)):
        Ts = ivfpq.lut_shift_fp64(Qs[pq[p]], ref.centroids[pl[p]], ref.books)
        T64 = ivfpq.lut_fp64(Qs[pq[p]], ref.centroids[pl[p]], ref.books)
        e = np.abs(T[p] - Ts)
        big = T64 > 1e-3 * T64.mean()
        rel = max(rel, float((e[big] / T64[big]).max()))
        mixed = max(mixed, float((e / (T64 + T64.mean())).max()))
    out["lut_fp32_max_rel"] = rel
    out["lut_fp32_max_err_over_T64_plus_mean"] = mixed
    # tensor-core coarse distances D~ (normwise per query row), per operand format
    for cl in ("bf16", "fp16", "fp8"):
        index.locate(Qd, nprobe, cl=cl, stream=stream)
        torch.cuda.synchronize()
        Dt = index.tap(abi.TAP_COARSE_APPROX, (nq_s, ref.nlist), np.float32).astype(np.float64)
        out[f"cl_{cl}_normwise_rel_max"] = float((np.linalg.norm(Dt - D64, axis=1) /
                                                  np.linalg.norm(D64, axis=1)).max())
    out["tolerances"] = {"fp32_lut": "per element <= 1e-5 (T64 + mean T64)", "fp32_distances": "rel <= 1e-5",
                         "bf16_fp16_fp8": "normwise rel <= 2e-2", "quantised": "<= M Delta / 2 (+ FP32 rounding)"}
    return {k2: (round(v2, 9) if isinstance(v2, float) else v2) for k2, v2 in out.items()}


def run_reference(args, rank: int):
    if rank != 0:
        return None
    # the workload (index training, ground truth) is built on the GPU when
    # there is one, as for the GPU arm; only the oracle's search is timed,
    # on the host
    import torch
    cfg, W = workload(args.config, device=torch.device("cuda", 0) if torch.cuda.is_available() else None)
    # the GPU arm's nprobe: the workload's own (SIFT-shaped: the largest of the
    # sweep; no nprobe of the sweep reaches recall@10 0.9 with these codes)
    nprobe = args.nprobe or (max(cfg["nprobe_sweep"]) if "nprobe_sweep" in cfg else cfg["nprobe"])
    from oracle import ivfpq
    ref = ivfpq.Index(W["centroids"], W["codebooks"], W["codes"], W["list_of"])
    Qs = W["queries"]
    per_step = max(4, args.ref_queries)
    for i in range(args.warmup):
        ivfpq.search(ref, Qs[:2], nprobe, cfg["k"], bits=8)
    ts, done = [], 0
    for i in range(args.steps):
        q = Qs[(i * per_step) % len(Qs):][:per_step]
        t = time.perf_counter()
        ivfpq.search(ref, q, nprobe, cfg["k"], bits=8)
        ts.append(time.perf_counter() - t)
        done += len(q)
    qps = done / sum(ts)
    wl = f"{cfg['name']} nq={len(Qs)} nprobe={nprobe} k={cfg['k']}"
    return {"impl": "reference", "metric": METRIC, "value": round(qps, 2), "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(ts) / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-rule/f64",
            "data": f"synthetic (seeded {cfg['name']} mixture; no public dataset)",
            "config": {"workload": wl, "policy": "fixed-8bit (the oracle's cost per pair is the same for every "
                                              "width)", "sample_queries_per_step": per_step},
            "cpu_baseline": {"value": round(qps, 2), "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} queries per step, numpy single thread"},
            "e2e": {"value": round(qps, 2), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=("gb300", "reference"))
    ap.add_argument("--config", default="C")
    ap.add_argument("--nprobe", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-queries", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cl-bench", action="store_true", help="skip the coarse-stage comparison")
    ap.add_argument("--no-second-point", action="store_true", help="skip the 1-recall@10 operating point")
    ap.add_argument("--no-svr", action="store_true", help="skip the SVR-RBF comparator")
    ap.add_argument("--no-build-bench", action="store_true", help="skip the index-training comparison")
    ap.add_argument("--no-subspace", action="store_true", help="skip the sub-space granularity sweep")
    ap.add_argument("--two-classes", action="store_true",
                    help="train the predictor on two GB300 tables (8-bit / wide) instead of three (4 / 8 / wide)")
    ap.add_argument("--no-nibble", action="store_true", help="4-bit pairs four per word (no nibble packing)")
    ap.add_argument("--qchunk", type=int, default=0, help="queries per chunk of the grouped work order (0 = auto)")
    ap.add_argument("--no-autotune", action="store_true", help="run the adaptive policies in the automatic configuration")
    ap.add_argument("--cl", default="auto", choices=("auto", "fp32", "bf16", "fp16", "fp8"),
                    help="CL of the adaptive policies: FP32 rule, tensor cores (BF16, FP16 or FP8 E4M3 "
                         "operands) + exact re-rank, or auto (FP32 or FP16, whichever the CL alone runs faster "
                         "on the workload's queries)")
    ap.add_argument("--nq", type=int, default=0, help="evaluate the first nq queries only (profiling)")
    ap.add_argument("--ntrain", type=int, default=10000, help="training queries for the predictor")
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--high-weight", type=float, default=10.0, help="loss weight of wide-table training samples")
    ap.add_argument("--only-cl", action="store_true",
                    help="run only the coarse-stage comparison (for profiling its kernels)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.only_cl:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        torch.cuda.set_device(dev)
        import __graft_entry__
        __graft_entry__.build()
        import paper_2606_07156_gb300 as amp
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps({"cl_fastpath": cl_tensor_bench(amp, dev, args.steps, args.warmup, flush)}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        from workloads import CONFIGS
        if args.config == "D":
            line = run_uneven(args, rank, world, local_rank)
        else:
            line = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
