"""Adaptive mixed-precision IVF-PQ search on one GB300 (sm_103a).

The compute lives in ``libanns_amp.so`` (hand-written CUDA kernels behind the C
ABI of include/anns_amp.h). This package is the thin Python side: ``abi``
binds the C entry points by name, and ``Index`` below marshals numpy arrays
and torch tensors (used only as device memory) into those calls.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import abi
from .abi import AnnsError  # noqa: F401

_MODES = {"plain": abi.LUT_PLAIN_FP32, "fixed": abi.LUT_FIXED_BITS, "eq2": abi.LUT_HEURISTIC_EQ2,
          "mlp": abi.LUT_MLP, "explicit": abi.LUT_EXPLICIT, "svr": abi.LUT_SVR}
# CL operands: FP32 on the CUDA cores, or a tensor-core GEMM (+ exact re-rank)
CL_PREC = {"fp32": abi.PREC_FP32, "bf16": abi.PREC_BF16, "fp16": abi.PREC_FP16, "fp8": abi.PREC_FP8E4M3}


def policy(mode: str = "plain", bits: int = 8, thresholds=(0.0, 0.0, 0.0, 0.0), margin: float = 0.0,
           pair_bits=None, width_map: bool = False, cl: str = "fp32") -> abi.anns_precision_policy:
    """Builds an anns_precision_policy. ``pair_bits`` (EXPLICIT) is a uint8 CUDA tensor
    [nq * nprobe], kept alive by the returned policy (the struct holds its device
    pointer); ``margin`` is the MLP round-up margin; ``width_map`` maps EQ2/MLP
    widths to this GPU's tables (6 -> 8 bits, 12 and 16 -> FP32)."""
    p = abi.anns_precision_policy()
    p.lut_mode = _MODES[mode]
    p.fixed_bits = int(bits)
    p.cl_prec = CL_PREC[cl]
    p.lc_prec = abi.PREC_FP32
    for i, t in enumerate(thresholds):
        p.eq2_thresholds[i] = float(t)
    p.fallback_margin = float(margin)
    p.pair_bits = None if pair_bits is None else pair_bits.data_ptr()
    p._pair_bits_ref = pair_bits  # the device memory the pointer refers to
    p.width_map = 1 if width_map else 0
    return p


_PRED_FIELDS = ("W1", "b1", "W2", "b2", "W3", "b3", "mean", "inv_std")
_PRED_SHAPES = {"W1": (32, 5), "b1": (32,), "W2": (32, 32), "b2": (32,), "W3": (5, 32), "b3": (5,),
                "mean": (5,), "inv_std": (5,)}


def predictor_to_struct(p: dict) -> abi.anns_predictor:
    """dict of numpy arrays (W1 [32,5] ... inv_std [5]) -> anns_predictor."""
    s = abi.anns_predictor()
    for f in _PRED_FIELDS:
        arr = np.ascontiguousarray(np.asarray(p[f], dtype=np.float32).reshape(-1))
        ctypes.memmove(getattr(s, f), arr.ctypes.data, arr.nbytes)
    return s


def predictor_to_dict(s: abi.anns_predictor) -> dict:
    return {f: np.ctypeslib.as_array(getattr(s, f)).copy().reshape(_PRED_SHAPES[f]) for f in _PRED_FIELDS}


def train_cfg(epochs: int = 10, batch: int = 1024, lr: float = 3e-3, seed: int = 0, gpu_classes: bool = False,
              high_weight: float = 1.0, nibble_classes: bool = False) -> abi.anns_train_cfg:
    """Training settings; ``gpu_classes`` trains on the two GB300 tables (8-bit / wide),
    ``nibble_classes`` on its three (4-bit nibble tables / 8-bit / wide)."""
    c = abi.anns_train_cfg()
    c.epochs, c.batch, c.lr, c.seed = epochs, batch, lr, seed
    c.label_map = 2 if nibble_classes else (1 if gpu_classes else 0)
    c.high_weight = high_weight
    return c


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class Graph:
    """A captured search (anns_graph); launch() replays it on a stream."""

    def __init__(self, handle):
        self.handle = handle

    def launch(self, stream=None):
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_graph_launch(self.handle, s)

    def close(self):
        if getattr(self, "handle", None):
            abi.anns_graph_free(self.handle)
            self.handle = None

    __del__ = close


class Index:
    """An index owned by the library, built from host arrays (Section 2.1)."""

    def __init__(self, centroids, codebooks, codes, list_of, ids=None, device: int = 0):
        cent = np.ascontiguousarray(centroids, dtype=np.float32)
        books = np.ascontiguousarray(codebooks, dtype=np.float32)
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        lo = np.ascontiguousarray(list_of, dtype=np.int32)
        uid = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
        d = abi.anns_build_desc()
        d.n, d.dim = codes.shape[0], cent.shape[1]
        d.nlist, d.M, d.ksub = cent.shape[0], codes.shape[1] if codes.ndim == 2 else books.shape[0], 256
        d.centroids, d.codebooks, d.codes = cent.ctypes.data, books.ctypes.data, codes.ctypes.data
        d.list_of = lo.ctypes.data
        d.ids = None if uid is None else uid.ctypes.data
        d.on_device, d.device = 0, device
        self.device = device
        self.handle = abi.anns_build_index_from_arrays(d)
        self.info = abi.anns_get_info(self.handle)
        self.dim, self.nlist, self.M = self.info.dim, self.info.nlist, self.info.M

    @classmethod
    def _wrap(cls, handle: int, device: int) -> "Index":
        self = cls.__new__(cls)
        self.device = device
        self.handle = handle
        self.info = abi.anns_get_info(self.handle)
        self.dim, self.nlist, self.M = self.info.dim, self.info.nlist, self.info.M
        return self

    @classmethod
    def train(cls, base, nlist: int, M: int, iters: int = 10, pq_iters: int = 10, seed: int = 0,
              per_centroid: int = 256, pq_sample: int = 65536, device: int = 0) -> "Index":
        """Trains and builds an index on the GPU (anns_train_index). ``base`` is a
        float32 numpy array or CUDA tensor [n, dim]."""
        d = abi.anns_train_desc()
        d.nlist, d.M, d.iters, d.pq_iters, d.seed = nlist, M, iters, pq_iters, seed
        d.per_centroid, d.pq_sample = per_centroid, pq_sample
        if isinstance(base, np.ndarray):
            base = np.ascontiguousarray(base, dtype=np.float32)
            h = abi.anns_train_index(base.ctypes.data, base.shape[0], base.shape[1], d, 0, device)
        else:
            h = abi.anns_train_index(base.data_ptr(), base.shape[0], base.shape[1], d, 1, device)
        return cls._wrap(h, device)

    @classmethod
    def load(cls, path: str, device: int = 0) -> "Index":
        return cls._wrap(abi.anns_load(path, device), device)

    def build_subspaces(self, slices: int, K: int, K_lc: int, iters: int = 10) -> None:
        """The paper's sub-space partitions of the centroids and codebooks (anns_build_subspaces)."""
        d = abi.anns_subspace_desc()
        d.slices, d.K, d.K_lc, d.iters = slices, K, K_lc, iters
        abi.anns_build_subspaces(self.handle, d)

    def search_subspace(self, queries, nprobe: int, k: int, th_cl=(np.inf,) * 3, th_lc=(np.inf,) * 3,
                        cl: bool = True, lc: bool = True, stream=None):
        """Search at sub-space precision; returns (ids, dists, low-precision counts [CL, LC])."""
        import torch
        nq = queries.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        low = torch.zeros(2, dtype=torch.int64, device=queries.device)
        p = abi.anns_subspace_policy()
        for i in range(3):
            p.th_cl[i], p.th_lc[i] = float(th_cl[i]), float(th_lc[i])
        p.cl, p.lc = int(cl), int(lc)
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_search_subspace(self.handle, _ptr(queries), nq, nprobe, k, p, _ptr(ids), _ptr(dists), _ptr(low), s)
        return ids, dists, low

    def save(self, path: str) -> None:
        abi.anns_save(self.handle, path)

    def export(self) -> dict:
        """The index's arrays in list order (anns_export_index)."""
        n, dim, nlist, M = self.info.n, self.dim, self.nlist, self.M
        out = dict(centroids=np.empty((nlist, dim), np.float32),
                   codebooks=np.empty((M, 256, dim // M), np.float32),
                   codes=np.empty((n, M), np.uint8), ids=np.empty(n, np.int64), list_len=np.empty(nlist, np.int64))
        abi.anns_export_index(self.handle, *(out[k].ctypes.data for k in
                                             ("centroids", "codebooks", "codes", "ids", "list_len")))
        return out

    def close(self):
        if getattr(self, "handle", None):
            abi.anns_free(self.handle)
            self.handle = None

    __del__ = close

    def search(self, queries, nprobe: int, k: int, pol=None, nprobe_per_q=None, k_per_q=None,
               stream=None, out=None):
        """queries: float32 CUDA tensor [nq, dim]. Returns (ids int64, dists float32) CUDA tensors."""
        import torch
        nq = queries.shape[0]
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
            dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        else:
            ids, dists = out
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_search(self.handle, _ptr(queries), nq, nprobe, _ptr(nprobe_per_q), k, _ptr(k_per_q),
                        pol, _ptr(ids), _ptr(dists), s)
        return ids, dists

    def search_host(self, queries, nprobe: int, k: int, pol=None, nprobe_per_q=None, k_per_q=None,
                    stream=None, out=None):
        """Host buffers in and out (pinned torch CPU tensors or numpy arrays); synchronous."""
        nq = queries.shape[0]
        if out is None:
            ids = np.empty((nq, k), dtype=np.int64)
            dists = np.empty((nq, k), dtype=np.float32)
        else:
            ids, dists = out
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_search_host(self.handle, _ptr(queries), nq, nprobe, _ptr(nprobe_per_q), k,
                             _ptr(k_per_q), pol, _ptr(ids), _ptr(dists), s)
        return ids, dists

    def set_kernel(self, which: str):
        """'auto', 'basic' (query-major), 'lists' (list-major, one warp per pair),
        'grouped' (narrow pairs packed four or eight queries to a gather) or 'split'
        (query-major in two passes: wide pairs, then 1..8-bit pairs on byte tables only)."""
        v = {"auto": abi.KERNEL_AUTO, "basic": abi.KERNEL_BASIC, "lists": abi.KERNEL_LIST_MAJOR,
             "grouped": abi.KERNEL_GROUPED, "split": abi.KERNEL_SPLIT}[which]
        abi.anns_set_option(self.handle, abi.OPT_KERNEL, v)

    def locate(self, queries, nprobe: int, cl: str = "fp32", nprobe_per_q=None, stream=None):
        """Coarse stage alone: (probes int32, probe_d2 float32) CUDA tensors [nq, nprobe]."""
        import torch
        nq = queries.shape[0]
        probes = torch.empty((nq, nprobe), dtype=torch.int32, device=queries.device)
        pd = torch.empty((nq, nprobe), dtype=torch.float32, device=queries.device)
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_locate(self.handle, _ptr(queries), nq, nprobe, _ptr(nprobe_per_q),
                        CL_PREC[cl], _ptr(probes), _ptr(pd), s)
        return probes, pd

    def set_qchunk(self, queries: int):
        """Queries per chunk of the grouped kernel's work order (0 = automatic)."""
        abi.anns_set_option(self.handle, abi.OPT_QCHUNK, int(queries))

    def set_nibble(self, on: bool):
        """Grouped search: pairs on <= 4-bit tables eight to a word (default on)."""
        abi.anns_set_option(self.handle, abi.OPT_NIBBLE, 1 if on else 0)

    def set_schedule(self, which: str):
        """'auto', 'natural' or 'lpt' (longest query first) for the query-major kernel."""
        v = {"auto": abi.SCHED_AUTO, "natural": abi.SCHED_NATURAL, "lpt": abi.SCHED_LPT}[which]
        abi.anns_set_option(self.handle, abi.OPT_SCHEDULE, v)

    def capture_graph(self, queries, nprobe: int, k: int, pol=None, nprobe_per_q=None, k_per_q=None, out=None):
        """CUDA graph of a whole search on fixed CUDA tensors; returns (Graph, ids, dists)."""
        import torch
        nq = queries.shape[0]
        if out is None:
            out = (torch.empty((nq, k), dtype=torch.int64, device=queries.device),
                   torch.empty((nq, k), dtype=torch.float32, device=queries.device))
        ids, dists = out
        h = abi.anns_graph_capture(self.handle, _ptr(queries), nq, nprobe, _ptr(nprobe_per_q), k, _ptr(k_per_q),
                                   pol, _ptr(ids), _ptr(dists))
        return Graph(h), ids, dists

    def autotune(self, queries, nprobe: int, k: int, pol=None, nprobe_per_q=None, k_per_q=None, reps: int = 3):
        """Times every (kernel, schedule, work-order chunk) choice, installs the fastest;
        returns [(kernel, schedule, ms, qchunk)]."""
        return abi.anns_autotune(self.handle, _ptr(queries), queries.shape[0], nprobe, _ptr(nprobe_per_q), k,
                                 _ptr(k_per_q), pol, reps)

    def set_predictor(self, p: dict):
        abi.anns_set_predictor(self.handle, predictor_to_struct(p))

    def get_predictor(self) -> dict:
        return predictor_to_dict(abi.anns_get_predictor(self.handle))

    def set_svr(self, sv, beta, gamma: float, mean, inv_std, table_n: int, table_ratio: float, inv_step: float):
        """Installs an SVR-RBF model for the 'svr' policy (host arrays: sv [nsv, 5], beta [nsv])."""
        sv = np.ascontiguousarray(sv, dtype=np.float32)
        beta = np.ascontiguousarray(beta, dtype=np.float32)
        m = abi.anns_svr_model()
        m.nsv, m.sv, m.beta = len(beta), sv.ctypes.data, beta.ctypes.data
        m.gamma = float(gamma)
        for i in range(5):
            m.mean[i] = float(mean[i])
            m.inv_std[i] = float(inv_std[i])
        m.table_n, m.table_ratio, m.inv_step = int(table_n), float(table_ratio), float(inv_step)
        abi.anns_set_svr(self.handle, m)

    def make_training_set(self, train_q, nprobe: int, k: int, stream=None):
        """Raw features [nq, nprobe, 5] and label bits [nq, nprobe] (CUDA tensors)."""
        import torch
        nq = train_q.shape[0]
        feat = torch.empty((nq, nprobe, 5), dtype=torch.float32, device=train_q.device)
        lab = torch.empty((nq, nprobe), dtype=torch.uint8, device=train_q.device)
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_make_training_set(self.handle, _ptr(train_q), nq, nprobe, k, _ptr(feat), _ptr(lab), s)
        return feat, lab

    def mlp_grad(self, p: dict, X, cls, high_weight: float = 1.0):
        """Gradient (dict of numpy arrays) and mean weighted loss over samples X [n, 5], cls [n] (CUDA tensors)."""
        g = np.empty(1413, dtype=np.float32)
        loss = abi.anns_mlp_grad(self.handle, predictor_to_struct(p), _ptr(X), _ptr(cls), X.shape[0], g.ctypes.data,
                                 high_weight)
        out, o = {}, 0
        for f in _PRED_FIELDS[:6]:
            n = int(np.prod(_PRED_SHAPES[f]))
            out[f] = g[o:o + n].reshape(_PRED_SHAPES[f])
            o += n
        return out, loss

    def mlp_train(self, p: dict, X, cls, cfg) -> dict:
        s = predictor_to_struct(p)
        abi.anns_mlp_train(self.handle, _ptr(X), _ptr(cls), X.shape[0], cfg, s)
        return predictor_to_dict(s)

    def train_predictor(self, train_q, nprobe: int, k: int, cfg) -> dict:
        return predictor_to_dict(abi.anns_train_predictor(self.handle, _ptr(train_q), train_q.shape[0],
                                                          nprobe, k, cfg))

    def tap(self, what: int, shape, dtype):
        out = np.empty(shape, dtype=dtype)
        abi.anns_debug_tap(self.handle, what, out.ctypes.data, out.nbytes)
        return out

    def list_sizes(self):
        return self.tap(abi.TAP_LIST_SIZES, (self.nlist,), np.int64)

    def list_radius(self):
        return self.tap(abi.TAP_LIST_RADIUS, (self.nlist,), np.float32)

    def packed_ids(self):
        return self.tap(abi.TAP_PACKED_IDS, (self.info.n,), np.int64)

    def compute_luts(self, queries, pair_q, pair_l, pair_bits, stream=None):
        """FP32 LUTs, quantised levels and (Delta, B, range, s) for explicit pairs (CUDA tensors)."""
        import torch
        n = pair_q.shape[0]
        dev = queries.device
        T = torch.empty((n, self.M, 256), dtype=torch.float32, device=dev)
        t = torch.empty((n, self.M, 256), dtype=torch.int16, device=dev)
        sc = torch.empty((n, 4), dtype=torch.float64, device=dev)
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_compute_luts(self.handle, _ptr(queries), queries.shape[0], _ptr(pair_q), _ptr(pair_l),
                              _ptr(pair_bits), n, _ptr(T), _ptr(t), _ptr(sc), s)
        return T, t, sc

    def scan_pairs(self, queries, pair_q, pair_l, pair_bits, stream=None):
        """Every distance (and integer sum) of each pair's list, concatenated in pair order."""
        import torch
        sizes = self.list_sizes()
        pl = pair_l.cpu().numpy()
        n_each = sizes[pl]
        off = np.concatenate([[0], np.cumsum(n_each)[:-1]]).astype(np.int64)
        total = int(n_each.sum())
        dev = queries.device
        offt = torch.from_numpy(off).to(dev)
        dist = torch.empty(max(total, 1), dtype=torch.float32, device=dev)
        S = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        abi.anns_scan_pairs(self.handle, _ptr(queries), queries.shape[0], _ptr(pair_q), _ptr(pair_l),
                            _ptr(pair_bits), pair_q.shape[0], _ptr(offt), _ptr(dist), _ptr(S), s)
        return dist[:total], S[:total], off, n_each
