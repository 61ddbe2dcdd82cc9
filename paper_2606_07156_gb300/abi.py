"""ctypes binding of include/anns_amp.h — argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the search: device buffers are passed as raw pointers (torch
tensors are used only to own device memory). If the shared library is
missing, importing this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libanns_amp.so")

ANNS_OK = 0
STATIC_SCRATCH_FLOATS = 1 << 21
MAX_M, MAX_NPROBE, MAX_K = 128, 128, 128
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "UNSUPPORTED"}
LUT_PLAIN_FP32, LUT_FIXED_BITS, LUT_HEURISTIC_EQ2, LUT_MLP, LUT_EXPLICIT, LUT_SVR = 0, 1, 2, 3, 4, 5
PREC_FP32, PREC_BF16, PREC_FP8E4M3, PREC_FP16 = 0, 1, 2, 3
TAP_PROBES, TAP_PROBE_D2, TAP_BITS, TAP_FEATURES = 0, 1, 2, 3
TAP_COARSE_APPROX, TAP_COARSE_CANDIDATES = 4, 5
TAP_LIST_SIZES, TAP_LIST_RADIUS, TAP_PACKED_IDS, TAP_STATUS = 10, 11, 12, 13
OPT_KERNEL, OPT_SCHEDULE, OPT_QCHUNK, OPT_WAIT_CYCLES, OPT_NIBBLE = 0, 1, 2, 3, 4
KERNEL_AUTO, KERNEL_BASIC, KERNEL_LIST_MAJOR, KERNEL_GROUPED, KERNEL_SPLIT = 0, 1, 2, 3, 4
SCHED_AUTO, SCHED_NATURAL, SCHED_LPT = 0, 1, 2

SYMBOLS = (
    "anns_build_index_from_arrays", "anns_free", "anns_search", "anns_search_host",
    "anns_get_info", "anns_debug_tap", "anns_compute_luts", "anns_scan_pairs", "anns_profile",
    "anns_set_option", "anns_locate_static", "anns_set_predictor", "anns_get_predictor",
    "anns_make_training_set", "anns_mlp_grad", "anns_mlp_train", "anns_train_predictor",
    "anns_graph_capture", "anns_graph_launch", "anns_graph_free", "anns_autotune", "anns_locate",
    "anns_kernel_launches", "anns_svr_fit", "anns_debug_exact_sum", "anns_sync_status", "anns_set_svr", "anns_train_index", "anns_export_index", "anns_save",
    "anns_load", "anns_build_subspaces", "anns_subspace_sizes", "anns_search_subspace", "anns_last_error",
)


class AnnsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class anns_build_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int64), ("nlist", ctypes.c_int64),
                ("M", ctypes.c_int64), ("ksub", ctypes.c_int64),
                ("centroids", ctypes.c_void_p), ("codebooks", ctypes.c_void_p),
                ("codes", ctypes.c_void_p), ("list_of", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("device", ctypes.c_int32)]


class anns_precision_policy(ctypes.Structure):
    _fields_ = [("lut_mode", ctypes.c_int32), ("fixed_bits", ctypes.c_int32),
                ("cl_prec", ctypes.c_int32), ("lc_prec", ctypes.c_int32),
                ("eq2_thresholds", ctypes.c_float * 4), ("fallback_margin", ctypes.c_float),
                ("pair_bits", ctypes.c_void_p), ("width_map", ctypes.c_int32)]


class anns_index_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int64), ("nlist", ctypes.c_int64),
                ("M", ctypes.c_int64), ("dsub", ctypes.c_int64), ("Mp", ctypes.c_int64),
                ("code_bytes", ctypes.c_int64), ("max_list", ctypes.c_int64),
                ("device", ctypes.c_int32)]


class anns_predictor(ctypes.Structure):
    _fields_ = [("W1", ctypes.c_float * 160), ("b1", ctypes.c_float * 32), ("W2", ctypes.c_float * 1024),
                ("b2", ctypes.c_float * 32), ("W3", ctypes.c_float * 160), ("b3", ctypes.c_float * 5),
                ("mean", ctypes.c_float * 5), ("inv_std", ctypes.c_float * 5)]


class anns_svr_model(ctypes.Structure):
    _fields_ = [("nsv", ctypes.c_int32), ("sv", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("gamma", ctypes.c_float), ("mean", ctypes.c_float * 5), ("inv_std", ctypes.c_float * 5),
                ("table_n", ctypes.c_int32), ("table_ratio", ctypes.c_double), ("inv_step", ctypes.c_float)]


class anns_train_desc(ctypes.Structure):
    _fields_ = [("nlist", ctypes.c_int64), ("M", ctypes.c_int64), ("iters", ctypes.c_int32),
                ("pq_iters", ctypes.c_int32), ("seed", ctypes.c_uint64), ("per_centroid", ctypes.c_int64),
                ("pq_sample", ctypes.c_int64)]


class anns_subspace_desc(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_int32), ("K", ctypes.c_int32), ("K_lc", ctypes.c_int32), ("iters", ctypes.c_int32)]


class anns_subspace_policy(ctypes.Structure):
    _fields_ = [("th_cl", ctypes.c_float * 3), ("th_lc", ctypes.c_float * 3), ("cl", ctypes.c_int32),
                ("lc", ctypes.c_int32)]


class anns_tune_result(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("schedule", ctypes.c_int32), ("ms", ctypes.c_float),
                ("qchunk", ctypes.c_int64)]


class anns_train_cfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("label_map", ctypes.c_int32), ("high_weight", ctypes.c_float)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2606_07156_gb300.build.build() "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
    sig = {
        "anns_build_index_from_arrays": ([ctypes.POINTER(anns_build_desc), ctypes.POINTER(vp)], i32),
        "anns_free": ([vp], None),
        "anns_search": ([vp, vp, i64, i32, vp, i32, vp, ctypes.POINTER(anns_precision_policy), vp, vp, vp], i32),
        "anns_search_host": ([vp, vp, i64, i32, vp, i32, vp, ctypes.POINTER(anns_precision_policy), vp, vp, vp], i32),
        "anns_get_info": ([vp, ctypes.POINTER(anns_index_info)], i32),
        "anns_debug_tap": ([vp, i32, vp, sz], i32),
        "anns_compute_luts": ([vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp], i32),
        "anns_scan_pairs": ([vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp], i32),
        "anns_profile": ([vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)], i32),
        "anns_kernel_launches": ([], i64),
        "anns_debug_exact_sum": ([vp, i64, i32, vp, vp], i32),
        "anns_sync_status": ([vp, vp], i32),
        "anns_set_svr": ([vp, ctypes.POINTER(anns_svr_model)], i32),
        "anns_train_index": ([vp, i64, i64, ctypes.POINTER(anns_train_desc), i32, i32, ctypes.POINTER(vp)], i32),
        "anns_export_index": ([vp, vp, vp, vp, vp, vp], i32),
        "anns_save": ([vp, ctypes.c_char_p], i32),
        "anns_build_subspaces": ([vp, ctypes.POINTER(anns_subspace_desc)], i32),
        "anns_subspace_sizes": ([vp, vp, vp], i32),
        "anns_search_subspace": ([vp, vp, i64, i32, i32, ctypes.POINTER(anns_subspace_policy), vp, vp, vp, vp], i32),
        "anns_load": ([ctypes.c_char_p, i32, ctypes.POINTER(vp)], i32),
        "anns_svr_fit": ([vp, vp, i64, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, i64,
                          vp, ctypes.POINTER(i64)], i32),
        "anns_set_option": ([vp, i32, i64], i32),
        "anns_locate_static": ([vp, vp, i64, i32, vp, vp, vp], i32),
        "anns_graph_capture": ([vp, vp, i64, i32, vp, i32, vp, ctypes.POINTER(anns_precision_policy), vp, vp,
                                ctypes.POINTER(vp)], i32),
        "anns_graph_launch": ([vp, vp], i32),
        "anns_locate": ([vp, vp, i64, i32, vp, i32, vp, vp, vp], i32),
        "anns_graph_free": ([vp], None),
        "anns_autotune": ([vp, vp, i64, i32, vp, i32, vp, ctypes.POINTER(anns_precision_policy), i32,
                           ctypes.POINTER(anns_tune_result), i32, ctypes.POINTER(i32), vp], i32),
        "anns_set_predictor": ([vp, ctypes.POINTER(anns_predictor)], i32),
        "anns_get_predictor": ([vp, ctypes.POINTER(anns_predictor)], i32),
        "anns_make_training_set": ([vp, vp, i64, i32, i32, vp, vp, vp], i32),
        "anns_mlp_grad": ([vp, ctypes.POINTER(anns_predictor), vp, vp, i64, ctypes.c_float, vp,
                           ctypes.POINTER(ctypes.c_double), vp], i32),
        "anns_mlp_train": ([vp, vp, vp, i64, ctypes.POINTER(anns_train_cfg), ctypes.POINTER(anns_predictor), vp], i32),
        "anns_train_predictor": ([vp, vp, i64, i32, i32, ctypes.POINTER(anns_train_cfg), ctypes.POINTER(anns_predictor), vp], i32),
        "anns_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def anns_last_error() -> str:
    return _lib.anns_last_error().decode()


def _check(rc: int):
    if rc != ANNS_OK:
        raise AnnsError(rc, anns_last_error())


def anns_build_index_from_arrays(desc: anns_build_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.anns_build_index_from_arrays(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def anns_free(index: int) -> None:
    _lib.anns_free(index)


def anns_search(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q, policy, ids_out, dists_out,
                stream=None) -> None:
    _check(_lib.anns_search(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q,
                            ctypes.byref(policy) if policy is not None else None,
                            ids_out, dists_out, stream))


def anns_search_host(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q, policy, ids_out,
                     dists_out, stream=None) -> None:
    _check(_lib.anns_search_host(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q,
                                 ctypes.byref(policy) if policy is not None else None,
                                 ids_out, dists_out, stream))


def anns_get_info(index) -> anns_index_info:
    info = anns_index_info()
    _check(_lib.anns_get_info(index, ctypes.byref(info)))
    return info


def anns_debug_tap(index, what: int, out_ptr: int, nbytes: int) -> None:
    _check(_lib.anns_debug_tap(index, what, out_ptr, nbytes))


def anns_compute_luts(index, queries, nq, pair_q, pair_l, pair_bits, npairs, T_out, t_out, scale_out,
                      stream=None) -> None:
    _check(_lib.anns_compute_luts(index, queries, nq, pair_q, pair_l, pair_bits, npairs,
                                  T_out, t_out, scale_out, stream))


def anns_scan_pairs(index, queries, nq, pair_q, pair_l, pair_bits, npairs, out_off, dist_out, S_out,
                    stream=None) -> None:
    _check(_lib.anns_scan_pairs(index, queries, nq, pair_q, pair_l, pair_bits, npairs,
                                out_off, dist_out, S_out, stream))


def anns_debug_exact_sum(vals, nsets, n, out, stream=None) -> None:
    """Per set of n device FP32 values, the exact sum rounded once to FP32 (the offset rule)."""
    _check(_lib.anns_debug_exact_sum(vals, nsets, n, out, stream))


PROFILE_STAGES = 7  # CL distances, CL selection, precision + query tables, search up to the
# grouped kernels, the grouped byte-table kernel, the grouped nibble kernel, the grouped merge


def anns_profile(index, enable: int):
    """Returns (ms per stage [PROFILE_STAGES], number of searches) accumulated since recording started."""
    ms = (ctypes.c_double * PROFILE_STAGES)()
    cnt = ctypes.c_int64()
    _check(_lib.anns_profile(index, enable, ms, ctypes.byref(cnt)))
    return list(ms), cnt.value


SVR_MAX_SAMPLES = 4096


def anns_svr_fit(X, y, C: float, gamma: float, eps: float, tol: float = 1e-10, max_sweeps: int = 10000):
    """SVR-RBF training on the host (numpy float64 X [n, dim], y [n]) -> (beta [n], sweeps)."""
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n, dim = X.shape
    beta = np.zeros(n, dtype=np.float64)
    sweeps = ctypes.c_int64()
    _check(_lib.anns_svr_fit(X.ctypes.data, y.ctypes.data, n, dim, C, gamma, eps, tol, max_sweeps,
                             beta.ctypes.data, ctypes.byref(sweeps)))
    return beta, sweeps.value


def anns_kernel_launches() -> int:
    """Kernels the library has enqueued since it was loaded (host-side count)."""
    return int(_lib.anns_kernel_launches())


def anns_train_index(base_ptr, n, dim, desc: "anns_train_desc", on_device: int, device: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.anns_train_index(base_ptr, n, dim, ctypes.byref(desc), on_device, device, ctypes.byref(h)))
    return h.value


def anns_export_index(index, centroids, codebooks, codes, ids, list_len) -> None:
    _check(_lib.anns_export_index(index, centroids, codebooks, codes, ids, list_len))


def anns_build_subspaces(index, desc: "anns_subspace_desc") -> None:
    _check(_lib.anns_build_subspaces(index, ctypes.byref(desc)))


def anns_subspace_sizes(index, cl_size, lc_size) -> None:
    _check(_lib.anns_subspace_sizes(index, cl_size, lc_size))


def anns_search_subspace(index, queries, nq, nprobe, k, policy: "anns_subspace_policy", ids_out, dists_out,
                         low_counts=None, stream=None) -> None:
    _check(_lib.anns_search_subspace(index, queries, nq, nprobe, k, ctypes.byref(policy), ids_out, dists_out,
                                     low_counts, stream))


def anns_save(index, path: str) -> None:
    _check(_lib.anns_save(index, path.encode()))


def anns_load(path: str, device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_lib.anns_load(path.encode(), device, ctypes.byref(h)))
    return h.value


def anns_set_svr(index, model: "anns_svr_model") -> None:
    _check(_lib.anns_set_svr(index, ctypes.byref(model)))


def anns_sync_status(index, stream=None) -> None:
    """Waits for the stream; raises AnnsError(TIMEOUT) if a bounded wait in a kernel ran out."""
    _check(_lib.anns_sync_status(index, stream))


def anns_set_option(index, option: int, value: int) -> None:
    _check(_lib.anns_set_option(index, option, value))


def anns_locate_static(index, queries, nq, nprobe, probes_out, probe_d2_out, stream=None) -> None:
    """Coarse stage with the library's fixed scratch array: no device allocation."""
    _check(_lib.anns_locate_static(index, queries, nq, nprobe, probes_out, probe_d2_out, stream))


def anns_set_predictor(index, pred: "anns_predictor") -> None:
    _check(_lib.anns_set_predictor(index, ctypes.byref(pred)))


def anns_get_predictor(index) -> "anns_predictor":
    out = anns_predictor()
    _check(_lib.anns_get_predictor(index, ctypes.byref(out)))
    return out


def anns_make_training_set(index, train_q, nq, nprobe, k, feat_out, label_out, stream=None) -> None:
    _check(_lib.anns_make_training_set(index, train_q, nq, nprobe, k, feat_out, label_out, stream))


def anns_mlp_grad(index, pred, X, cls, n, grad_out, high_weight=1.0, stream=None) -> float:
    loss = ctypes.c_double()
    _check(_lib.anns_mlp_grad(index, ctypes.byref(pred), X, cls, n, high_weight, grad_out, ctypes.byref(loss),
                              stream))
    return loss.value


def anns_mlp_train(index, X, cls, n, cfg, pred, stream=None) -> None:
    _check(_lib.anns_mlp_train(index, X, cls, n, ctypes.byref(cfg), ctypes.byref(pred), stream))


def anns_train_predictor(index, train_q, nq, nprobe, k, cfg, out=None, stream=None) -> "anns_predictor":
    out = out if out is not None else anns_predictor()
    _check(_lib.anns_train_predictor(index, train_q, nq, nprobe, k, ctypes.byref(cfg), ctypes.byref(out), stream))
    return out


def anns_graph_capture(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q, policy, ids_out, dists_out):
    out = ctypes.c_void_p()
    pol = ctypes.byref(policy) if policy is not None else None
    _check(_lib.anns_graph_capture(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q, pol, ids_out,
                                   dists_out, ctypes.byref(out)))
    return out.value


def anns_graph_launch(graph, stream=None) -> None:
    _check(_lib.anns_graph_launch(graph, stream))


def anns_graph_free(graph) -> None:
    _lib.anns_graph_free(graph)


def anns_autotune(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q, policy, reps, stream=None):
    res = (anns_tune_result * 16)()
    n = ctypes.c_int32()
    pol = ctypes.byref(policy) if policy is not None else None
    _check(_lib.anns_autotune(index, queries, nq, nprobe, nprobe_per_q, k, k_per_q, pol, reps, res, 16,
                              ctypes.byref(n), stream))
    return [(res[i].kernel, res[i].schedule, res[i].ms, res[i].qchunk) for i in range(n.value)]


def anns_locate(index, queries, nq, nprobe, nprobe_per_q, cl_prec, probes_out, probe_d2_out, stream=None) -> None:
    _check(_lib.anns_locate(index, queries, nq, nprobe, nprobe_per_q, cl_prec, probes_out, probe_d2_out, stream))
