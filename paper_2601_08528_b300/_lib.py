"""ctypes binding of libsvf.so (include/svf.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
passes pointers and sizes.  There is no fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvf.so")

SVF_OK, SVF_EINVAL, SVF_ECAPACITY, SVF_ECUDA, SVF_ETIMEOUT, SVF_EBOUNDS, SVF_EDEVICE = 0, -1, -2, -3, -4, -5, -6
EMPTY = 0xFFFFFFFF
F32, U8, BF16, FP8 = 0, 1, 2, 3
L2, IP = 0, 1
PRUNE_RNG, PRUNE_RANK = 0, 1
MLP_PARAMS, MLP_PACKED = 1153, 1160

# every symbol include/svf.h declares
SYMBOLS = ["svf_last_error", "svf_buffer_sizes", "svf_create", "svf_destroy", "svf_attach", "svf_build", "svf_search",
           "svf_insert", "svf_delete", "svf_consolidate_sizes", "svf_consolidate_begin", "svf_consolidate_run",
           "svf_consolidate_commit", "svf_consolidate_abort", "svf_sync", "svf_stats", "svf_stats_reset", "svf_encode_bf16",
           "svf_encode_fp8", "svf_knn", "svf_mlp_grad", "svf_mlp_partial_floats", "svf_mlp_adam", "svf_mlp_pack",
           "svf_mlp_forward", "svf_tier_buffer_sizes", "svf_tier_enable", "svf_tier_maintain", "svf_tier_theta", "svf_tier_reset",
           "svf_serve_now", "svf_serve_version_bytes", "svf_serve_start", "svf_serve_submit", "svf_serve_poll", "svf_serve_drain",
           "svf_serve_stop", "svf_knn_tc_scratch_bytes", "svf_knn_tc", "svf_wait_limit", "svf_selftest_wait_timeout",
           "svf_knn_static", "svf_knn_static_capacity", "svf_knn_static_error", "svf_gather_probe"]


class Params(C.Structure):
    _fields_ = [("d", C.c_int32), ("dtype", C.c_int32), ("metric", C.c_int32), ("R", C.c_int32),
                ("n_cap", C.c_int64), ("prune", C.c_int32), ("repair_c", C.c_int32), ("lowp", C.c_int32),
                ("reserved0", C.c_int32), ("seed", C.c_uint64)]


class Sizes(C.Structure):
    _fields_ = [("vecs", C.c_size_t), ("vecs_bf16", C.c_size_t), ("vecs_fp8", C.c_size_t), ("graph", C.c_size_t),
                ("del_bits", C.c_size_t), ("workspace", C.c_size_t), ("status", C.c_size_t)]


class Buffers(C.Structure):
    _fields_ = [("vecs", C.c_void_p), ("vecs_bf16", C.c_void_p), ("vecs_fp8", C.c_void_p), ("graph", C.c_void_p),
                ("del_bits", C.c_void_p), ("workspace", C.c_void_p), ("ws_bytes", C.c_size_t),
                ("status", C.c_void_p), ("status_bytes", C.c_size_t)]


class SearchParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("L", C.c_int32), ("T", C.c_int32), ("precision", C.c_int32),
                ("rerank", C.c_int32), ("t_min", C.c_int32), ("mlp", C.c_void_p), ("z_tau", C.c_float),
                ("hash_log2", C.c_int32), ("qkeys", C.c_void_p), ("seed", C.c_uint64), ("trace_feat", C.c_void_p),
                ("trace_meta", C.c_void_p), ("pool_out", C.c_void_p), ("t_every", C.c_int32),
                ("W", C.c_int32)]


class Counters(C.Structure):
    _fields_ = [("n_used", C.c_int64), ("n_deleted", C.c_int64), ("search_queries", C.c_uint64),
                ("search_iters", C.c_uint64), ("search_evals", C.c_uint64), ("hash_resets", C.c_uint64),
                ("repaired_rows", C.c_uint64), ("reverse_targets", C.c_uint64), ("cache_hits", C.c_uint64),
                ("cache_misses", C.c_uint64), ("promoted", C.c_uint64), ("evicted", C.c_uint64),
                ("build_fallback", C.c_uint64), ("build_tensor_core", C.c_uint64)]


class TierParams(C.Structure):
    _fields_ = [("M", C.c_int64), ("qcap", C.c_uint32), ("promote_batch", C.c_int32), ("sweep", C.c_int32),
                ("alpha", C.c_float), ("beta", C.c_float), ("theta0", C.c_float), ("decay_every", C.c_uint64),
                ("policy", C.c_int32), ("lrfu_lambda", C.c_float)]


TIER_POLICIES = {"wavp": 0, "clock": 1, "lfu": 2, "static": 3, "lru": 4, "lrfu": 5}


class TierSizes(C.Structure):
    _fields_ = [(f, C.c_size_t) for f in ("cache", "map", "owner", "ref", "freq", "ein", "queue", "scratch", "host",
                                          "slot_stat")]


class TierBuffers(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("cache", "map", "owner", "ref", "freq", "ein", "queue", "scratch", "host",
                                          "slot_stat")]


OP_SEARCH, OP_INSERT, OP_DELETE = 0, 1, 2


class ServeCfg(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("n_streams", C.c_int32), ("maintain_every", C.c_int32),
                ("consistency", C.c_int32), ("versions", C.c_void_p), ("versions_bytes", C.c_size_t),
                ("shadow_rows", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("op", C.c_int32), ("count", C.c_int32), ("data", C.c_void_p), ("sp", SearchParams),
                ("out_ids", C.c_void_p), ("out_dist", C.c_void_p), ("out_new_ids", C.c_void_p), ("L_ins", C.c_int32),
                ("T_ins", C.c_int32), ("tag", C.c_uint64), ("t_arrival", C.c_double)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("op", C.c_int32), ("status", C.c_int32), ("epoch", C.c_uint64),
                ("count", C.c_int64), ("t_arrival", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]


class SvfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"svf error {code}: {msg}")
        self.code = code


_lib = None


def load() -> C.CDLL:
    """Load libsvf.so from the package directory (no other location)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2601_08528_b300/build.py (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "svf_last_error": (C.c_char_p, []),
        "svf_buffer_sizes": (I32, [C.POINTER(Params), I64, C.POINTER(Sizes)]),
        "svf_create": (I32, [C.POINTER(Params), C.POINTER(Buffers), C.POINTER(C.c_void_p)]),
        "svf_destroy": (I32, [P]),
        "svf_attach": (I32, [P, I64]),
        "svf_build": (I32, [P, P, I64, P]),
        "svf_search": (I32, [P, P, I64, C.POINTER(SearchParams), P, P, P]),
        "svf_insert": (I32, [P, P, I64, I32, I32, P, P]),
        "svf_delete": (I32, [P, P, I64, P, P]),
        "svf_consolidate_sizes": (I32, [C.POINTER(Params), I64, C.POINTER(C.c_size_t)]),
        "svf_consolidate_begin": (I32, [P, P, C.c_size_t, I64, P]),
        "svf_consolidate_run": (I32, [P, I32, C.POINTER(C.c_int64), P]),
        "svf_consolidate_commit": (I32, [P, P]),
        "svf_consolidate_abort": (I32, [P]),
        "svf_sync": (I32, [P]),
        "svf_stats": (I32, [P, C.POINTER(Counters)]),
        "svf_stats_reset": (I32, [P]),
        "svf_encode_bf16": (I32, [P, I64, I32, P, P]),
        "svf_encode_fp8": (I32, [P, I64, I32, P, I64, P]),
        "svf_knn": (I32, [P, I64, I32, I32, I32, P, I64, P, I32, P, P, P, P]),
        "svf_mlp_grad": (I32, [P, P, I32, P, I64, P, P, P, P, P]),
        "svf_mlp_partial_floats": (I64, [I64]),
        "svf_mlp_adam": (I32, [P, P, P, P, I64, C.c_float, C.c_float, C.c_float, C.c_float, P]),
        "svf_mlp_pack": (I32, [P, P, P]),
        "svf_mlp_forward": (I32, [P, P, I64, P, P]),
        "svf_tier_buffer_sizes": (I32, [C.POINTER(Params), C.POINTER(TierParams), C.POINTER(TierSizes)]),
        "svf_tier_enable": (I32, [P, C.POINTER(TierParams), C.POINTER(TierBuffers), P]),
        "svf_tier_maintain": (I32, [P, C.POINTER(C.c_int64), P]),
        "svf_tier_theta": (C.c_float, [P]),
        "svf_tier_reset": (I32, [P, C.POINTER(TierParams), P]),
        "svf_serve_now": (C.c_double, []),
        "svf_serve_version_bytes": (C.c_size_t, [P, I64]),
        "svf_serve_start": (I32, [P, C.POINTER(ServeCfg), C.POINTER(C.c_void_p)]),
        "svf_serve_submit": (I32, [P, C.POINTER(Request)]),
        "svf_serve_poll": (I32, [P, C.POINTER(Completion), I32, C.POINTER(C.c_int32)]),
        "svf_serve_drain": (I32, [P, C.c_double]),
        "svf_serve_stop": (I32, [P]),
        "svf_knn_tc_scratch_bytes": (C.c_size_t, [I64, I64, I32, I32]),
        "svf_knn_tc": (I32, [P, I64, I32, I32, P, I64, I32, P, C.c_size_t, P, P, C.POINTER(C.c_int64), P]),
        "svf_wait_limit": (C.c_uint32, []),
        "svf_selftest_wait_timeout": (I32, [C.c_uint32, P, C.POINTER(C.c_double), P]),
        "svf_knn_static": (I32, [P, I64, I32, I32, I32, P, I64, P, I32, P, P, P]),
        "svf_knn_static_capacity": (I64, []),
        "svf_knn_static_error": (C.c_char_p, []),
        "svf_gather_probe": (I32, [P, I64, I32, I32, I64, I32, U64, P, C.POINTER(C.c_int64), C.POINTER(C.c_float), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(rc: int) -> None:
    if rc != SVF_OK:
        raise SvfError(rc, load().svf_last_error().decode())
