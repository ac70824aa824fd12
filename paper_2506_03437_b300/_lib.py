"""ctypes binding of the C ABI in include/quake_b300.h (argument marshalling only).

Every function here forwards to the CUDA library; nothing is computed in
Python.  Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA); they must be C-contiguous with the documented dtype.  If the library
is missing the import fails: there is no fallback.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("QK_LIBRARY") or os.path.join(HERE, "libquake_b300.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_DUP_ID, ERR_STATE, ERR_UNSUPPORTED, ERR_INTERNAL, ERR_IO = range(10)
METRIC_L2, METRIC_IP = 0, 1
BETA_TABLE, BETA_EXACT = 0, 1
STORE_F32, STORE_BF16, STORE_FP8 = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT",
                5: "ERR_DUP_ID", 6: "ERR_STATE", 7: "ERR_UNSUPPORTED", 8: "ERR_INTERNAL", 9: "ERR_IO"}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = [
    "qk_config_default", "qk_create", "qk_destroy", "qk_last_error", "qk_build", "qk_load", "qk_set_search_upper",
    "qk_search", "qk_search_scanned", "qk_stats", "qk_insert", "qk_delete", "qk_check", "qk_info", "qk_export_level", "qk_export_quantized", "qk_get_hits", "qk_cap_fraction",
    "qk_kmeans_step", "qk_kmeans_step_noalloc", "qk_maintain", "qk_nearest_centroids",
    "qk_search_nprobe", "qk_search_ratio", "qk_batch_create", "qk_batch_destroy", "qk_batch_get_tiles", "qk_batch_set_tiles",
    "qk_batch_search", "qk_batch_capture", "qk_batch_replay", "qk_batch_autotune", "qk_batch_set_timing",
    "qk_batch_stage_times", "qk_maintain_prepare", "qk_maintain_commit", "qk_profile_scan", "qk_save", "qk_restore",
    "qk_server_config_default", "qk_server_create", "qk_server_destroy", "qk_server_submit_search",
    "qk_server_submit_insert", "qk_server_submit_delete", "qk_server_play", "qk_server_results", "qk_server_drain",
    "qk_server_get_stats", "qk_aps_batch_create", "qk_aps_batch_destroy", "qk_aps_batch_set_rounds",
    "qk_aps_batch_set_tiles", "qk_aps_batch_autotune", "qk_aps_batch_search", "qk_aps_batch_capture", "qk_aps_batch_replay",
    "qk_aps_batch_round_stats", "qk_aps_batch_set_timing", "qk_aps_batch_stage_times",
]


class QkConfig(C.Structure):
    _fields_ = [
        ("d", C.c_int32), ("metric", C.c_int32), ("n_leaf", C.c_int32), ("n_parent", C.c_int32),
        ("kmeans_iters", C.c_int32), ("beta_mode", C.c_int32), ("seed", C.c_uint64),
        ("f_M_leaf", C.c_double), ("f_M_parent", C.c_double), ("tau_rho", C.c_double),
        ("upper_recall", C.c_double), ("storage", C.c_int32), ("rerank", C.c_int32),
    ]


class QkMaintParams(C.Structure):
    _fields_ = [
        ("lambda_sizes", C.POINTER(C.c_double)), ("lambda_us", C.POINTER(C.c_double)),
        ("lambda_points", C.c_int32), ("refine_radius", C.c_int32), ("refine_iters", C.c_int32),
        ("split_iters", C.c_int32), ("s_min", C.c_int32), ("refine", C.c_int32),
        ("tau_us", C.c_double), ("alpha", C.c_double), ("window", C.c_int64),
        ("level_band", C.c_int32), ("level_iters", C.c_int32),
    ]


class QkMaintAction(C.Structure):
    _fields_ = [("level", C.c_int32), ("kind", C.c_int32), ("partition", C.c_int32),
                ("committed", C.c_int32), ("estimate", C.c_double), ("delta", C.c_double)]


class QkBatchTiles(C.Structure):
    _fields_ = [("queries_per_warp", C.c_int32), ("tile_rows", C.c_int32), ("chunk_rows", C.c_int32),
                ("rows_per_thread", C.c_int32)]


class QkServerConfig(C.Structure):
    _fields_ = [("k", C.c_int32), ("recall_target", C.c_float), ("max_batch", C.c_int32), ("streams", C.c_int32),
                ("min_free_bytes", C.c_int64), ("maintain_every", C.c_int64), ("update_batch", C.c_int32),
                ("update_wait_s", C.c_double), ("concurrent_maintenance", C.c_int32),
                ("maint", C.POINTER(QkMaintParams)), ("batched_from", C.c_int32)]


class QkIndexStats(C.Structure):
    _fields_ = [("n_vectors", C.c_int64), ("levels", C.c_int32), ("n_partitions", C.c_int32 * 2),
                ("d", C.c_int32), ("metric", C.c_int32), ("storage", C.c_int32),
                ("min_size", C.c_int32), ("max_size", C.c_int32), ("mean_size", C.c_double),
                ("arena_rows", C.c_int64), ("arena_used", C.c_int64), ("arena_holes", C.c_int64),
                ("arena_free", C.c_int64), ("arena_bytes", C.c_int64), ("hits", C.c_int64 * 2),
                ("queries_seen", C.c_int64), ("version", C.c_uint64), ("searches_in_flight", C.c_int64),
                ("retired_rows", C.c_int64)]


class QkServerStats(C.Structure):
    _fields_ = [("searches", C.c_int64), ("inserts", C.c_int64), ("deletes", C.c_int64), ("batches", C.c_int64),
                ("update_groups", C.c_int64), ("maintenance_passes", C.c_int64), ("update_s", C.c_double),
                ("maintenance_stall_s", C.c_double), ("maintenance_prepare_s", C.c_double)]


class QkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2506_03437_b300.build")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, f32, f64 = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_double
    sig = {
        "qk_set_search_upper": (i32, [vp, i32]),
        "qk_config_default": (None, [C.POINTER(QkConfig)]),
        "qk_create": (i32, [C.POINTER(QkConfig), C.POINTER(vp)]),
        "qk_destroy": (None, [vp]),
        "qk_last_error": (C.c_char_p, []),
        "qk_build": (i32, [vp, vp, vp, i64, vp]),
        "qk_load": (i32, [vp, vp, vp, i64, vp, vp, vp, vp, vp]),
        "qk_search": (i32, [vp, vp, i64, i32, f32, i32, vp, vp, vp, vp, vp]),
        "qk_search_scanned": (i32, [vp, vp, i64, i32, f32, i32, vp, vp, vp, vp, vp, i32, vp, i32, vp]),
        "qk_stats": (i32, [vp, C.POINTER(QkIndexStats)]),
        "qk_check": (i32, [vp, vp]),
        "qk_info": (i32, [vp, vp, vp, vp, vp]),
        "qk_insert": (i32, [vp, vp, vp, i64, vp]),
        "qk_delete": (i32, [vp, vp, i64, vp, vp]),
        "qk_export_level": (i32, [vp, i32, vp, vp, vp, vp]),
        "qk_export_quantized": (i32, [vp, vp, vp]),
        "qk_get_hits": (i32, [vp, i32, vp, i32]),
        "qk_cap_fraction": (i32, [i32, i32, vp, vp, i64, vp, vp]),
        "qk_kmeans_step": (i32, [vp, i64, i32, vp, i32, vp, vp, vp, vp]),
        "qk_nearest_centroids": (i32, [vp, i64, i32, vp, i32, i32, i32, vp, vp, vp]),
        "qk_kmeans_step_noalloc": (i32, [vp, i64, i32, vp, i32, vp, vp, vp, vp]),
        "qk_maintain": (i32, [vp, C.POINTER(QkMaintParams), C.POINTER(QkMaintAction), i32,
                              C.POINTER(C.c_int32), vp]),
        "qk_search_nprobe": (i32, [vp, vp, i64, i32, vp, vp, vp, vp]),
        "qk_search_ratio": (i32, [vp, vp, i64, i32, f32, vp, vp, vp, vp, i32, vp]),
        "qk_maintain_prepare": (i32, [vp, C.POINTER(QkMaintParams), C.POINTER(QkMaintAction), i32,
                                      C.POINTER(C.c_int32), vp]),
        "qk_maintain_commit": (i32, [vp, vp]),
        "qk_profile_scan": (i32, [vp, i32, vp, i32, i32, vp, vp]),
        "qk_save": (i32, [vp, C.c_char_p]),
        "qk_restore": (i32, [C.c_char_p, vp, vp]),
        "qk_server_config_default": (None, [C.POINTER(QkServerConfig)]),
        "qk_server_create": (i32, [vp, C.POINTER(QkServerConfig), C.POINTER(vp)]),
        "qk_server_destroy": (None, [vp]),
        "qk_server_submit_search": (i32, [vp, vp, C.POINTER(C.c_int64)]),
        "qk_server_submit_insert": (i32, [vp, vp, i64, C.POINTER(C.c_int64)]),
        "qk_server_submit_delete": (i32, [vp, i64, C.POINTER(C.c_int64)]),
        "qk_server_play": (i32, [vp, i64, vp, vp, vp, vp, vp]),
        "qk_server_results": (i32, [vp, i64, i64, vp, vp, vp, vp]),
        "qk_server_drain": (i32, [vp, f64]),
        "qk_server_get_stats": (i32, [vp, C.POINTER(QkServerStats)]),
        "qk_batch_create": (i32, [vp, i64, i32, i32, C.POINTER(vp)]),
        "qk_batch_destroy": (None, [vp]),
        "qk_batch_get_tiles": (i32, [vp, C.POINTER(QkBatchTiles)]),
        "qk_batch_set_tiles": (i32, [vp, C.POINTER(QkBatchTiles)]),
        "qk_batch_search": (i32, [vp, vp, i64, vp, vp, vp, vp]),
        "qk_batch_capture": (i32, [vp, vp, i64, vp, vp, vp, vp]),
        "qk_batch_replay": (i32, [vp, vp]),
        "qk_batch_set_timing": (i32, [vp, i32]),
        "qk_batch_stage_times": (i32, [vp, vp]),
        "qk_batch_autotune": (i32, [vp, vp, i64, vp, vp, vp, i32, C.POINTER(QkBatchTiles), vp]),
        "qk_aps_batch_create": (i32, [vp, i64, i32, C.POINTER(vp)]),
        "qk_aps_batch_destroy": (None, [vp]),
        "qk_aps_batch_set_rounds": (i32, [vp, i32]),
        "qk_aps_batch_set_tiles": (i32, [vp, C.POINTER(QkBatchTiles)]),
        "qk_aps_batch_autotune": (i32, [vp, vp, i64, C.c_float, vp, vp, i32, C.POINTER(QkBatchTiles), vp]),
        "qk_aps_batch_search": (i32, [vp, vp, i64, f32, vp, vp, vp, vp, vp, i32, vp]),
        "qk_aps_batch_capture": (i32, [vp, vp, i64, f32, vp, vp, vp, vp, vp]),
        "qk_aps_batch_replay": (i32, [vp, vp]),
        "qk_aps_batch_round_stats": (i32, [vp, vp, vp]),
        "qk_aps_batch_set_timing": (i32, [vp, i32]),
        "qk_aps_batch_stage_times": (i32, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def check(status):
    if status != OK:
        raise QkError(status, lib.qk_last_error().decode())


def ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)
