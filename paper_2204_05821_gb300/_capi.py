"""ctypes declarations mirroring include/kbisim.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

KB_OK = 0
KB_ERR_INVALID_ARG = 1
KB_ERR_OOM = 2
KB_ERR_TABLE_FULL = 3
KB_ERR_TIMEOUT = 4
KB_ERR_CUDA = 5
KB_ERR_DEVICE_CHECK = 6
KB_ERR_NOT_FOUND = 7

KB_DIR_OUT, KB_DIR_IN, KB_DIR_BOTH = 0, 1, 2
KB_SUBJECT_PREVIOUS, KB_SUBJECT_ALL, KB_SUBJECT_LABEL, KB_SUBJECT_ID = 0, 1, 2, 3
KB_KERNEL_COUNT = 6
KERNEL_NAMES = ("small", "medium", "hub_chunk", "hub_final", "renumber", "other")


class KbGraph(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("row_offsets", ctypes.c_void_p),
        ("col_indices", ctypes.c_void_p),
        ("edge_labels", ctypes.c_void_p),
        ("vertex_labels", ctypes.c_void_p),
    ]


class KbOptions(ctypes.Structure):
    _fields_ = [
        ("direction", ctypes.c_int32),
        ("use_vertex_labels", ctypes.c_int32),
        ("use_edge_labels", ctypes.c_int32),
        ("early_stop", ctypes.c_int32),
        ("load_factor", ctypes.c_float),
        ("hub_threshold", ctypes.c_int32),
        ("hash_mode", ctypes.c_int32),
        ("validate", ctypes.c_int32),
        ("small_task_vertices", ctypes.c_int32),
        ("reorder", ctypes.c_int32),
        ("subject", ctypes.c_int32),
        ("rekey_all", ctypes.c_int32),
        ("hub_chunk_edges", ctypes.c_int32),
        ("medium_split", ctypes.c_int32),
        ("small_max_degree", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class KbPreparedInfo(ctypes.Structure):
    _fields_ = [
        ("device_bytes", ctypes.c_size_t),
        ("n_hubs", ctypes.c_int64),
        ("n_hub_chunks", ctypes.c_int64),
        ("n_medium", ctypes.c_int64),
        ("reorder", ctypes.c_int32),
        ("hub_threshold", ctypes.c_int32),
        ("small_max_degree", ctypes.c_int32),
        ("hub_chunk_edges", ctypes.c_int32),
        ("build_ms", ctypes.c_float),
        ("reserved", ctypes.c_int32 * 3),
    ]


class KbTuning(ctypes.Structure):
    _fields_ = [
        ("load_factor", ctypes.c_float),
        ("hub_threshold", ctypes.c_int32),
        ("small_task_vertices", ctypes.c_int32),
        ("hub_chunk_edges", ctypes.c_int32),
        ("medium_split", ctypes.c_int32),
        ("small_max_degree", ctypes.c_int32),
        ("ms", ctypes.c_float),
        ("default_ms", ctypes.c_float),
        ("size_class", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


class KbServerConfig(ctypes.Structure):
    _fields_ = [
        ("max_vertices", ctypes.c_int64),
        ("max_edges", ctypes.c_int64),
        ("max_requests", ctypes.c_int32),
        ("hub_threshold", ctypes.c_int32),
        ("memory_budget", ctypes.c_size_t),
        ("load_factor", ctypes.c_float),
        ("hash_mode", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 6),
    ]


class KbServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("running", ctypes.c_int64),
        ("waiting", ctypes.c_int64),
        ("steps", ctypes.c_int64),
        ("compactions", ctypes.c_int64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double),
        ("requests_per_s", ctypes.c_double),
        ("edge_rounds_per_s", ctypes.c_double),
        ("failed", ctypes.c_int64),
    ]


# (name, restype, argtypes) for every symbol the header declares
_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
SIGNATURES = [
    ("kb_options_default", KbOptions, []),
    ("kb_options_schaetzle", KbOptions, []),
    ("kb_options_kaushik", KbOptions, []),
    ("kb_status_string", ctypes.c_char_p, [_I]),
    ("kb_create", _I, [ctypes.POINTER(_P), _I, _P]),
    ("kb_destroy", _I, [_P]),
    ("kb_last_error", ctypes.c_char_p, [_P]),
    ("kb_workspace_size", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _I,
                               ctypes.POINTER(ctypes.c_size_t)]),
    ("kb_set_workspace", _I, [_P, _P, ctypes.c_size_t]),
    ("kb_refine", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _I, _P, _P, _P]),
    ("kb_refine_from", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _P, _I, _I, _P, _P, _P]),
    ("kb_refine_host", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _I, _P, _P, _P]),
    ("kb_refine_fixpoint", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _P, _I, _P, _P, _P, _P]),
    ("kb_summary", _I, [_P, ctypes.POINTER(KbGraph), _I, _I, _P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    ("kb_graph_prepare", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), ctypes.POINTER(_P)]),
    ("kb_graph_release", _I, [_P]),
    ("kb_prepared_get_info", _I, [_P, ctypes.POINTER(KbPreparedInfo)]),
    ("kb_refine_prepared", _I, [_P, _P, ctypes.POINTER(KbOptions), _I, _P, _P, _P]),
    ("kb_refine_update", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _I, _P, ctypes.c_int64, _P, _P,
                              _P, _P]),
    ("kb_set_timing", _I, [_P, _I]),
    ("kb_get_timing", _I, [_P, _P, _I, _P, _P, _P]),
    ("kb_get_round_work", _I, [_P, _P, _P, _I, _P]),
    ("kb_refine_batch", _I, [_P, ctypes.POINTER(KbGraph), _P, _I64, _P, ctypes.POINTER(KbOptions), _P, _P, _P]),
    ("kb_autotune", _I, [_P, ctypes.POINTER(KbGraph), _P, _I64, _P, ctypes.POINTER(KbOptions), _I,
                         ctypes.POINTER(KbTuning)]),
    ("kb_clear_tuning", _I, [_P]),
    ("kb_server_config_default", KbServerConfig, []),
    ("kb_server_create", _I, [ctypes.POINTER(_P), _I, _P, ctypes.POINTER(KbServerConfig)]),
    ("kb_server_destroy", _I, [_P]),
    ("kb_server_last_error", ctypes.c_char_p, [_P]),
    ("kb_server_submit", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _I, _P,
                          ctypes.POINTER(_I64)]),
    ("kb_server_step", _I, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    ("kb_server_poll", _I, [_P, _I64, ctypes.POINTER(_I32)]),
    ("kb_server_fetch", _I, [_P, _I64, _P, _P, ctypes.POINTER(_I32)]),
    ("kb_server_get_stats", _I, [_P, ctypes.POINTER(KbServerStats)]),
    ("kb_refine_round_noalloc", _I, [_P, ctypes.POINTER(KbGraph), ctypes.POINTER(KbOptions), _P, _P,
                                     ctypes.POINTER(ctypes.c_int64)]),
]
NOALLOC_MAX_VERTICES = 1 << 20

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libkbisim.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libkbisim.so is not built; run paper_2204_05821_gb300._build.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class KbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (status_name(status), message))
        self.status = status


def status_name(status: int) -> str:
    return load().kb_status_string(int(status)).decode()


def check(status: int, ctx=None):
    if status != KB_OK:
        msg = load().kb_last_error(ctx).decode() if ctx else ""
        raise KbError(status, msg)
