"""Multi-core CPU baseline for k-bisimulation (OpenMP, all host cores).

A comparison point for the GPU library, not part of it and not the oracle:
``kbisim_omp.cpp`` builds every vertex's signature in parallel and assigns
canonical ids through a parallel sort with full signature compares (paper
Section 4.1, Alg. 1; Def. "signature").  Tests check it against the oracle;
``bench.py`` times it beside the single-threaded oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbisim_omp.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkbisim_omp.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile with the host C++ compiler and OpenMP (no CUDA involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.cpu_parallel_refine.restype = ctypes.c_int
            lib.cpu_parallel_refine.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.cpu_parallel_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads a call uses (OMP_NUM_THREADS, else every host core)."""
    return int(_load().cpu_parallel_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def refine(n, row_offsets, col, elabel=None, vlabel=None, direction=0, use_vertex_labels=True,
           use_edge_labels=True, k=10, early_stop=True):
    """Levels 0..k.  Returns (levels int32[k+1, n], counts int64[k+1], levels_computed)."""
    lib = _load()
    row = np.ascontiguousarray(row_offsets, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    el = None if elabel is None else np.ascontiguousarray(elabel, dtype=np.int32)
    vl = None if vlabel is None else np.ascontiguousarray(vlabel, dtype=np.int32)
    levels = np.zeros((k + 1, max(n, 0)), dtype=np.int32)
    counts = np.zeros(k + 1, dtype=np.int64)
    lc = ctypes.c_int(0)
    rc = lib.cpu_parallel_refine(int(n), int(col.shape[0]), _ptr(row), _ptr(col), _ptr(el), _ptr(vl),
                                 int(direction), int(bool(use_vertex_labels)), int(bool(use_edge_labels)), int(k),
                                 int(bool(early_stop)), _ptr(levels), _ptr(counts), ctypes.byref(lc))
    if rc != 0:
        raise ValueError("cpu_parallel_refine rejected its arguments")
    return levels, counts, int(lc.value)


def refine_graph(g, direction=0, use_vertex_labels=True, use_edge_labels=True, k=10, early_stop=True):
    """:func:`refine` on a :class:`graphgen.Graph`."""
    return refine(g.n, g.row_offsets, g.col, g.elabel, g.vlabel, direction, use_vertex_labels, use_edge_labels,
                  k, early_stop)
