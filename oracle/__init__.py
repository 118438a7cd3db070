"""CPU oracle for stratified k-bisimulation (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports, links or
executes anything here, and nothing here imports the GPU library.

* :func:`refine` -- the plain C++ refinement in ``kbisim_oracle.cpp`` (map of
  (own previous block, sorted unique signature) -> id, vertices visited in id
  order so ids come out canonical).  Paper Section 4.1 (Alg. 1) with the
  signature of Def. "signature" and the definitions of Section 3.2-3.3.
* :mod:`oracle.bruteforce` -- the k-bisimilarity relation iterated pair by
  pair straight from the definitions, for tiny graphs.  It pins the C++
  oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbisim_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

DIR_OUT, DIR_IN, DIR_BOTH = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no CUDA involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_refine_init.restype = ctypes.c_int
            lib.oracle_refine_init.argtypes = [
                ctypes.c_int64, ctypes.c_int64, P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, P, P, P, P,
            ]
            lib.oracle_refine_cse.restype = ctypes.c_int
            lib.oracle_refine_cse.argtypes = [
                ctypes.c_int64, ctypes.c_int64, P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P,
            ]
            lib.oracle_summary.restype = ctypes.c_int64
            lib.oracle_summary.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def refine(n, row_offsets, col, elabel=None, vlabel=None, direction=DIR_OUT, use_vertex_labels=True,
           use_edge_labels=True, k=10, early_stop=True, initial=None, subject=0):
    """Run the oracle.  Returns (levels int32[k+1, n], counts int64[k+1], levels_computed).
    ``subject`` selects the subject part of the key (see oracle_refine_cse)."""
    lib = _load()
    row = np.ascontiguousarray(row_offsets, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    m = int(col.shape[0])
    el = None if elabel is None else np.ascontiguousarray(elabel, dtype=np.int32)
    vl = None if vlabel is None else np.ascontiguousarray(vlabel, dtype=np.int32)
    ini = None if initial is None else np.ascontiguousarray(initial, dtype=np.int32)
    levels = np.zeros((k + 1, max(n, 0)), dtype=np.int32)
    counts = np.zeros(k + 1, dtype=np.int64)
    lc = ctypes.c_int(0)
    rc = lib.oracle_refine_cse(
        int(n), m, _ptr(row), _ptr(col), _ptr(el), _ptr(vl), int(direction), int(bool(use_vertex_labels)),
        int(bool(use_edge_labels)), int(subject), int(k), int(bool(early_stop)), _ptr(ini), _ptr(levels),
        _ptr(counts), ctypes.byref(lc),
    )
    if rc != 0:
        raise ValueError("oracle_refine rejected its arguments")
    return levels, counts, int(lc.value)


def refine_graph(g, direction=DIR_OUT, use_vertex_labels=True, use_edge_labels=True, k=10, early_stop=True,
                 initial=None, subject=0):
    """:func:`refine` on a :class:`graphgen.Graph`."""
    return refine(g.n, g.row_offsets, g.col, g.elabel, g.vlabel, direction, use_vertex_labels,
                  use_edge_labels, k, early_stop, initial, subject)


def summary(g, direction, use_edge_labels, src_level, dst_level):
    """Summary-graph triples of a graph under (src_level, dst_level), as three
    int32 arrays in order of first occurrence (see oracle_summary)."""
    lib = _load()
    row = np.ascontiguousarray(g.row_offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    el = None if g.elabel is None else np.ascontiguousarray(g.elabel, dtype=np.int32)
    a = np.ascontiguousarray(src_level, dtype=np.int32)
    b = np.ascontiguousarray(dst_level, dtype=np.int32)
    m = int(col.shape[0])
    out = [np.zeros(max(m, 1), dtype=np.int32) for _ in range(3)]
    cnt = lib.oracle_summary(int(g.n), _ptr(row), _ptr(col), _ptr(el), int(direction), int(bool(use_edge_labels)),
                             _ptr(a), _ptr(b), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
    if cnt < 0:
        raise ValueError("oracle_summary takes direction out (0) or in (1)")
    return tuple(o[:cnt].copy() for o in out)


def signature(row_offsets, col, elabel, prev, v, direction=DIR_OUT, use_edge_labels=True, in_lists=None):
    """The signature set of one vertex w.r.t. the partition ``prev``
    (Def. "signature"), as a sorted tuple of (d, label, block).  Used by the
    sampled checks at sizes where the full oracle would take too long.
    ``in_lists`` maps a vertex to its (source, label) in-edges when the in
    direction is needed."""
    out = set()
    if direction in (DIR_OUT, DIR_BOTH):
        for e in range(int(row_offsets[v]), int(row_offsets[v + 1])):
            lab = int(elabel[e]) if (use_edge_labels and elabel is not None) else 0
            out.add((0, lab, int(prev[int(col[e])])))
    if direction in (DIR_IN, DIR_BOTH):
        for (u, lab) in in_lists.get(int(v), ()):
            out.add((1, int(lab) if use_edge_labels else 0, int(prev[int(u)])))
    return tuple(sorted(out))
