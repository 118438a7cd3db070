"""GB300 stratified k-bisimulation by signature refinement.

Thin Python binding over the C ABI in ``include/kbisim.h`` (argument
marshalling only: every step of every refinement round runs in the CUDA
kernels of ``libkbisim.so``).  PyTorch provides device memory and streams.

Method: paper Section 4.1 (Alg. 1) with the signature of Def. "signature" and
the equivalences of Sections 3.2-3.3.  Levels come back with canonical block
ids (blocks numbered by their smallest member vertex).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _capi
from ._capi import KB_DIR_BOTH as DIR_BOTH
from ._capi import KB_DIR_IN as DIR_IN
from ._capi import KB_DIR_OUT as DIR_OUT
from ._capi import KB_SUBJECT_ALL as SUBJECT_ALL
from ._capi import KB_SUBJECT_ID as SUBJECT_ID
from ._capi import KB_SUBJECT_LABEL as SUBJECT_LABEL
from ._capi import KB_SUBJECT_PREVIOUS as SUBJECT_PREVIOUS
from ._capi import KbError

__all__ = [
    "DIR_OUT", "DIR_IN", "DIR_BOTH", "SUBJECT_PREVIOUS", "SUBJECT_ALL", "SUBJECT_LABEL", "SUBJECT_ID", "Options", "DeviceGraph", "Context", "Result", "KbError", "refine",
    "refine_round_noalloc", "library_path", "Server",
]


def library_path() -> str:
    return _capi.library_path()


@dataclass
class Options:
    """Mirror of ``kb_options`` (see include/kbisim.h for every field)."""

    direction: int = DIR_OUT
    use_vertex_labels: bool = True
    use_edge_labels: bool = True
    early_stop: bool = True
    load_factor: float = 0.0
    hub_threshold: int = 0
    hash_mode: int = 0
    validate: bool = True
    small_task_vertices: int = 0
    reorder: int = 0  # 0 automatic, 1 off, 2 on
    subject: int = 0  # SUBJECT_PREVIOUS, SUBJECT_ALL, SUBJECT_LABEL or SUBJECT_ID (generic CSE rounds)
    rekey_all: bool = False  # True: re-key every vertex every round (no skipping of frozen blocks)
    hub_chunk_edges: int = 0  # 0 or 256, 512, 1024
    medium_split: int = 0  # 0 or 1..256
    small_max_degree: int = 0  # 0 or 1..32

    @classmethod
    def schaetzle(cls, **kw) -> "Options":
        """Edge-labelled forward bisimulation (Def. "edge-labeled-fw-bisimulation")."""
        return cls(direction=DIR_OUT, use_vertex_labels=False, use_edge_labels=True, **kw)

    @classmethod
    def kaushik(cls, **kw) -> "Options":
        """Vertex-labelled backward bisimulation (Def. "vertex-labeled-bw-bisimulation")."""
        return cls(direction=DIR_IN, use_vertex_labels=True, use_edge_labels=False, **kw)

    def to_c(self) -> _capi.KbOptions:
        o = _capi.load().kb_options_default()
        o.direction = int(self.direction)
        o.use_vertex_labels = int(bool(self.use_vertex_labels))
        o.use_edge_labels = int(bool(self.use_edge_labels))
        o.early_stop = int(bool(self.early_stop))
        o.load_factor = float(self.load_factor)
        o.hub_threshold = int(self.hub_threshold)
        o.hash_mode = int(self.hash_mode)
        o.validate = int(bool(self.validate))
        o.small_task_vertices = int(self.small_task_vertices)
        o.reorder = int(self.reorder)
        o.subject = int(self.subject)
        o.rekey_all = int(bool(self.rekey_all))
        o.hub_chunk_edges = int(self.hub_chunk_edges)
        o.medium_split = int(self.medium_split)
        o.small_max_degree = int(self.small_max_degree)
        return o


class PreparedGraph:
    """A graph prepared by ``Context.prepare`` (``kb_graph_prepare``)."""

    def __init__(self, lib, handle, graph, options):
        self._lib = lib
        self._h = handle
        self.graph = graph  # keeps the tensors alive
        self.options = options

    @property
    def handle(self):
        if not self._h.value:
            raise KbError(1, "prepared graph released")
        return self._h

    def info(self) -> dict:
        i = _capi.KbPreparedInfo()
        _capi.check(self._lib.kb_prepared_get_info(self.handle, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in _capi.KbPreparedInfo._fields_ if name != "reserved"}

    def release(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.kb_graph_release(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.release()


class DeviceGraph:
    """A CSR graph held in torch tensors on one CUDA device.

    row_offsets int64[n+1], col int32[m], elabel int32[m] or None,
    vlabel int32[n] or None (the layout of ``kb_graph``)."""

    def __init__(self, row_offsets, col, elabel=None, vlabel=None):
        import torch

        self.row_offsets = row_offsets
        self.col = col
        self.elabel = elabel
        self.vlabel = vlabel
        self.n = int(row_offsets.shape[0]) - 1
        self.m = int(col.shape[0])
        for name, t, dt in (("row_offsets", row_offsets, torch.int64), ("col", col, torch.int32),
                            ("elabel", elabel, torch.int32), ("vlabel", vlabel, torch.int32)):
            if t is None:
                continue
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dt))

    @classmethod
    def from_numpy(cls, g, device="cuda") -> "DeviceGraph":
        import torch

        def t(a):
            return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)

        return cls(t(g.row_offsets.astype(np.int64)), t(g.col.astype(np.int32)),
                   t(None if g.elabel is None else g.elabel.astype(np.int32)),
                   t(None if g.vlabel is None else g.vlabel.astype(np.int32)))

    @classmethod
    def from_tensors(cls, d: dict) -> "DeviceGraph":
        return cls(d["row_offsets"], d["col"], d.get("elabel"), d.get("vlabel"))

    def to_c(self) -> _capi.KbGraph:
        def p(t):
            return None if t is None else t.data_ptr()

        return _capi.KbGraph(self.n, self.m, p(self.row_offsets), p(self.col), p(self.elabel), p(self.vlabel))

    @property
    def device(self):
        return self.row_offsets.device


@dataclass
class Result:
    levels: "object"  # torch int32 [k+1, n] on the device (numpy for host calls)
    counts: np.ndarray  # int64 [k+1]
    levels_computed: int


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """A ``kb_context``: one device, one stream, cached scratch."""

    def __init__(self, device: int = 0, stream=None, torch_workspace: bool = False):
        import torch

        self._lib = _capi.load()
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        _capi.check(self._lib.kb_create(ctypes.byref(h), self.device, ctypes.c_void_p(stream.cuda_stream)))
        self._h = h
        self._torch_ws = torch_workspace
        self._ws = None
        self._ws_key = None

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.kb_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        _capi.check(st, self._h)

    # -- scratch
    def workspace_size(self, graph: DeviceGraph, k: int, options: Options = None) -> int:
        options = options or Options()
        g, o = graph.to_c(), options.to_c()
        b = ctypes.c_size_t(0)
        self._check(self._lib.kb_workspace_size(self._h, ctypes.byref(g), ctypes.byref(o), int(k), ctypes.byref(b)))
        return int(b.value)

    def _prepare_workspace(self, graph: DeviceGraph, k: int, options: Options):
        if not self._torch_ws:
            return
        import torch

        key = (graph.row_offsets.data_ptr(), graph.n, graph.m, options.direction, options.hub_threshold,
               options.load_factor, options.use_edge_labels, options.reorder, options.subject,
               bool(options.rekey_all), k)
        if self._ws is not None and self._ws_key == key:
            return
        need = self.workspace_size(graph, k, options)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=graph.device)
        self._ws_key = key
        self._check(self._lib.kb_set_workspace(self._h, ctypes.c_void_p(self._ws.data_ptr()),
                                               self._ws.numel()))

    # -- prepared graphs
    def prepare(self, graph: DeviceGraph, options: Options = None) -> "PreparedGraph":
        """``kb_graph_prepare``: the per-graph structures of every refinement
        call (validation, processed CSR, degree classes, hub plan, edgeless
        bits, locality order), built once.  Pass the result to ``refine`` in
        place of the graph.  The graph's tensors must stay unchanged while it
        lives (the prepared graph keeps a reference to them)."""
        options = options or Options()
        g, o = graph.to_c(), options.to_c()
        h = ctypes.c_void_p()
        self._check(self._lib.kb_graph_prepare(self._h, ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)))
        return PreparedGraph(self._lib, h, graph, options)

    # -- refinement
    def refine(self, graph, k: int, options: Options = None, out=None) -> Result:
        """``kb_refine`` of a DeviceGraph, or ``kb_refine_prepared`` of a
        PreparedGraph (``options`` then defaults to the preparation's)."""
        import torch

        prepared = isinstance(graph, PreparedGraph)
        if prepared:
            options = options or graph.options
            dg = graph.graph
        else:
            options = options or Options()
            dg = graph
            self._prepare_workspace(graph, k, options)
        levels = out if out is not None else torch.empty((k + 1, dg.n), dtype=torch.int32, device=dg.device)
        counts = np.zeros(k + 1, dtype=np.int64)
        lc = ctypes.c_int(0)
        o = options.to_c()
        if prepared:
            self._check(self._lib.kb_refine_prepared(self._h, graph.handle, ctypes.byref(o), int(k),
                                                     ctypes.c_void_p(levels.data_ptr()), _np_ptr(counts),
                                                     ctypes.byref(lc)))
        else:
            g = dg.to_c()
            self._check(self._lib.kb_refine(self._h, ctypes.byref(g), ctypes.byref(o), int(k),
                                            ctypes.c_void_p(levels.data_ptr()), _np_ptr(counts), ctypes.byref(lc)))
        return Result(levels, counts, int(lc.value))

    def refine_from(self, graph: DeviceGraph, start, i_start: int, k: int, options: Options = None,
                    levels=None, counts=None) -> Result:
        import torch

        options = options or Options()
        self._prepare_workspace(graph, k, options)
        if levels is None:
            levels = torch.zeros((k + 1, graph.n), dtype=torch.int32, device=graph.device)
        if counts is None:
            counts = np.zeros(k + 1, dtype=np.int64)
        lc = ctypes.c_int(0)
        g, o = graph.to_c(), options.to_c()
        self._check(self._lib.kb_refine_from(self._h, ctypes.byref(g), ctypes.byref(o),
                                             ctypes.c_void_p(start.data_ptr()), int(i_start), int(k),
                                             ctypes.c_void_p(levels.data_ptr()), _np_ptr(counts), ctypes.byref(lc)))
        return Result(levels, counts, int(lc.value))

    def refine_fixpoint(self, graph: DeviceGraph, max_rounds: int, options: Options = None, initial=None, out=None):
        """kb_refine_fixpoint: refine until stable (full bisimulation, or the
        coarsest stable refinement of ``initial``).  Returns
        ``(final_level, count, rounds, stable)``."""
        import torch

        options = options or Options()
        self._prepare_workspace(graph, max_rounds, options)
        final = out if out is not None else torch.empty(graph.n, dtype=torch.int32, device=graph.device)
        cnt, rounds, stable = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_int(0)
        g, o = graph.to_c(), options.to_c()
        init = ctypes.c_void_p(initial.data_ptr()) if initial is not None else None
        self._check(self._lib.kb_refine_fixpoint(self._h, ctypes.byref(g), ctypes.byref(o), init, int(max_rounds),
                                                 ctypes.c_void_p(final.data_ptr()), ctypes.byref(cnt),
                                                 ctypes.byref(rounds), ctypes.byref(stable)))
        return final, int(cnt.value), int(rounds.value), bool(stable.value)

    def summary(self, graph: DeviceGraph, src_level, dst_level=None, direction: int = DIR_OUT,
                use_edge_labels: bool = True, capacity: int = None):
        """kb_summary: the summary graph of (src_level, dst_level) as three
        int32 device tensors (source block, label, target block) in order of
        first occurrence.  dst_level defaults to src_level (quotient graph)."""
        import torch

        if dst_level is None:
            dst_level = src_level
        cap = graph.m if capacity is None else int(capacity)
        outs = [torch.empty(max(cap, 1), dtype=torch.int32, device=graph.device) for _ in range(3)]
        cnt = ctypes.c_int64(0)
        g = graph.to_c()
        self._check(self._lib.kb_summary(self._h, ctypes.byref(g), int(direction), int(bool(use_edge_labels)),
                                         ctypes.c_void_p(src_level.data_ptr()), ctypes.c_void_p(dst_level.data_ptr()),
                                         *[ctypes.c_void_p(o.data_ptr()) for o in outs], cap, ctypes.byref(cnt)))
        c = int(cnt.value)
        return tuple(o[:c] for o in outs)

    def summary_count(self, graph: DeviceGraph, src_level, dst_level=None, direction: int = DIR_OUT,
                      use_edge_labels: bool = True) -> int:
        """Number of summary edges only (kb_summary with capacity 0)."""
        if dst_level is None:
            dst_level = src_level
        cnt = ctypes.c_int64(0)
        g = graph.to_c()
        st = self._lib.kb_summary(self._h, ctypes.byref(g), int(direction), int(bool(use_edge_labels)),
                                  ctypes.c_void_p(src_level.data_ptr()), ctypes.c_void_p(dst_level.data_ptr()),
                                  None, None, None, 0, ctypes.byref(cnt))
        if st != 0 and not (st == 1 and cnt.value > 0):
            self._check(st)
        return int(cnt.value)

    def refine_update(self, graph: DeviceGraph, levels, changed, options: Options = None):
        """kb_refine_update: ``levels`` (a [k+1, n] int32 device tensor holding the
        levels of the graph before the change, same options) is updated in place
        to the levels of ``graph``; ``changed`` is an int32 device tensor of the
        vertices whose edge lists changed.  Returns ``(Result, work)`` with the
        vertices re-keyed per level."""
        options = options or Options()
        k = int(levels.shape[0]) - 1
        counts = np.zeros(k + 1, dtype=np.int64)
        work = np.zeros(k + 1, dtype=np.int64)
        lc = ctypes.c_int(0)
        g, o = graph.to_c(), options.to_c()
        ch = ctypes.c_void_p(changed.data_ptr()) if changed is not None and changed.numel() else None
        nch = int(changed.numel()) if changed is not None else 0
        self._check(self._lib.kb_refine_update(self._h, ctypes.byref(g), ctypes.byref(o), k, ch, nch,
                                               ctypes.c_void_p(levels.data_ptr()), _np_ptr(counts), ctypes.byref(lc),
                                               _np_ptr(work)))
        return Result(levels, counts, int(lc.value)), work

    def refine_host(self, row_offsets, col, elabel, vlabel, k: int, options: Options = None, out=None) -> Result:
        """kb_refine_host: numpy (ideally pinned) host arrays in and out."""
        options = options or Options()
        row_offsets = np.ascontiguousarray(row_offsets, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n, m = row_offsets.shape[0] - 1, col.shape[0]
        el = None if elabel is None else np.ascontiguousarray(elabel, dtype=np.int32)
        vl = None if vlabel is None else np.ascontiguousarray(vlabel, dtype=np.int32)
        levels = out if out is not None else np.empty((k + 1, n), dtype=np.int32)
        counts = np.zeros(k + 1, dtype=np.int64)
        lc = ctypes.c_int(0)
        g = _capi.KbGraph(n, m, _np_ptr(row_offsets), _np_ptr(col), _np_ptr(el), _np_ptr(vl))
        o = options.to_c()
        self._check(self._lib.kb_refine_host(self._h, ctypes.byref(g), ctypes.byref(o), int(k), _np_ptr(levels),
                                             _np_ptr(counts), ctypes.byref(lc)))
        return Result(levels, counts, int(lc.value))

    def refine_batch(self, union: DeviceGraph, vertex_offsets: Sequence[int], ks: Sequence[int],
                     options: Options = None) -> Tuple[object, np.ndarray, np.ndarray]:
        """kb_refine_batch over a disjoint union.  Returns (levels [k_max+1, n]
        with graph-local ids, counts [G, k_max+1], levels_computed [G])."""
        import torch

        options = options or Options()
        voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        G = int(ks.shape[0])
        kmax = int(ks.max()) if G else 0
        levels = torch.empty((kmax + 1, union.n), dtype=torch.int32, device=union.device)
        counts = np.zeros((G, kmax + 1), dtype=np.int64)
        lc = np.zeros(G, dtype=np.int32)
        g, o = union.to_c(), options.to_c()
        self._check(self._lib.kb_refine_batch(self._h, ctypes.byref(g), _np_ptr(voff), G, _np_ptr(ks),
                                              ctypes.byref(o), ctypes.c_void_p(levels.data_ptr()), _np_ptr(counts),
                                              _np_ptr(lc)))
        return levels, counts, lc

    def autotune(self, graph: DeviceGraph, options: Options = None, rounds: int = 2, vertex_offsets=None,
                 ks=None) -> dict:
        """``kb_autotune``: time ``rounds`` rounds of ``graph`` (or, with
        ``vertex_offsets``, kb_refine_batch of the union with k = ``rounds`` or
        ``ks`` per graph) over the tuning fields, cache the choice in this
        context for the call's size class and return it as a dict (the
        kb_tuning fields: the chosen values, ``ms`` and ``default_ms``)."""
        options = options or Options()
        g, o = graph.to_c(), options.to_c()
        t = _capi.KbTuning()
        voff_p, G, ks_p = None, 0, None
        if vertex_offsets is not None:
            voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
            G = voff.shape[0] - 1
            voff_p = _np_ptr(voff)
            if ks is not None:
                ks = np.ascontiguousarray(ks, dtype=np.int32)
                if ks.shape[0] != G:
                    raise ValueError("ks needs one entry per graph")
                ks_p = _np_ptr(ks)
        self._check(self._lib.kb_autotune(self._h, ctypes.byref(g), voff_p, G, ks_p, ctypes.byref(o), int(rounds),
                                          ctypes.byref(t)))
        return {name: (float(getattr(t, name)) if name in ("load_factor", "ms", "default_ms") else
                       int(getattr(t, name))) for name, _ in _capi.KbTuning._fields_ if name != "reserved"}

    def clear_tuning(self):
        """Forget every tuning ``autotune`` cached in this context."""
        self._check(self._lib.kb_clear_tuning(self._h))

    # -- timing
    def set_timing(self, enable=True):
        """0/False: off; 1/True: CUDA events per round and kernel family;
        2: also the vertices and edges every round re-keys (round_work())."""
        self._check(self._lib.kb_set_timing(self._h, int(enable)))

    def round_work(self):
        """Per round of the last refinement call (``kb_get_round_work``): a
        dict of vertices and edges re-keyed by the small, medium and hub
        kernels, e.g. {"small": (v, e), "medium": (v, e), "hub": (v, e)}."""
        nr = ctypes.c_int(0)
        v = np.zeros(3 * 4096, dtype=np.int64)
        e = np.zeros(3 * 4096, dtype=np.int64)
        self._check(self._lib.kb_get_round_work(self._h, _np_ptr(v), _np_ptr(e), 4096, ctypes.byref(nr)))
        fam = ("small", "medium", "hub")
        return [{fam[f]: (int(v[3 * i + f]), int(e[3 * i + f])) for f in range(3)} for i in range(nr.value)]

    def timing(self):
        """(round_ms list, {kernel family: (ms, launches)}) of the last call."""
        nr = ctypes.c_int(0)
        rm = np.zeros(4096, dtype=np.float32)
        km = np.zeros(_capi.KB_KERNEL_COUNT, dtype=np.float32)
        kl = np.zeros(_capi.KB_KERNEL_COUNT, dtype=np.int64)
        self._check(self._lib.kb_get_timing(self._h, _np_ptr(rm), 4096, ctypes.byref(nr), _np_ptr(km), _np_ptr(kl)))
        fam = {name: (float(km[i]), int(kl[i])) for i, name in enumerate(_capi.KERNEL_NAMES)}
        return rm[: nr.value].tolist(), fam


class Server:
    """Continuous-batching summarisation server (``kb_server_*`` in the C ABI).

    ``submit`` queues a host graph (numpy CSR; the arrays are kept referenced
    until the request is fetched, since the library reads them at admission)
    with a host array for its levels; every ``step`` admits what fits (arena
    space, request slots, device memory), runs one refinement round for all
    in-flight requests at once and retires finished ones.  ``fetch`` returns
    (levels [k+1, n], counts, levels_computed), or raises KbError for a
    request rejected at admission (state FAILED)."""

    WAITING, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, device: int = 0, stream=None, max_vertices: int = 1 << 26, max_edges: int = 1 << 28,
                 max_requests: int = 256, memory_budget: int = 0, load_factor: float = 0.0,
                 hub_threshold: int = 0, hash_mode: int = 0):
        import torch

        self._lib = _capi.load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        cfg = self._lib.kb_server_config_default()
        cfg.max_vertices, cfg.max_edges, cfg.max_requests = int(max_vertices), int(max_edges), int(max_requests)
        cfg.memory_budget, cfg.load_factor = int(memory_budget), float(load_factor)
        cfg.hub_threshold, cfg.hash_mode = int(hub_threshold), int(hash_mode)
        h = ctypes.c_void_p()
        _capi.check(self._lib.kb_server_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream.cuda_stream),
                                                ctypes.byref(cfg)))
        self._h = h
        self._meta = {}

    def _check(self, st):
        if st != _capi.KB_OK:
            raise KbError(st, self._lib.kb_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.kb_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, row_offsets, col, elabel, vlabel, k: int, options: Options = None, out=None) -> int:
        """Queue a request; ``out`` (int32 [k+1, n], C-contiguous) receives
        its levels when it finishes (a new array when None)."""
        options = options or Options()
        row = np.ascontiguousarray(row_offsets, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        el = None if elabel is None else np.ascontiguousarray(elabel, dtype=np.int32)
        vl = None if vlabel is None else np.ascontiguousarray(vlabel, dtype=np.int32)
        n = row.shape[0] - 1
        g = _capi.KbGraph(n, col.shape[0], _np_ptr(row), _np_ptr(col), _np_ptr(el), _np_ptr(vl))
        o = options.to_c()
        t = ctypes.c_int64(0)
        levels = out if out is not None else np.empty((int(k) + 1, n), dtype=np.int32)
        if levels.dtype != np.int32 or levels.shape != (int(k) + 1, n) or not levels.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous int32 array of shape (k+1, n)")
        self._check(self._lib.kb_server_submit(self._h, ctypes.byref(g), ctypes.byref(o), int(k), _np_ptr(levels),
                                               ctypes.byref(t)))
        self._meta[t.value] = (levels, (row, col, el, vl))
        return int(t.value)

    def submit_graph(self, g, k: int, options: Options = None) -> int:
        return self.submit(g.row_offsets, g.col, g.elabel, g.vlabel, k, options)

    def step(self):
        """One scheduling step; returns (running, waiting)."""
        r, w = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._lib.kb_server_step(self._h, ctypes.byref(r), ctypes.byref(w)))
        return int(r.value), int(w.value)

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int32(0)
        self._check(self._lib.kb_server_poll(self._h, int(ticket), ctypes.byref(st)))
        return int(st.value)

    def fetch(self, ticket: int):
        levels, _graph = self._meta.pop(ticket)
        counts = np.zeros(levels.shape[0], dtype=np.int64)
        lc = ctypes.c_int32(0)
        self._check(self._lib.kb_server_fetch(self._h, int(ticket), _np_ptr(levels), _np_ptr(counts), ctypes.byref(lc)))
        return levels, counts, int(lc.value)

    def stats(self) -> dict:
        st = _capi.KbServerStats()
        self._check(self._lib.kb_server_get_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in _capi.KbServerStats._fields_}


def refine_round_noalloc(graph: DeviceGraph, prev, out, options: Options = None, stream=None) -> int:
    """One refinement round (level i from level i-1, out-edges) through
    ``kb_refine_round_noalloc``: the library allocates no device memory for
    it, using a fixed static scratch array instead (n <= 2^20, no vertex above
    the hub threshold).  ``prev`` and ``out`` are contiguous int32 CUDA tensors
    of length n on the graph's device.  Returns the number of blocks of the new
    level."""
    import torch

    options = options or Options()
    for name, t in (("prev", prev), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != torch.int32 or not t.is_contiguous() or t.numel() != graph.n or t.device != graph.device:
            raise ValueError("%s must be a contiguous int32 tensor of %d entries on %s (got %s, %d entries on %s)"
                             % (name, graph.n, graph.device, t.dtype, t.numel(), t.device))
    with torch.cuda.device(graph.device):
        if stream is None:
            stream = torch.cuda.current_stream(graph.device)
        lib = _capi.load()
        cnt = ctypes.c_int64(0)
        g, o = graph.to_c(), options.to_c()
        st = lib.kb_refine_round_noalloc(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(g), ctypes.byref(o),
                                         ctypes.c_void_p(prev.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.byref(cnt))
    if st != _capi.KB_OK:
        raise KbError(st, "kb_refine_round_noalloc")
    return int(cnt.value)


_default = {}


def refine(graph: DeviceGraph, k: int, options: Options = None) -> Result:
    """Refine with a per-device default context on the current stream."""
    dev = graph.device.index or 0
    ctx = _default.get(dev)
    if ctx is None:
        ctx = _default[dev] = Context(dev)
    return ctx.refine(graph, k, options)
