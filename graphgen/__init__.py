"""Seeded synthetic labelled directed graphs in CSR form.

This module only draws random graphs; it contains none of the refinement
arithmetic.  Both the CPU oracle tests and the CUDA path take their inputs
from here, so the two sides always see identical graphs for a given seed.

The paper evaluates on RDF dumps (Laundromat, BTC2019) and BSBM output
(Section 5.1, Table "statistics-datasets"), none of which ship with this
project.  The generators below stand in for them with the shapes the paper
reports: power-law out/in degrees with a few very large hubs, Zipf-distributed
vertex and edge labels, self loops and parallel edges kept.

All CSR graphs use: ``row_offsets`` int64[n+1] (monotone, row_offsets[0]=0,
row_offsets[n]=m), ``col`` int32[m] (out-neighbour of each edge),
``elabel`` int32[m], ``vlabel`` int32[n].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Graph",
    "from_edges",
    "erdos_renyi",
    "chung_lu",
    "chung_lu_torch",
    "zipf_labels",
    "paper_example",
    "tiny_random",
    "batch_workload",
    "serve_workload",
    "disjoint_union",
    "path_graph",
    "cycle_graph",
    "binary_tree",
    "CONFIG_TINY",
    "CONFIG_RDF",
    "CONFIG_LARGE",
]


@dataclass
class Graph:
    """A labelled directed multigraph in out-edge CSR form (numpy arrays)."""

    n: int
    m: int
    row_offsets: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[m]
    elabel: np.ndarray  # int32[m]
    vlabel: np.ndarray  # int32[n]
    names: Optional[List[str]] = field(default=None, repr=False)

    def edges(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(src, dst, label) arrays in CSR order."""
        deg = np.diff(self.row_offsets)
        src = np.repeat(np.arange(self.n, dtype=np.int64), deg)
        return src, self.col.astype(np.int64), self.elabel.copy()


# --------------------------------------------------------------------------
# CSR construction helpers
# --------------------------------------------------------------------------


def from_edges(n: int, src, dst, elabel=None, vlabel=None, names=None) -> Graph:
    """Build a CSR graph from an edge list (stable order within a source)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    m = int(src.shape[0])
    if elabel is None:
        elabel = np.zeros(m, dtype=np.int32)
    if vlabel is None:
        vlabel = np.zeros(n, dtype=np.int32)
    order = np.argsort(src, kind="stable")
    deg = np.bincount(src, minlength=n).astype(np.int64)
    row = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row[1:])
    return Graph(
        n=n,
        m=m,
        row_offsets=row,
        col=dst[order].astype(np.int32),
        elabel=np.asarray(elabel, dtype=np.int32)[order],
        vlabel=np.asarray(vlabel, dtype=np.int32),
        names=names,
    )


def _rows_from_degrees(deg: np.ndarray) -> np.ndarray:
    row = np.zeros(deg.shape[0] + 1, dtype=np.int64)
    np.cumsum(deg, out=row[1:])
    return row


# --------------------------------------------------------------------------
# Counter-based random numbers, identical in numpy and torch
# --------------------------------------------------------------------------
#
# Draw i of stream s under seed S is fmix64(key(S, s) + (i + 1) * W) mod 2^64:
# a Weyl sequence with increment W = floor(2^64 / golden ratio) passed through
# the 64-bit finalizer of MurmurHash3 (Austin Appleby, public domain).  Only
# wrapping 64-bit integer multiply, add, xor and shifts are involved, so numpy
# (uint64) and torch (int64, logical shifts emulated) give the same bits on
# any machine, and a graph drawn on the GPU equals the one drawn on the host.
_W = 0x9E3779B97F4A7C15
_F1 = 0xFF51AFD7ED558CCD
_F2 = 0xC4CEB9FE1A85EC53
_MASK64 = (1 << 64) - 1
_CHUNK = 1 << 24

# streams of the power-law recipe
_S_OUT, _S_PERM_OUT, _S_PERM_IN, _S_IN, _S_ELABEL, _S_VLABEL = range(6)


def _fmix64(x: int) -> int:
    x &= _MASK64
    x ^= x >> 33
    x = (x * _F1) & _MASK64
    x ^= x >> 33
    x = (x * _F2) & _MASK64
    x ^= x >> 33
    return x


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of random stream ``stream`` under ``seed``."""
    return _fmix64(_fmix64(int(seed) * _W + 0x632BE59BD9B4E019) ^ (int(stream) * 0xD6E8FEB86659FD93))


def ctr_bits(key: int, a: int, b: int) -> np.ndarray:
    """Draws a..b-1 of the stream with this key, as uint64 (numpy)."""
    i = np.arange(a + 1, b + 1, dtype=np.uint64)
    x = i * np.uint64(_W) + np.uint64(key)
    x ^= x >> np.uint64(33)
    x *= np.uint64(_F1)
    x ^= x >> np.uint64(33)
    x *= np.uint64(_F2)
    x ^= x >> np.uint64(33)
    return x


def ctr_uniform(key: int, a: int, b: int) -> np.ndarray:
    """Draws a..b-1 as float64 in [0, 1): the top 53 bits times 2^-53 (exact)."""
    return (ctr_bits(key, a, b) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(x, s: int):
    """Logical right shift of an int64 torch tensor."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def ctr_bits_torch(key: int, a: int, b: int, device):
    """:func:`ctr_bits` with torch on ``device``, as int64 holding the same bits."""
    import torch

    x = torch.arange(a + 1, b + 1, dtype=torch.int64, device=device) * _i64(_W) + _i64(key)
    x ^= _srl(x, 33)
    x *= _i64(_F1)
    x ^= _srl(x, 33)
    x *= _i64(_F2)
    x ^= _srl(x, 33)
    return x


def ctr_uniform_torch(key: int, a: int, b: int, device):
    import torch

    return _srl(ctr_bits_torch(key, a, b, device), 11).to(torch.float64) * (2.0 ** -53)


# --------------------------------------------------------------------------
# Platform-independent power-law weights
# --------------------------------------------------------------------------
#
# A graph is drawn by inverting cumulative distributions, so a weight that
# differs in its last bit between two machines moves draws from one vertex to
# another.  libm's pow and numpy's SIMD pow are not bit-identical across
# platforms, so the weights r^-a are computed here with correctly rounded basic
# operations only (numpy never fuses them): ln r from frexp and the series
# ln f = 2 atanh((f-1)/(f+1)), exp by reduction to exp(t) 2^k and Taylor's
# series, and every sum is a sequential cumulative sum.
_LN2 = 0.6931471805599453


def _det_log(x: np.ndarray) -> np.ndarray:
    f, e = np.frexp(x)
    low = f < 0.7071067811865476
    f = np.where(low, f * 2.0, f)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (f - 1.0) / (f + 1.0)  # |s| < 0.172
    s2 = s * s
    acc = np.full_like(s, 1.0 / 29.0)
    for j in range(13, -1, -1):
        acc = acc * s2 + 1.0 / (2 * j + 1)
    return e * _LN2 + 2.0 * s * acc


def _det_exp(y: np.ndarray) -> np.ndarray:
    k = np.rint(y / _LN2)
    t = y - k * _LN2  # |t| <= ~0.35
    fact = [1.0]
    for j in range(1, 19):
        fact.append(fact[-1] * j)
    acc = np.full_like(t, 1.0 / fact[18])
    for j in range(17, -1, -1):
        acc = acc * t + 1.0 / fact[j]
    return np.ldexp(acc, k.astype(np.int64))


def det_pow(x: np.ndarray, a: float) -> np.ndarray:
    """x^a for positive float64 x, bit-identical on every platform (relative
    error about 1e-15)."""
    return _det_exp(a * _det_log(np.asarray(x, dtype=np.float64)))


def _seqsum(x: np.ndarray) -> float:
    return float(np.cumsum(x)[-1]) if x.shape[0] else 0.0


def _capped_powerlaw_degrees(n: int, m: int, gamma: float, cap: float) -> np.ndarray:
    """Chung-Lu expected degrees: rank r (1-based) gets weight r^(-1/(gamma-1)),
    scaled to sum m, with the largest clipped at ``cap`` and the remainder
    rescaled so the total stays m."""
    r = np.arange(1, n + 1, dtype=np.float64)
    w = det_pow(r, -1.0 / (gamma - 1.0))
    d = w * (m / _seqsum(w))
    for _ in range(50):
        over = d > cap
        if not over.any():
            break
        d[over] = cap
        free = ~over
        rest = m - cap * float(np.count_nonzero(over))
        d[free] *= rest / _seqsum(d[free])
    return d


def _cdf(weights: np.ndarray) -> np.ndarray:
    c = np.cumsum(weights)
    c /= c[-1]
    return c


def _zipf_cdf(n_labels: int, s: float) -> np.ndarray:
    return _cdf(det_pow(np.arange(1, max(1, n_labels) + 1, dtype=np.float64), -s))


def _pool_map(fn, spans):
    """Run fn(a, b) over spans on host threads (numpy releases the GIL in the
    loops used here); every span writes only its own slice."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    workers = max(1, min(len(spans), os.cpu_count() or 1))
    if workers == 1:
        for a, b in spans:
            fn(a, b)
        return
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(lambda ab: fn(*ab), spans))


def _spans(count: int):
    return [(a, min(count, a + _CHUNK)) for a in range(0, count, _CHUNK)]


def _inverse_cdf(cdf: np.ndarray, key: int, count: int, out: np.ndarray) -> None:
    """out[i] = the bin of draw i: the first j with cdf[j] > u_i (clipped)."""
    last = cdf.shape[0] - 1

    def work(a, b):
        out[a:b] = np.minimum(np.searchsorted(cdf, ctr_uniform(key, a, b), side="right"), last)

    _pool_map(work, _spans(count))


def _random_permutation(key: int, n: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1: the stable argsort of n
    random 63-bit keys."""
    keys = np.empty(n, dtype=np.int64)

    def work(a, b):
        keys[a:b] = (ctr_bits(key, a, b) >> np.uint64(1)).astype(np.int64)

    _pool_map(work, _spans(n))
    return np.argsort(keys, kind="stable")


def zipf_labels(seed: int, stream: int, count: int, n_labels: int, s: float) -> np.ndarray:
    """Labels 0..n_labels-1 with P(label = j) proportional to (j+1)^-s."""
    out = np.zeros(count, dtype=np.int32)
    if n_labels > 1:
        _inverse_cdf(_zipf_cdf(n_labels, s), stream_key(seed, stream), count, out)
    return out


# --------------------------------------------------------------------------
# Workload generators
# --------------------------------------------------------------------------


def erdos_renyi(n: int, m: int, n_vlabels: int, n_elabels: int, seed: int) -> Graph:
    """Directed Erdos-Renyi multigraph: m edges with source and target uniform
    (with replacement; self loops and parallel edges kept); vertex and edge
    labels uniform over 0..n_vlabels-1 and 0..n_elabels-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    src = rng.integers(0, n, size=m, dtype=np.int64)
    dst = rng.integers(0, n, size=m, dtype=np.int64)
    el = rng.integers(0, max(1, n_elabels), size=m, dtype=np.int64).astype(np.int32)
    vl = rng.integers(0, max(1, n_vlabels), size=n, dtype=np.int64).astype(np.int32)
    return from_edges(n, src, dst, el, vl)


def chung_lu(
    n: int,
    m: int,
    gamma_out: float,
    gamma_in: float,
    max_out_deg: float,
    max_in_deg: float,
    n_vlabels: int,
    zipf_v: float,
    n_elabels: int,
    zipf_e: float,
    seed: int,
) -> Graph:
    """Power-law directed multigraph (static Chung-Lu model).

    Out-degrees are one multinomial draw of m edges over the capped
    out-weights (m independent draws of a source rank, counted); every edge's
    target is drawn independently from the capped in-weights ("preferential by
    in-degree").  Out-rank and in-rank are mapped to vertex ids by two
    independent random permutations, so hub ids carry no locality.  Vertices
    that draw no out-edges are the "literal" sinks of RDF data.  All draws come
    from the counter-based streams above: :func:`chung_lu_torch` with the same
    arguments returns the identical graph.
    """
    cdf_out = _cdf(_capped_powerlaw_degrees(n, m, gamma_out, max_out_deg))
    ranks = np.empty(m, dtype=np.int32)
    _inverse_cdf(cdf_out, stream_key(seed, _S_OUT), m, ranks)
    deg_rank = np.bincount(ranks, minlength=n).astype(np.int64)
    del ranks, cdf_out
    perm_out = _random_permutation(stream_key(seed, _S_PERM_OUT), n)
    deg = np.empty(n, dtype=np.int64)
    deg[perm_out] = deg_rank
    del perm_out, deg_rank
    row = _rows_from_degrees(deg)
    del deg

    cdf_in = _cdf(_capped_powerlaw_degrees(n, m, gamma_in, max_in_deg))
    perm_in = _random_permutation(stream_key(seed, _S_PERM_IN), n).astype(np.int32)
    col = np.empty(m, dtype=np.int32)
    _inverse_cdf(cdf_in, stream_key(seed, _S_IN), m, col)
    del cdf_in

    def remap(a, b):
        col[a:b] = perm_in[col[a:b]]

    _pool_map(remap, _spans(m))
    del perm_in
    el = zipf_labels(seed, _S_ELABEL, m, n_elabels, zipf_e)
    vl = zipf_labels(seed, _S_VLABEL, n, n_vlabels, zipf_v)
    return Graph(n=n, m=m, row_offsets=row, col=col, elabel=el, vlabel=vl)


def chung_lu_torch(
    n: int,
    m: int,
    gamma_out: float,
    gamma_in: float,
    max_out_deg: float,
    max_in_deg: float,
    n_vlabels: int,
    zipf_v: float,
    n_elabels: int,
    zipf_e: float,
    seed: int,
    device="cuda",
):
    """:func:`chung_lu` drawn with torch on ``device``, so that billion-edge
    graphs are generated in seconds: the same counter-based streams, the same
    host-computed cumulative distributions, the same inverse-CDF searches and
    stable sorts, hence the identical graph.  Returns a dict of torch tensors
    (row_offsets int64, col int32, elabel int32, vlabel int32)."""
    import torch

    chunk = 1 << 27

    def draw(cdf_np, key, count, put):
        cdf = torch.from_numpy(cdf_np).to(device)
        for a in range(0, count, chunk):
            b = min(count, a + chunk)
            u = ctr_uniform_torch(key, a, b, device)
            put(a, b, torch.searchsorted(cdf, u, right=True).clamp_(max=cdf.shape[0] - 1))
            del u

    def permutation(key):
        keys = torch.empty(n, dtype=torch.int64, device=device)
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            keys[a:b] = _srl(ctr_bits_torch(key, a, b, device), 1)
        return torch.sort(keys, stable=True).indices

    deg_rank = torch.zeros(n, dtype=torch.int64, device=device)

    def acc_deg(a, b, idx):
        deg_rank.add_(torch.bincount(idx, minlength=n))

    draw(_cdf(_capped_powerlaw_degrees(n, m, gamma_out, max_out_deg)), stream_key(seed, _S_OUT), m, acc_deg)
    perm_out = permutation(stream_key(seed, _S_PERM_OUT))
    deg = torch.empty(n, dtype=torch.int64, device=device)
    deg[perm_out] = deg_rank
    del deg_rank, perm_out
    row = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg, 0, out=row[1:])
    del deg

    perm_in = permutation(stream_key(seed, _S_PERM_IN)).to(torch.int32)
    col = torch.empty(m, dtype=torch.int32, device=device)

    def put_col(a, b, idx):
        col[a:b] = perm_in[idx]

    draw(_cdf(_capped_powerlaw_degrees(n, m, gamma_in, max_in_deg)), stream_key(seed, _S_IN), m, put_col)
    del perm_in

    def labels(count, n_labels, s, stream):
        out = torch.zeros(count, dtype=torch.int32, device=device)
        if n_labels > 1:
            def put(a, b, idx):
                out[a:b] = idx.to(torch.int32)

            draw(_zipf_cdf(n_labels, s), stream_key(seed, stream), count, put)
        return out

    el = labels(m, n_elabels, zipf_e, _S_ELABEL)
    vl = labels(n, n_vlabels, zipf_v, _S_VLABEL)
    return {"n": n, "m": m, "row_offsets": row, "col": col, "elabel": el, "vlabel": vl}


# Named workloads (sizes from the workload descriptions; seeds fixed).
CONFIG_TINY = dict(kind="er", n=10_000, m=50_000, n_vlabels=8, n_elabels=4, seed=0)
CONFIG_RDF = dict(
    kind="chung_lu",
    n=10_000_000,
    m=100_000_000,
    gamma_out=2.1,
    gamma_in=2.1,
    max_out_deg=1_000_000,
    max_in_deg=1_000_000,
    n_vlabels=1000,
    zipf_v=1.5,
    n_elabels=200,
    zipf_e=1.2,
    seed=1,
)
CONFIG_LARGE = dict(
    kind="chung_lu",
    n=200_000_000,
    m=2_000_000_000,
    gamma_out=2.0,
    gamma_in=2.0,
    max_out_deg=67_000_000,
    max_in_deg=4_000_000,
    n_vlabels=5000,
    zipf_v=1.5,
    n_elabels=500,
    zipf_e=1.2,
    seed=2,
)


def scaled(config: dict, factor: float, seed: Optional[int] = None) -> dict:
    """The same recipe with n, m (and the degree caps) scaled by ``factor``."""
    c = dict(config)
    c["n"] = max(1, int(round(c["n"] * factor)))
    c["m"] = max(0, int(round(c["m"] * factor)))
    for key in ("max_out_deg", "max_in_deg"):
        if key in c:
            c[key] = max(1.0, c[key] * factor)
    if seed is not None:
        c["seed"] = seed
    return c


def make(config: dict) -> Graph:
    """Build a numpy graph from one of the named configurations."""
    c = dict(config)
    kind = c.pop("kind")
    if kind == "er":
        return erdos_renyi(c["n"], c["m"], c["n_vlabels"], c["n_elabels"], c["seed"])
    if kind == "chung_lu":
        return chung_lu(**c)
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Small structured graphs
# --------------------------------------------------------------------------

PAPER_VERTICES = [
    "asc",
    "dri",
    "jra",
    "uess",
    "uulm",
    "Ansgar Scherp",
    "David Richerby",
    "Jannik Rau",
    "University of Essex",
    "University of Ulm",
]


def paper_example() -> Graph:
    """The running example of Section 3 (figure "simple_example_graph"): two
    universities and three employees.  Vertex labels: 0 Lecturer, 1 Literal,
    2 Organization, 3 Professor, 4 Student.  Edge labels: 0 name, 1 worksAt."""
    idx = {v: i for i, v in enumerate(PAPER_VERTICES)}
    LEC, LIT, ORG, PROF, STUD = 0, 1, 2, 3, 4
    NAME, WORKS = 0, 1
    vl = [PROF, LEC, STUD, ORG, ORG, LIT, LIT, LIT, LIT, LIT]
    e = [
        ("asc", "Ansgar Scherp", NAME),
        ("asc", "uulm", WORKS),
        ("dri", "David Richerby", NAME),
        ("dri", "uess", WORKS),
        ("jra", "Jannik Rau", NAME),
        ("jra", "uulm", WORKS),
        ("uess", "University of Essex", NAME),
        ("uulm", "University of Ulm", NAME),
    ]
    src = [idx[a] for a, _, _ in e]
    dst = [idx[b] for _, b, _ in e]
    lab = [l for _, _, l in e]
    return from_edges(len(PAPER_VERTICES), src, dst, lab, vl, names=list(PAPER_VERTICES))


def tiny_random(rng: np.random.Generator, n_max: int = 12, m_max: int = 30, n_labels: int = 3) -> Graph:
    """A random tiny multigraph for exhaustive checks."""
    n = int(rng.integers(1, n_max + 1))
    m = int(rng.integers(0, m_max + 1))
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    el = rng.integers(0, n_labels, size=m).astype(np.int32)
    vl = rng.integers(0, n_labels, size=n).astype(np.int32)
    return from_edges(n, src, dst, el, vl)


def path_graph(n: int) -> Graph:
    """Directed path 0 -> 1 -> ... -> n-1, unlabelled."""
    src = np.arange(max(0, n - 1))
    return from_edges(n, src, src + 1)


def cycle_graph(n: int) -> Graph:
    """Directed cycle 0 -> 1 -> ... -> n-1 -> 0, unlabelled."""
    src = np.arange(n)
    return from_edges(n, src, (src + 1) % n)


def binary_tree(height: int) -> Graph:
    """Complete binary tree with edges parent -> child, 2^(height+1)-1 vertices."""
    n = (1 << (height + 1)) - 1
    parents = np.arange(n)
    kids = []
    srcs = []
    for p in parents:
        for c in (2 * p + 1, 2 * p + 2):
            if c < n:
                srcs.append(p)
                kids.append(c)
    return from_edges(n, srcs, kids)


def disjoint_union(graphs: Sequence[Graph]) -> Tuple[Graph, np.ndarray]:
    """Concatenate graphs into one vertex space.  Returns the union and the
    int64[G+1] vertex offsets of each member graph."""
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        voff[i + 1] = voff[i] + g.n
    n = int(voff[-1])
    m = int(sum(g.m for g in graphs))
    row = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(m, dtype=np.int32)
    el = np.empty(m, dtype=np.int32)
    vl = np.empty(n, dtype=np.int32)
    e0 = 0
    for i, g in enumerate(graphs):
        a, b = int(voff[i]), int(voff[i + 1])
        row[a + 1 : b + 1] = g.row_offsets[1:] + e0
        col[e0 : e0 + g.m] = g.col + a
        el[e0 : e0 + g.m] = g.elabel
        vl[a:b] = g.vlabel
        e0 += g.m
    return Graph(n=n, m=m, row_offsets=row, col=col, elabel=el, vlabel=vl), voff


def batch_workload(G: int = 4096, seed: int = 3, median_m: float = 5e4, sigma: float = 1.25,
                   m_lo: int = 1000, m_hi: int = 2_000_000, k_max: int = 10,
                   n_vlabels: int = 16, n_elabels: int = 8):
    """Many independent graphs of uneven size: edge counts lognormal (median
    ``median_m``, sigma ``sigma``) clipped to [m_lo, m_hi], n = m/5, uniform
    labels, and a per-graph k uniform on 1..k_max.  Returns (graphs, ks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ms = np.clip(np.exp(rng.normal(np.log(median_m), sigma, size=G)), m_lo, m_hi).astype(np.int64)
    ks = rng.integers(1, k_max + 1, size=G).astype(np.int32)
    seeds = rng.integers(0, 2**31 - 1, size=G)
    graphs = [
        erdos_renyi(max(1, int(mm) // 5), int(mm), n_vlabels, n_elabels, int(s)) for mm, s in zip(ms, seeds)
    ]
    return graphs, ks


def serve_workload(duration_s: float = 60.0, rate: float = 200.0, seed: int = 4,
                   median_m: float = 7e5, sigma: float = 1.4, m_lo: int = 10_000,
                   m_hi: int = 50_000_000, k_max: int = 10):
    """A Poisson stream of summarisation requests.  Returns a list of
    (arrival_time_s, m, k, graph_seed); graphs are built by the caller with
    :func:`chung_lu` (exponent 2.1, 64 vertex / 32 edge labels, Zipf)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration_s:
            break
        mm = int(np.clip(np.exp(rng.normal(np.log(median_m), sigma)), m_lo, m_hi))
        k = int(rng.integers(1, k_max + 1))
        out.append((t, mm, k, int(rng.integers(0, 2**31 - 1))))
    return out


def serve_graph(m: int, seed: int) -> Graph:
    """One serving request's graph: power law (exponent 2.1), n = m/5,
    64 vertex labels Zipf(1.5), 32 edge labels Zipf(1.2)."""
    n = max(1, m // 5)
    return chung_lu(n, m, 2.1, 2.1, max(1.0, m / 10), max(1.0, m / 10), 64, 1.5, 32, 1.2, seed)


def batch_union_torch(G: int = 4096, seed: int = 3, median_m: float = 5e4, sigma: float = 1.25,
                      m_lo: int = 1000, m_hi: int = 2_000_000, k_max: int = 10, n_vlabels: int = 16,
                      n_elabels: int = 8, device="cuda"):
    """The batching workload drawn with torch on ``device``: G Erdos-Renyi
    graphs with lognormal edge counts (clipped to [m_lo, m_hi]), n = m/5,
    uniform labels and k uniform on 1..k_max, laid out as one disjoint union.
    Returns (union dict of tensors, vertex offsets int64[G+1] numpy, ks int32[G]
    numpy)."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    ms = np.clip(np.exp(rng.normal(np.log(median_m), sigma, size=G)), m_lo, m_hi).astype(np.int64)
    ns = np.maximum(1, ms // 5)
    ks = rng.integers(1, k_max + 1, size=G).astype(np.int32)
    voff = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ns, out=voff[1:])
    eoff = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ms, out=eoff[1:])
    n, m = int(voff[-1]), int(eoff[-1])
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    gid = torch.repeat_interleave(torch.arange(G, device=device), torch.from_numpy(ms).to(device))
    base = torch.from_numpy(voff[:-1]).to(device)[gid]
    size = torch.from_numpy(ns).to(device)[gid]
    src = base + (torch.rand(m, generator=gen, device=device, dtype=torch.float64) * size).long().clamp_(max=size - 1)
    dst = base + (torch.rand(m, generator=gen, device=device, dtype=torch.float64) * size).long().clamp_(max=size - 1)
    del gid, base, size
    order = torch.argsort(src, stable=True)
    col = dst[order].to(torch.int32)
    deg = torch.bincount(src, minlength=n)
    del src, dst, order
    row = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg, 0, out=row[1:])
    el = torch.randint(0, max(1, n_elabels), (m,), generator=gen, device=device, dtype=torch.int32)
    vl = torch.randint(0, max(1, n_vlabels), (n,), generator=gen, device=device, dtype=torch.int32)
    return ({"n": n, "m": m, "row_offsets": row, "col": col, "elabel": el, "vlabel": vl}, voff, ks)
