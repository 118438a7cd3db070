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


def zipf_labels(rng: np.random.Generator, count: int, n_labels: int, s: float) -> np.ndarray:
    """Labels 0..n_labels-1 with P(label = j) proportional to (j+1)^-s."""
    if n_labels <= 1:
        return np.zeros(count, dtype=np.int32)
    p = np.arange(1, n_labels + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    out = np.empty(count, dtype=np.int32)
    chunk = 1 << 24
    for a in range(0, count, chunk):
        b = min(count, a + chunk)
        out[a:b] = np.minimum(np.searchsorted(cdf, rng.random(b - a), side="right"), n_labels - 1)
    return out


def _capped_powerlaw_degrees(n: int, m: int, gamma: float, cap: float) -> np.ndarray:
    """Chung-Lu expected degrees: rank r (1-based) gets weight r^(-1/(gamma-1)),
    scaled to sum m, with the largest clipped at ``cap`` and the remainder
    rescaled so the total stays m."""
    r = np.arange(1, n + 1, dtype=np.float64)
    w = r ** (-1.0 / (gamma - 1.0))
    d = w * (m / w.sum())
    for _ in range(50):
        over = d > cap
        if not over.any():
            break
        d[over] = cap
        free = ~over
        rest = m - cap * over.sum()
        d[free] *= rest / d[free].sum()
    return d


def _sample_ranks(rng: np.random.Generator, cdf: np.ndarray, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    chunk = 1 << 24
    for a in range(0, count, chunk):
        b = min(count, a + chunk)
        out[a:b] = np.minimum(np.searchsorted(cdf, rng.random(b - a), side="right"), cdf.shape[0] - 1)
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

    Out-degrees are one multinomial draw of m edges over the capped out-weights;
    every edge's target is drawn independently from the capped in-weights
    ("preferential by in-degree").  Out-rank and in-rank are mapped to vertex
    ids by two independent random permutations, so hub ids carry no locality.
    Vertices that draw no out-edges are the "literal" sinks of RDF data.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    d_out = _capped_powerlaw_degrees(n, m, gamma_out, max_out_deg)
    deg_rank = rng.multinomial(m, d_out / d_out.sum()).astype(np.int64)
    perm_out = rng.permutation(n)
    deg = np.empty(n, dtype=np.int64)
    deg[perm_out] = deg_rank
    row = _rows_from_degrees(deg)

    d_in = _capped_powerlaw_degrees(n, m, gamma_in, max_in_deg)
    cdf_in = np.cumsum(d_in)
    cdf_in /= cdf_in[-1]
    perm_in = rng.permutation(n).astype(np.int32)
    col = perm_in[_sample_ranks(rng, cdf_in, m)]
    el = zipf_labels(rng, m, n_elabels, zipf_e)
    vl = zipf_labels(rng, n, n_vlabels, zipf_v)
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
    """The same recipe as :func:`chung_lu`, drawn with torch on ``device`` so
    that billion-edge graphs are generated in seconds.  Returns a dict of torch
    tensors (row_offsets int64, col int32, elabel int32, vlabel int32).  The
    random stream differs from the numpy version; each is its own seeded
    workload."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    chunk = 1 << 27

    # Cumulative distributions are summed on the host: a floating-point scan on
    # the device may combine partial sums in a different order from run to run,
    # which would move a few draws across bin boundaries.
    def capped_cdf(gamma, cap):
        c = np.cumsum(_capped_powerlaw_degrees(n, m, gamma, cap))
        c /= c[-1]
        return torch.from_numpy(c).to(device)

    def draw(cdf, count, out, transform):
        for a in range(0, count, chunk):
            b = min(count, a + chunk)
            u = torch.rand(b - a, generator=g, device=device, dtype=torch.float64)
            idx = torch.searchsorted(cdf, u, right=True).clamp_(max=cdf.shape[0] - 1)
            transform(a, b, idx)

    cdf_out = capped_cdf(gamma_out, max_out_deg)
    deg_rank = torch.zeros(n, dtype=torch.int64, device=device)

    def acc_deg(a, b, idx):
        deg_rank.add_(torch.bincount(idx, minlength=n))

    draw(cdf_out, m, None, acc_deg)
    perm_out = torch.randperm(n, generator=g, device=device)
    deg = torch.empty(n, dtype=torch.int64, device=device)
    deg[perm_out] = deg_rank
    del deg_rank, perm_out
    row = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg, 0, out=row[1:])
    del deg

    cdf_in = capped_cdf(gamma_in, max_in_deg)
    perm_in = torch.randperm(n, generator=g, device=device).to(torch.int32)
    col = torch.empty(m, dtype=torch.int32, device=device)

    def put_col(a, b, idx):
        col[a:b] = perm_in[idx]

    draw(cdf_in, m, None, put_col)
    del perm_in

    def zipf_cdf(L, s):
        c = np.cumsum(np.arange(1, L + 1, dtype=np.float64) ** (-s))
        return torch.from_numpy(c / c[-1]).to(device)

    el = torch.empty(m, dtype=torch.int32, device=device)

    def put_el(a, b, idx):
        el[a:b] = idx.to(torch.int32)

    draw(zipf_cdf(max(1, n_elabels), zipf_e), m, None, put_el)
    vl = torch.empty(n, dtype=torch.int32, device=device)

    def put_vl(a, b, idx):
        vl[a:b] = idx.to(torch.int32)

    draw(zipf_cdf(max(1, n_vlabels), zipf_v), n, None, put_vl)
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
