"""Brute-force k-bisimilarity, pair by pair, straight from the definitions
(TEST INFRASTRUCTURE ONLY).

This is the independent pin for the C++ oracle: it never builds a signature
or a key.  It keeps the relation R_i as an n x n boolean matrix and applies the
recursive step of the paper's definitions literally:

* Def. "fw-bisim" / "edge-labeled-fw-bisimulation" (Section 3.2, 3.3):
  u R_{i+1} v iff u R_i v and every edge (u, u') has an edge (v, v') with the
  same label (when labels are used) and u' R_i v', and vice versa.
* Def. "bw-bisim" / "vertex-labeled-bw-bisimulation": the same over in-edges.
  The unlabelled backward definition omits "vice versa"; we read it as
  symmetric, as its labelled variant and its example table are.
* BOTH: the forward and the backward conditions must hold together.
* R_0: everything related, or equal vertex label (Def. "vertex-labeled-bw-
  bisimulation", first bullet).
* Generic CSE rounds (Def. "cse", Def. "chaining-parameterization"): the
  first condition u ~s v replaces "u R_i v" -- T, equal labels or id -- and
  the nested CSE^{i-1} is R_i.

Only for tiny graphs: cost is O(k n^2 deg^2).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def _adjacency(n, src, dst, lab, direction_in: bool):
    adj = [[] for _ in range(n)]
    for s, d, l in zip(src, dst, lab):
        if direction_in:
            adj[d].append((s, l))
        else:
            adj[s].append((d, l))
    return adj


def _matches(adj, R, u, v, use_labels):
    # every edge of u has a partner edge of v with the same label and related ends
    for (u2, lu) in adj[u]:
        ok = False
        for (v2, lv) in adj[v]:
            if (not use_labels or lu == lv) and R[u2][v2]:
                ok = True
                break
        if not ok:
            return False
    return True


def relations(n: int, src: Sequence[int], dst: Sequence[int], elabel: Sequence[int], vlabel: Sequence[int],
              direction: int, use_vertex_labels: bool, use_edge_labels: bool, k: int,
              subject: int = 0) -> List[List[List[bool]]]:
    """R_0..R_k as n x n boolean matrices.  ``subject`` is the first condition
    of Def. "cse" (v ~s v'): 0 keeps R_i itself (stratified bisimulation),
    1 is T, 2 equal vertex labels, 3 id."""
    src = [int(x) for x in src]
    dst = [int(x) for x in dst]
    lab = [int(x) for x in elabel] if elabel is not None else [0] * len(src)
    out_adj = _adjacency(n, src, dst, lab, False)
    in_adj = _adjacency(n, src, dst, lab, True)
    if use_vertex_labels:
        R = [[int(vlabel[u]) == int(vlabel[v]) for v in range(n)] for u in range(n)]
    else:
        R = [[True] * n for _ in range(n)]
    Rs = [R]
    for _ in range(k):
        nR = [[False] * n for _ in range(n)]
        for u in range(n):
            for v in range(n):
                if subject == 0 and not R[u][v]:
                    continue
                if subject == 2 and int(vlabel[u]) != int(vlabel[v]):
                    continue
                if subject == 3 and u != v:
                    continue
                ok = True
                if direction in (0, 2):
                    ok = ok and _matches(out_adj, R, u, v, use_edge_labels) and _matches(out_adj, R, v, u, use_edge_labels)
                if direction in (1, 2):
                    ok = ok and _matches(in_adj, R, u, v, use_edge_labels) and _matches(in_adj, R, v, u, use_edge_labels)
                nR[u][v] = ok
        R = nR
        Rs.append(R)
    return Rs


def canonical_ids(R: List[List[bool]]) -> List[int]:
    """Block ids numbered by smallest member (R must be an equivalence)."""
    n = len(R)
    ids = [-1] * n
    nxt = 0
    for v in range(n):
        if ids[v] >= 0:
            continue
        for u in range(v, n):
            if R[v][u]:
                ids[u] = nxt
        nxt += 1
    return ids


def is_equivalence(R: List[List[bool]]) -> bool:
    n = len(R)
    for u in range(n):
        if not R[u][u]:
            return False
        for v in range(n):
            if R[u][v] != R[v][u]:
                return False
            if R[u][v]:
                for w in range(n):
                    if R[v][w] and not R[u][w]:
                        return False
    return True


def levels(n, src, dst, elabel, vlabel, direction, use_vertex_labels, use_edge_labels, k,
           subject=0) -> Tuple[List[List[int]], List[List[List[bool]]]]:
    Rs = relations(n, src, dst, elabel, vlabel, direction, use_vertex_labels, use_edge_labels, k, subject)
    return [canonical_ids(R) for R in Rs], Rs
