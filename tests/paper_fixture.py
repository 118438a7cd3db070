"""Parsers for tests/golden/paper_example.txt (the paper's worked example) and
tests/golden/paper_summary.txt (its summary graphs)."""
import os

import numpy as np

import graphgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_example.txt")
DIRS = {"out": 0, "in": 1, "both": 2}


def load():
    vlabels, names, edges, tables = {}, {}, [], {}
    cur = None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "vertex":
            vid = int(tok[1])
            vlabels[vid] = tok[2]
            names[vid] = " ".join(tok[3:])
        elif tok[0] == "edge":
            edges.append((int(tok[1]), int(tok[2]), tok[3]))
        elif tok[0] == "table":
            cur = tok[1]
            tables[cur] = dict(direction=DIRS[tok[2]], use_vertex_labels=bool(int(tok[3])),
                               use_edge_labels=bool(int(tok[4])), levels={})
        elif tok[0] == "level":
            body = line.split(None, 2)[2]
            blocks = [frozenset(int(x) for x in b.split()) for b in body.split("|")]
            tables[cur]["levels"][int(tok[1])] = frozenset(blocks)
    n = len(names)
    vnames = sorted(set(vlabels.values()))
    enames = sorted(set(e[2] for e in edges))
    vl = np.array([vnames.index(vlabels[v]) for v in range(n)], dtype=np.int32)
    g = graphgen.from_edges(n, [e[0] for e in edges], [e[1] for e in edges],
                            [enames.index(e[2]) for e in edges], vl,
                            names=[names[v] for v in range(n)])
    return g, tables


def partition(ids):
    blocks = {}
    for v, b in enumerate(ids):
        blocks.setdefault(int(b), set()).add(v)
    return frozenset(frozenset(s) for s in blocks.values())


SUMMARY_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_summary.txt")


def canonical_ids(blocks, n):
    """Block ids of a partition (a set of frozensets) numbered by smallest member."""
    ids = np.zeros(n, dtype=np.int32)
    for rank, b in enumerate(sorted(blocks, key=min)):
        for v in b:
            ids[v] = rank
    return ids


def load_summary():
    """The hand-derived summary graphs: a list of (table, source level, target
    level, [(source block, label id, target block), ...]).  Label names map to
    the ids load() gives them; "0" stands for an unlabelled edge."""
    edges = [line.split() for line in open(GOLDEN) if line.startswith("edge ")]
    enames = sorted(set(e[3] for e in edges))
    cases = []
    for line in open(SUMMARY_GOLDEN):
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        if tok[0] == "case":
            cases.append((tok[1], int(tok[2]), int(tok[3]), []))
        elif tok[0] == "summary":
            lab = 0 if tok[2] == "0" else enames.index(tok[2])
            cases[-1][3].append((int(tok[1]), lab, int(tok[3])))
    return cases
