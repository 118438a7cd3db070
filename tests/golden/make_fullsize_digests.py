"""Write the oracle's levels of the full-size RDF-like graph as digests.

The RDF-like workload (graphgen.CONFIG_RDF: Chung-Lu exponent 2.1, n = 10^7,
m = 10^8, degree cap 10^6, 1,000 vertex labels Zipf(1.5), 200 edge labels
Zipf(1.2), seed 1) stands in for BTC150M / Laundromat100M (paper Section 5.1,
Table "statistics-datasets").  Its levels 0..k (int32[n] each, 40 MB) are too
large to store, so this script stores, per direction and level, the SHA-256 of
the level's little-endian int32 bytes, the digests of 16 equal vertex ranges
(to localise a mismatch) and the block count, all computed from the CPU oracle
(oracle/, the plain map refinement) and nothing else.  The graph itself is
identified by the SHA-256 of its four arrays, so a test can check that the
graph it drew (on the GPU, with graphgen.chung_lu_torch) is this one.

Run:  python tests/golden/make_fullsize_digests.py  (about 10 minutes, 8 GB)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rdf_10m_levels.json")
K = 10
CHUNKS = 16


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def level_entry(level, count):
    n = level.shape[0]
    bounds = [n * j // CHUNKS for j in range(CHUNKS + 1)]
    return {"count": int(count), "sha256": sha(level),
            "chunks": [sha(level[bounds[j]:bounds[j + 1]])[:16] for j in range(CHUNKS)]}


def main():
    t0 = time.time()
    cfg = graphgen.CONFIG_RDF
    g = graphgen.make(cfg)
    out = {
        "about": "oracle levels 0..%d of graphgen.CONFIG_RDF (Chung-Lu 2.1, n=1e7, m=1e8, seed 1), written by "
                 "tests/golden/make_fullsize_digests.py from oracle/ only; stand-in for the paper's BTC150M / "
                 "Laundromat100M (Section 5.1, Table statistics-datasets)" % K,
        "config": {key: cfg[key] for key in cfg},
        "k": K,
        "chunks": CHUNKS,
        "graph_sha256": sha(g.row_offsets, g.col, g.elabel, g.vlabel),
        "directions": {},
    }
    print("graph drawn in %.0f s" % (time.time() - t0), flush=True)
    for name, d in (("out", oracle.DIR_OUT), ("both", oracle.DIR_BOTH)):
        t1 = time.time()
        L, C, lc = oracle.refine_graph(g, d, True, True, k=K, early_stop=True)
        out["directions"][name] = {"levels_computed": int(lc),
                                   "levels": [level_entry(L[i], C[i]) for i in range(K + 1)]}
        print("%s: levels computed %d, counts %s, %.0f s" % (name, lc, list(C), time.time() - t1), flush=True)
        del L
    with open(OUT_PATH, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote %s in %.0f s" % (OUT_PATH, time.time() - t0))


if __name__ == "__main__":
    main()
