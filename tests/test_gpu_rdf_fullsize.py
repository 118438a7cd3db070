"""Parity at full size on the RDF-like workload (n = 10^7, m = 10^8, Chung-Lu
exponent 2.1, Zipf labels: the stand-in for BTC150M / Laundromat100M of the
paper's Section 5.1), out-edges and both directions, k = 10, early stop on and
off, every element of every level.

The oracle's levels of this graph are stored as SHA-256 digests of each
level's int32 bytes (tests/golden/rdf_10m_levels.json, written by
tests/golden/make_fullsize_digests.py from oracle/ only); equal digests mean
equal levels, element by element.  The graph is drawn on the GPU with the
same counter-based generator the script used on the host, and its own digest
is checked first.  On a mismatch the digests of 16 vertex ranges say where.
Both the plain call and a prepared graph (locality order on) are checked.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402

GOLD_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rdf_10m_levels.json")


def _gold():
    with open(GOLD_PATH) as f:
        return json.load(f)


def _sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def rdf():
    gold = _gold()
    free, _ = torch.cuda.mem_get_info(0)
    if free < 12e9:
        pytest.skip("the 1e8-edge graph needs about 8 GB of device memory")
    cfg = dict(gold["config"])
    cfg.pop("kind")
    wl = graphgen.chung_lu_torch(device="cuda:0", **cfg)
    torch.cuda.synchronize()
    host = [wl[name].cpu().numpy() for name in ("row_offsets", "col", "elabel", "vlabel")]
    assert _sha(*host) == gold["graph_sha256"], "the device-drawn graph is not the one the oracle saw"
    del host
    dg = kb.DeviceGraph(wl["row_offsets"], wl["col"], wl["elabel"], wl["vlabel"])
    ctx = kb.Context(0)
    yield gold, dg, ctx
    ctx.close()
    del dg, wl
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prepared", [False, True])
@pytest.mark.parametrize("early_stop", [True, False])
@pytest.mark.parametrize("direction", ["out", "both"])
def test_rdf_full_size_levels_equal_oracle(rdf, direction, early_stop, prepared):
    G, dg, ctx = rdf
    K = G["k"]
    gold = G["directions"][direction]
    d = kb.DIR_OUT if direction == "out" else kb.DIR_BOTH
    opts = kb.Options(direction=d, early_stop=early_stop)
    if prepared:  # a prepared graph, with the locality order (automatic at this size)
        with ctx.prepare(dg, opts) as pg:
            assert pg.info()["reorder"] == 1
            res = ctx.refine(pg, K, opts)
    else:
        res = ctx.refine(dg, K, opts)
    torch.cuda.synchronize()
    chunks = G["chunks"]
    for i in range(K + 1):
        want = gold["levels"][i]
        level = res.levels[i].cpu().numpy()
        assert int(res.counts[i]) == want["count"], ("count", direction, i, int(res.counts[i]), want["count"])
        if _sha(level) != want["sha256"]:
            n = level.shape[0]
            bad = [j for j in range(chunks)
                   if _sha(level[n * j // chunks:n * (j + 1) // chunks])[:16] != want["chunks"][j]]
            raise AssertionError("level %d (%s) differs from the oracle in vertex ranges %s of %d"
                                 % (i, direction, bad, chunks))
    if early_stop:
        assert res.levels_computed == gold["levels_computed"]
    else:
        assert res.levels_computed == K
