"""Parity at the full size of the benchmark workload: the 2e9-edge Chung-Lu
graph (n = 2e8, exponent 2.0, hub cap 6.7e7, Zipf labels), out-edges, k = 10,
early stop, default options: the launch configuration bench.py times.  The
whole-graph oracle would take hours there, so every level is checked against
properties that hold at any size (canonical numbering, nesting, counts,
early-stop copies), and sampled vertices -- random ones, whole sampled blocks
and hubs -- against the CPU oracle's signature (Def. "signature") one by one:
within the sample, two vertices share a block exactly when they share the
previous block and the signature.  The levels come from a prepared graph with
the locality order, as bench.py times them, and must equal a plain kb_refine.
"""
import os

import numpy as np
import pytest

import cpu_parallel
import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402

K = 10


@pytest.fixture(scope="module")
def run():
    free, _ = torch.cuda.mem_get_info(0)
    if free < 90e9:
        pytest.skip("the 2e9-edge graph needs about 70 GB of device memory")
    cfg = dict(graphgen.CONFIG_LARGE)
    cfg.pop("kind")
    wl = graphgen.chung_lu_torch(device="cuda:0", **cfg)
    dg = kb.DeviceGraph(wl["row_offsets"], wl["col"], wl["elabel"], wl["vlabel"])
    ctx = kb.Context(0)
    opts = kb.Options(direction=kb.DIR_OUT)
    # the bench's path: a prepared graph (locality order on), then one call
    with ctx.prepare(dg, opts) as pg:
        assert pg.info()["reorder"] == 1
        res = ctx.refine(pg, K, opts)
    torch.cuda.synchronize()
    yield wl, dg, ctx, res
    ctx.close()
    del wl, dg, res
    torch.cuda.empty_cache()


def test_prepared_equals_plain_call(run):
    # the prepared path (locality order on) and a plain kb_refine (off) agree
    wl, dg, ctx, res = run
    plain = ctx.refine(dg, K, kb.Options(direction=kb.DIR_OUT))
    assert torch.equal(plain.levels, res.levels)
    assert np.array_equal(plain.counts, res.counts) and plain.levels_computed == res.levels_computed
    del plain


def _block_minima(L, cnt):
    n = L.numel()
    idx = torch.arange(n, device=L.device, dtype=torch.int64)
    mins = torch.full((cnt,), n, device=L.device, dtype=torch.int64)
    return mins.scatter_reduce_(0, L.long(), idx, reduce="amin")


def test_levels_are_canonical_nested_partitions(run):
    wl, _, _, res = run
    L, counts, lc = res.levels, res.counts, res.levels_computed
    n = wl["n"]
    assert counts[0] == 5000 and 1 <= lc <= K
    for i in range(K + 1):
        cnt = int(counts[i])
        Li = L[i]
        assert int(Li.min()) == 0 and int(Li.max()) == cnt - 1
        mins = _block_minima(Li, cnt)
        # every id is used, and ids are the ranks of the blocks' smallest members
        assert int(mins.max()) < n
        assert bool(torch.all(mins[1:] > mins[:-1]))
        if i >= 1:
            assert counts[i] >= counts[i - 1]
            # level i refines level i-1: a block's members share their previous block
            rep = mins[Li.long()]
            assert bool(torch.equal(L[i - 1], L[i - 1][rep]))
        if i > lc:
            assert bool(torch.equal(Li, L[lc])) and counts[i] == counts[lc]
    if lc < K:
        assert counts[lc] == counts[lc - 1]  # the run stopped at a stable level


def _sample(wl, L_i, rng):
    deg = wl["row_offsets"][1:] - wl["row_offsets"][:-1]
    n = wl["n"]
    picks = []
    # random vertices of modest degree (edgeless ones included)
    cand = torch.from_numpy(rng.integers(0, n, size=6000)).to(deg.device)
    picks.append(cand[deg[cand] <= 4096][:3000])
    # whole blocks around random vertices: up to 16 members each
    for v in rng.integers(0, n, size=120).tolist():
        members = torch.nonzero(L_i == L_i[v]).flatten()
        members = members[deg[members] <= 4096][:16]
        picks.append(members)
    # hubs of up to 1e5 edges
    hubs = torch.nonzero((deg > 1024) & (deg <= 100_000)).flatten()
    if hubs.numel():
        picks.append(hubs[torch.from_numpy(rng.integers(0, hubs.numel(), size=12)).to(hubs.device)])
    return torch.unique(torch.cat(picks)).cpu().numpy()


@pytest.mark.parametrize("level", [1, 2, "last"])
def test_sampled_keys_match_oracle(run, level):
    wl, _, _, res = run
    i = res.levels_computed if level == "last" else level
    rng = np.random.Generator(np.random.PCG64(100 + i))
    L_prev, L_i = res.levels[i - 1], res.levels[i]
    vs = _sample(wl, L_i, rng)
    row = wl["row_offsets"]
    starts = row[torch.from_numpy(vs).to(row.device)].cpu().numpy()
    ends = row[torch.from_numpy(vs + 1).to(row.device)].cpu().numpy()
    # one gather of every sampled edge: neighbour, label, neighbour's previous block
    eidx = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]).astype(np.int64)
    e_t = torch.from_numpy(eidx).to(row.device)
    nb = wl["col"][e_t]
    labs = wl["elabel"][e_t].cpu().numpy()
    blocks = L_prev[nb.long()].cpu().numpy()
    own_prev = L_prev[torch.from_numpy(vs).to(row.device)].cpu().numpy()
    got = L_i[torch.from_numpy(vs).to(row.device)].cpu().numpy()
    key_to_id, id_to_key = {}, {}
    off = 0
    for j, v in enumerate(vs.tolist()):
        d = int(ends[j] - starts[j])
        mini_row = np.array([0, d], dtype=np.int64)
        sig = oracle.signature(mini_row, np.arange(d), labs[off:off + d], blocks[off:off + d], 0)
        off += d
        key = (int(own_prev[j]), sig)
        b = int(got[j])
        # same key <=> same block, within the sample
        assert key_to_id.setdefault(key, b) == b, ("equal keys, different blocks", v, i)
        assert id_to_key.setdefault(b, key) == key, ("one block, different keys", v, i)
    # the sample must contain both shared and separate blocks to mean anything
    assert len(id_to_key) > 100 and len(id_to_key) < len(vs)


def _host_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        return 0


def test_every_level_equals_the_openmp_implementation(run):
    # A cross-check over all 2e8 vertices and every level: the multi-core CPU
    # implementation (cpu_parallel/, written apart from the library and
    # compared with the oracle on smaller graphs in test_cpu_parallel.py)
    # refines the same graph, and every id of every level must agree.
    if _host_bytes() < 120e9:
        pytest.skip("the CPU run on the 2e9-edge graph needs about 70 GB of host memory")
    wl, _, _, res = run
    host = [wl[name].cpu().numpy() for name in ("row_offsets", "col", "elabel", "vlabel")]
    L, C, lc = cpu_parallel.refine(wl["n"], host[0], host[1], host[2], host[3], 0, True, True, k=K)
    del host
    assert np.array_equal(res.counts, C) and res.levels_computed == lc
    for i in range(K + 1):
        assert np.array_equal(res.levels[i].cpu().numpy(), L[i]), i
