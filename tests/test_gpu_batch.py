"""Batched refinement (kb_refine_batch): every graph's levels, counts and last
refined level in the batch equal its solo result from the oracle, exactly."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = kb.Context(0)
    yield c
    c.close()


def mixed_graphs(seed, count):
    rng = np.random.Generator(np.random.PCG64(seed))
    gs = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            gs.append(graphgen.erdos_renyi(int(rng.integers(1, 400)), int(rng.integers(0, 2000)), 3, 3,
                                           int(rng.integers(0, 1 << 30))))
        elif kind == 1:
            gs.append(graphgen.tiny_random(rng, n_max=30, m_max=80, n_labels=3))
        elif kind == 2:
            n = int(rng.integers(50, 3000))
            gs.append(graphgen.chung_lu(n, 6 * n, 2.1, 2.1, n, n, 5, 1.5, 4, 1.2, int(rng.integers(0, 1 << 30))))
        else:
            gs.append(graphgen.from_edges(int(rng.integers(1, 20)), [], [], [], rng.integers(0, 2, size=0)))
            gs[-1].vlabel = rng.integers(0, 3, size=gs[-1].n).astype(np.int32)
    ks = rng.integers(0, 7, size=count).astype(np.int32)
    return gs, ks


def check_batch(ctx, graphs, ks, d, vl, el, early=True, **kw):
    union, voff = graphgen.disjoint_union(graphs)
    dg = kb.DeviceGraph.from_numpy(union, "cuda:0")
    levels, counts, lc = ctx.refine_batch(dg, voff, ks, kb.Options(direction=d, use_vertex_labels=vl,
                                                                    use_edge_labels=el, early_stop=early, **kw))
    levels = levels.cpu().numpy()
    kmax = int(ks.max())
    for j, g in enumerate(graphs):
        L, C, lcj = oracle.refine_graph(g, d, vl, el, k=int(ks[j]), early_stop=early)
        a, b = int(voff[j]), int(voff[j + 1])
        for i in range(kmax + 1):
            src = min(i, int(ks[j]))
            assert np.array_equal(levels[i, a:b], L[src]), (j, i, d, vl, el, kw)
            assert counts[j, i] == C[src], (j, i)
        assert lc[j] == lcj, (j, lc[j], lcj)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_batch_equals_solo(ctx, d):
    graphs, ks = mixed_graphs(10 + d, 60)
    check_batch(ctx, graphs, ks, d, True, True)


@pytest.mark.parametrize("vl,el", [(False, True), (True, False), (False, False)])
def test_batch_label_variants(ctx, vl, el):
    graphs, ks = mixed_graphs(20, 40)
    check_batch(ctx, graphs, ks, 0, vl, el)
    check_batch(ctx, graphs, ks, 2, vl, el, early=False)


def test_batch_weak_hash_and_hubs(ctx):
    graphs, ks = mixed_graphs(30, 40)
    check_batch(ctx, graphs, ks, 0, True, True, hash_mode=1)
    check_batch(ctx, graphs, ks, 1, True, True, hub_threshold=4)
    check_batch(ctx, graphs, ks, 2, True, True, hub_threshold=2, hash_mode=1)


def test_batch_single_and_degenerate(ctx):
    g = graphgen.make(graphgen.CONFIG_TINY)
    check_batch(ctx, [g], np.array([10], dtype=np.int32), 0, True, True)
    check_batch(ctx, [g, g, g], np.array([0, 3, 10], dtype=np.int32), 1, True, True)
    empty = graphgen.from_edges(1, [], [], [], [4])
    check_batch(ctx, [empty, g, empty], np.array([2, 2, 0], dtype=np.int32), 2, True, True)


TUNING_FIELDS = ("load_factor", "hub_threshold", "small_task_vertices", "hub_chunk_edges", "medium_split",
                 "small_max_degree")


def _check_tuning(t):
    assert min(abs(t["load_factor"] - x) for x in (0.35, 0.5, 0.7)) < 1e-6
    assert t["hub_threshold"] in (256, 512, 1024)
    assert t["small_task_vertices"] in (64, 128, 256, 512)
    assert t["hub_chunk_edges"] in (256, 512, 1024)
    assert t["medium_split"] in (64, 128, 256)
    assert t["small_max_degree"] in (16, 24, 32)
    assert 0 < t["ms"] <= t["default_ms"]


def test_autotune_keeps_results(ctx):
    # an RDF-like graph with hubs, so every tuning field has work to act on
    g = graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.002, seed=5))
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    ctx.clear_tuning()
    t = ctx.autotune(dg, kb.Options(), rounds=2)
    _check_tuning(t)
    L, C, lc = oracle.refine_graph(g, 0, True, True, k=6)
    res = ctx.refine(dg, 6, kb.Options())  # takes the cached tuning of this size class
    assert np.array_equal(res.levels.cpu().numpy(), L) and np.array_equal(res.counts, C)
    explicit = kb.Options(**{f: t[f] for f in TUNING_FIELDS})
    res = ctx.refine(dg, 6, explicit)
    assert np.array_equal(res.levels.cpu().numpy(), L)
    ctx.clear_tuning()


def test_autotune_batch_keeps_results(ctx):
    gs, ks = mixed_graphs(40, 48)
    union, voff = graphgen.disjoint_union(gs)
    dg = kb.DeviceGraph.from_numpy(union, "cuda:0")
    ctx.clear_tuning()
    t = ctx.autotune(dg, kb.Options(), rounds=3, vertex_offsets=voff, ks=ks)
    _check_tuning(t)
    assert t["size_class"] >= 64
    check_batch(ctx, gs, ks, 0, True, True)  # refine_batch now uses the cached choice
    ctx.clear_tuning()


@pytest.mark.parametrize("fields", [
    dict(small_max_degree=1, medium_split=1),
    dict(small_max_degree=16, medium_split=64, small_task_vertices=32),
    dict(hub_chunk_edges=256, hub_threshold=64, medium_split=33),
    dict(hub_chunk_edges=1024, hub_threshold=8, small_max_degree=4),
    dict(small_max_degree=32, medium_split=256, hub_chunk_edges=512, small_task_vertices=65536),
])
def test_tuning_fields_keep_results(ctx, fields):
    # extreme values of every tuning field against the oracle, one graph and a batch
    g = graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.001, seed=9))
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    for d in (kb.DIR_OUT, kb.DIR_BOTH):
        L, C, _ = oracle.refine_graph(g, d, True, True, k=5, early_stop=False)
        for rekey_all in (False, True):
            res = ctx.refine(dg, 5, kb.Options(direction=d, early_stop=False, rekey_all=rekey_all, **fields))
            assert np.array_equal(res.levels.cpu().numpy(), L), (d, rekey_all)
            assert np.array_equal(res.counts, C)
    gs, ks = mixed_graphs(41, 24)
    union, voff = graphgen.disjoint_union(gs)
    dgu = kb.DeviceGraph.from_numpy(union, "cuda:0")
    levels, counts, lc = ctx.refine_batch(dgu, voff, ks, kb.Options(**fields))
    for j, gj in enumerate(gs):
        Lj, Cj, lcj = oracle.refine_graph(gj, 0, True, True, k=int(ks[j]), early_stop=True)
        got = levels[:, int(voff[j]):int(voff[j + 1])].cpu().numpy()
        for i in range(int(ks.max()) + 1):
            assert np.array_equal(got[i], Lj[min(i, int(ks[j]))]), (j, i)


def test_tuning_fields_are_range_checked(ctx):
    g = graphgen.make(graphgen.CONFIG_TINY)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    for bad in (dict(hub_chunk_edges=300), dict(hub_chunk_edges=2048), dict(medium_split=257),
                dict(medium_split=-1), dict(small_max_degree=33), dict(small_max_degree=-2)):
        with pytest.raises(kb.KbError):
            ctx.refine(dg, 2, kb.Options(**bad))


def test_batch_rejects_cse_subjects(ctx):
    g = graphgen.make(graphgen.CONFIG_TINY)
    union, voff = graphgen.disjoint_union([g, g])
    dg = kb.DeviceGraph.from_numpy(union, "cuda:0")
    with pytest.raises(kb.KbError):
        ctx.refine_batch(dg, voff, np.array([2, 2], dtype=np.int32), kb.Options(subject=kb.SUBJECT_ALL))


def test_bench_batch_workload_subset_equals_oracle(ctx):
    # The batching workload bench.py times (4,096 Erdos-Renyi graphs, edges
    # lognormal in [1e3, 2e6], k uniform 1..10), refined in one kb_refine_batch
    # call; a deterministic subset of its graphs -- the smallest, the largest,
    # the ones with k = 1 and k = 10 at both ends of the size range, and random
    # ones -- is compared with the oracle graph by graph, every level.
    union, voff, ks = graphgen.batch_union_torch(device="cuda:0")
    dg = kb.DeviceGraph(union["row_offsets"], union["col"], union["elabel"], union["vlabel"])
    levels, counts, lc = ctx.refine_batch(dg, voff, ks, kb.Options())
    torch.cuda.synchronize()
    sizes = np.diff(voff)
    order = np.argsort(sizes, kind="stable")
    pick = {int(order[0]), int(order[1]), int(order[-1]), int(order[-2])}
    for kk in (1, 10):
        idx = np.nonzero(ks == kk)[0]
        if idx.size:
            pick |= {int(idx[np.argmin(sizes[idx])]), int(idx[np.argmax(sizes[idx])])}
    rng = np.random.Generator(np.random.PCG64(77))
    pick |= set(int(x) for x in rng.choice(len(ks), size=10, replace=False))
    row = union["row_offsets"]
    kmax = int(ks.max())
    for j in sorted(pick):
        a, b = int(voff[j]), int(voff[j + 1])
        e0, e1 = int(row[a].item()), int(row[b].item())
        g = graphgen.Graph(n=b - a, m=e1 - e0, row_offsets=(row[a:b + 1] - e0).cpu().numpy(),
                           col=(union["col"][e0:e1] - a).cpu().numpy(), elabel=union["elabel"][e0:e1].cpu().numpy(),
                           vlabel=union["vlabel"][a:b].cpu().numpy())
        L, C, lcj = oracle.refine_graph(g, 0, True, True, k=int(ks[j]), early_stop=True)
        got = levels[:, a:b].cpu().numpy()
        for i in range(kmax + 1):
            src = min(i, int(ks[j]))
            assert np.array_equal(got[i], L[src]), (j, i, g.n, g.m)
            assert counts[j, i] == C[src], (j, i)
        assert lc[j] == lcj, (j, lc[j], lcj)
    del levels, dg, union
    torch.cuda.empty_cache()
