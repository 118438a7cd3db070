"""Prepared graphs (kb_graph_prepare / kb_refine_prepared): the per-graph
structures built once give, call after call, exactly the oracle's levels for
every per-call option, with the locality order on and off."""
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


def _graphs():
    rng = np.random.Generator(np.random.PCG64(12))
    # hubs (multi-chunk), medium and small vertices, edgeless vertices
    n = 6000
    deg = rng.integers(0, 6, size=n)
    deg[::301] = rng.integers(33, 900, size=deg[::301].shape[0])
    deg[[5, 17]] = [3000, 1500]
    src = np.repeat(np.arange(n), deg)
    dst = rng.integers(0, n, size=src.shape[0])
    mixed = graphgen.from_edges(n, src, dst, rng.integers(0, 4, size=src.shape[0]), rng.integers(0, 3, size=n))
    return [graphgen.make(graphgen.CONFIG_TINY), graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.002, seed=7)),
            mixed]


@pytest.mark.parametrize("reorder", [1, 2])
@pytest.mark.parametrize("d", [kb.DIR_OUT, kb.DIR_IN, kb.DIR_BOTH])
def test_prepared_equals_oracle_for_every_call_option(ctx, d, reorder):
    for g in _graphs():
        dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
        base = kb.Options(direction=d, reorder=reorder, hub_threshold=512)
        with ctx.prepare(dg, base) as pg:
            assert pg.info()["reorder"] == (1 if reorder == 2 else 0)
            # several calls on one prepared graph, varying the per-call fields
            calls = [dict(), dict(early_stop=False), dict(use_vertex_labels=False), dict(rekey_all=True),
                     dict(hash_mode=1, load_factor=0.8), dict(small_task_vertices=32, medium_split=64)]
            for kw in calls:
                o = kb.Options(direction=d, reorder=reorder, hub_threshold=512, **kw)
                res = ctx.refine(pg, 6, o)
                L, C, lc = oracle.refine_graph(g, d, o.use_vertex_labels, True, k=6, early_stop=o.early_stop)
                assert np.array_equal(res.levels.cpu().numpy(), L), (d, reorder, kw)
                assert np.array_equal(res.counts, C) and res.levels_computed == lc, (d, reorder, kw)


def test_prepared_cse_subjects(ctx):
    g = _graphs()[2]
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    with ctx.prepare(dg, kb.Options(reorder=2)) as pg:
        for subj in (kb.SUBJECT_ALL, kb.SUBJECT_LABEL, kb.SUBJECT_ID):
            o = kb.Options(reorder=2, subject=subj, early_stop=False)
            res = ctx.refine(pg, 4, o)
            L, C, _ = oracle.refine_graph(g, 0, True, True, k=4, early_stop=False, subject=subj)
            assert np.array_equal(res.levels.cpu().numpy(), L), subj


def test_prepared_locality_order_on_by_default_for_large_graphs(ctx):
    # 2^22 processed edges or more: the automatic locality order is on
    g = graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.045, seed=3))
    assert g.m >= 1 << 22
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    with ctx.prepare(dg) as pg:
        info = pg.info()
        assert info["reorder"] == 1 and info["n_hubs"] > 0 and info["device_bytes"] > 4 * g.m
        res = ctx.refine(pg, 4)
        again = ctx.refine(pg, 4)
    L, C, lc = oracle.refine_graph(g, 0, True, True, k=4)
    assert np.array_equal(res.levels.cpu().numpy(), L) and np.array_equal(res.counts, C)
    assert torch.equal(res.levels, again.levels)


def test_prepared_rejects_other_direction_and_released_handle(ctx):
    g = graphgen.make(graphgen.CONFIG_TINY)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    pg = ctx.prepare(dg, kb.Options(direction=kb.DIR_OUT))
    with pytest.raises(kb.KbError):
        ctx.refine(pg, 2, kb.Options(direction=kb.DIR_IN))
    with pytest.raises(kb.KbError):
        ctx.refine(pg, 2, kb.Options(use_edge_labels=False))
    res = ctx.refine(pg, 2)  # still usable after the rejections
    L, _, _ = oracle.refine_graph(g, 0, True, True, k=2)
    assert np.array_equal(res.levels.cpu().numpy(), L)
    pg.release()
    with pytest.raises(kb.KbError):
        ctx.refine(pg, 2)


def test_prepare_validates_once(ctx):
    g = graphgen.make(graphgen.CONFIG_TINY)
    col = g.col.copy()
    col[7] = g.n + 5  # a neighbour id out of range
    bad = graphgen.Graph(n=g.n, m=g.m, row_offsets=g.row_offsets, col=col, elabel=g.elabel, vlabel=g.vlabel)
    dg = kb.DeviceGraph.from_numpy(bad, "cuda:0")
    with pytest.raises(kb.KbError) as e:
        ctx.prepare(dg)
    assert e.value.status == 1
