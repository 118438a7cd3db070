"""Summary graph (kb_summary) on the GPU against the CPU oracle: the same
triples in the same order (first occurrence in the edge list)."""
import numpy as np
import pytest

import graphgen
import oracle
from paper_fixture import canonical_ids, load, load_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = kb.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to("cuda:0")


def assert_summary(ctx, g, d, el, a, b):
    exp = oracle.summary(g, d, el, a, b)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    got = ctx.summary(dg, _dev(a), _dev(b), direction=d, use_edge_labels=el)
    for x, y in zip(got, exp):
        assert np.array_equal(x.cpu().numpy(), y)
    assert ctx.summary_count(dg, _dev(a), _dev(b), direction=d, use_edge_labels=el) == len(exp[0])
    return len(exp[0])


def test_paper_example(ctx):
    g, tables = load()
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    for table, i_src, i_dst, expected in load_summary():
        t = tables[table]
        a = canonical_ids(t["levels"][i_src], g.n)
        b = canonical_ids(t["levels"][i_dst], g.n)
        s, l, d = ctx.summary(dg, _dev(a), _dev(b), direction=t["direction"], use_edge_labels=t["use_edge_labels"])
        assert list(zip(s.tolist(), l.tolist(), d.tolist())) == expected, table


@pytest.fixture(scope="module")
def er_tiny():
    return graphgen.make(graphgen.CONFIG_TINY)


@pytest.fixture(scope="module")
def power_law():
    return graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.002, seed=21))


@pytest.mark.parametrize("d", [0, 1])
@pytest.mark.parametrize("el", [True, False])
def test_levels_of_a_refinement(ctx, er_tiny, power_law, d, el):
    for g in (er_tiny, power_law):
        L, _, _ = oracle.refine_graph(g, d, True, el, k=4, early_stop=False)
        for i in (1, 2, 4):
            assert assert_summary(ctx, g, d, el, L[i], L[i - 1]) > 0  # the paper's layering
            assert_summary(ctx, g, d, el, L[i], L[i])  # quotient graph


def test_special_partitions(ctx, power_law):
    g = power_law
    ident = np.arange(g.n, dtype=np.int32)
    zero = np.zeros(g.n, dtype=np.int32)
    assert_summary(ctx, g, 0, True, ident, ident)
    assert assert_summary(ctx, g, 1, True, zero, zero) == len(np.unique(g.elabel))
    rng = np.random.Generator(np.random.PCG64(5))
    extreme = rng.choice(np.array([-2147483648, -1, 0, 7, 2147483647], dtype=np.int32), size=g.n)
    assert_summary(ctx, g, 0, True, extreme, rng.integers(-3, 3, size=g.n).astype(np.int32))


def test_larger_graph(ctx):
    # 2e6 edges, Chung-Lu with hubs: many table probes, hot triples, several tiles per CTA
    g = graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.02, seed=22))
    L, _, _ = oracle.refine_graph(g, 0, True, True, k=3, early_stop=False)
    assert_summary(ctx, g, 0, True, L[3], L[2])
    assert_summary(ctx, g, 1, False, L[3], L[3])


def test_edge_cases_and_errors(ctx, er_tiny):
    cases = [graphgen.from_edges(1, [0, 0, 0], [0, 0, 0], [1, 1, 2], [5]),
             graphgen.from_edges(4, [], [], [], [1, 2, 3, 4]),
             graphgen.path_graph(1000)]
    for g in cases:
        for d in (0, 1):
            ids = np.arange(g.n, dtype=np.int32)
            assert_summary(ctx, g, d, True, ids, ids)
    dg = kb.DeviceGraph.from_numpy(er_tiny, "cuda:0")
    ids = _dev(np.arange(er_tiny.n))
    with pytest.raises(kb.KbError):
        ctx.summary(dg, ids, ids, direction=2)
    with pytest.raises(kb.KbError):
        ctx.summary(dg, ids, ids, capacity=10)  # far fewer entries than summary edges
    bad = graphgen.Graph(n=er_tiny.n, m=er_tiny.m, row_offsets=er_tiny.row_offsets, col=er_tiny.col.copy(),
                         elabel=er_tiny.elabel, vlabel=er_tiny.vlabel)
    bad.col[3] = er_tiny.n + 5
    with pytest.raises(kb.KbError):
        ctx.summary(kb.DeviceGraph.from_numpy(bad, "cuda:0"), ids, ids)
    # the context stays usable
    assert_summary(ctx, er_tiny, 0, True, np.arange(er_tiny.n), np.arange(er_tiny.n))
