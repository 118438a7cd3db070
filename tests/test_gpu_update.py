"""Incremental refinement (kb_refine_update): the levels of a graph, updated
after edge insertions, deletions and relabellings (and vertex relabellings),
must equal the oracle's levels of the new graph, element by element."""
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


def mutate(g, rng, n_ins=0, n_del=0, n_relabel=0, n_vrelabel=0, hot=None):
    """A changed copy of g and the (source, target) ends of every touched edge."""
    src, dst, lab = g.edges()
    keep = np.ones(src.shape[0], dtype=bool)
    if n_del and src.shape[0]:
        keep[rng.choice(src.shape[0], size=min(n_del, src.shape[0]), replace=False)] = False
    ts, td = [src[~keep]], [dst[~keep]]
    src, dst, lab = src[keep], dst[keep], lab[keep].copy()
    if n_relabel and src.shape[0]:
        idx = rng.choice(src.shape[0], size=min(n_relabel, src.shape[0]), replace=False)
        lab[idx] = lab[idx] + 1 + rng.integers(0, 3, size=idx.shape[0])
        ts.append(src[idx])
        td.append(dst[idx])
    if n_ins:
        s = rng.integers(0, g.n, size=n_ins)
        d = rng.integers(0, g.n, size=n_ins) if hot is None else rng.choice(hot, size=n_ins)
        src = np.concatenate([src, s])
        dst = np.concatenate([dst, d])
        lab = np.concatenate([lab, rng.integers(0, 4, size=n_ins)])
        ts.append(s)
        td.append(d)
    vl = g.vlabel.copy()
    if n_vrelabel:
        vl[rng.choice(g.n, size=n_vrelabel, replace=False)] = rng.integers(0, 50, size=n_vrelabel)
    g2 = graphgen.from_edges(g.n, src, dst, lab, vl)
    return g2, np.concatenate(ts).astype(np.int64), np.concatenate(td).astype(np.int64)


def changed_for(d, ts, td):
    return {0: ts, 1: td, 2: np.concatenate([ts, td])}[d]


def check(ctx, g, g2, changed, d, vl, el, k, early_stop=True, **kw):
    opts = kb.Options(direction=d, use_vertex_labels=vl, use_edge_labels=el, early_stop=early_stop, **kw)
    old = ctx.refine(kb.DeviceGraph.from_numpy(g, "cuda:0"), k, opts).levels.clone()
    ch = torch.from_numpy(np.asarray(changed, dtype=np.int32)).to("cuda:0")
    res, work = ctx.refine_update(kb.DeviceGraph.from_numpy(g2, "cuda:0"), old, ch, opts)
    L, C, lc = oracle.refine_graph(g2, d, vl, el, k=k, early_stop=early_stop)
    got = res.levels.cpu().numpy()
    for i in range(k + 1):
        if not np.array_equal(got[i], L[i]):
            bad = np.nonzero(got[i] != L[i])[0]
            raise AssertionError("level %d differs at %d vertices (dir %d vl %s el %s %s)" % (i, bad.size, d, vl, el, kw))
    assert np.array_equal(res.counts, C) and res.levels_computed == lc
    return work


@pytest.fixture(scope="module")
def er_tiny():
    return graphgen.make(graphgen.CONFIG_TINY)


@pytest.fixture(scope="module")
def power_law():
    return graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.002, seed=21))


def _ran_full(work, n):
    # the call ran as a full refinement: every computed level reports n
    return work[0] == n and all(w in (0, n) for w in work[1:])


@pytest.mark.parametrize("d", [0, 1, 2])
def test_small_changes(ctx, er_tiny, power_law, d):
    rng = np.random.Generator(np.random.PCG64(40 + d))
    for g in (er_tiny, power_law):
        g2, ts, td = mutate(g, rng, n_ins=5, n_del=5, n_relabel=3)
        work = check(ctx, g, g2, changed_for(d, ts, td), d, True, True, 8, early_stop=False)
        # level 1 re-keys whole label classes: either later levels re-key only
        # part of the graph, or the first round's work set was so large that
        # the call ran as a full refinement
        assert work[2:].max() < g.n or _ran_full(work, g.n)
        # without vertex labels level 0 is one block: always the full refinement
        work = check(ctx, g, g2, changed_for(d, ts, td), d, False, True, 6, early_stop=False)
        assert _ran_full(work, g.n) or len(ts) + len(td) == 0
        check(ctx, g, g2, changed_for(d, ts, td), d, True, False, 6)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_incremental_path_on_fine_level0(ctx, d):
    # thousands of vertex labels make level-0 blocks small: a few changed
    # edges touch few of them, so the rounds re-key only work sets
    g = graphgen.erdos_renyi(20_000, 60_000, 4000, 3, seed=70 + d)
    rng = np.random.Generator(np.random.PCG64(71 + d))
    g2, ts, td = mutate(g, rng, n_ins=4, n_del=4, n_relabel=2)
    work = check(ctx, g, g2, changed_for(d, ts, td), d, True, True, 6, early_stop=False)
    assert not _ran_full(work, g.n) and 0 < work[1] < g.n // 4


def test_no_change_rekeys_nothing(ctx, power_law):
    work = check(ctx, power_law, power_law, np.zeros(0, dtype=np.int32), 0, True, True, 6, early_stop=False)
    assert work[1:].sum() == 0


@pytest.mark.parametrize("d", [0, 1, 2])
def test_large_and_hub_changes(ctx, power_law, d):
    rng = np.random.Generator(np.random.PCG64(50 + d))
    # half the edges replaced; edges into the hottest vertices; hub paths and weak hash
    g2, ts, td = mutate(power_law, rng, n_ins=power_law.m // 2, n_del=power_law.m // 2)
    check(ctx, power_law, g2, changed_for(d, ts, td), d, True, True, 6)
    hot = np.argsort(np.bincount(power_law.col, minlength=power_law.n))[-5:]
    g3, ts, td = mutate(power_law, rng, n_ins=200, n_del=50, hot=hot)
    check(ctx, power_law, g3, changed_for(d, ts, td), d, True, True, 6, hub_threshold=40)
    check(ctx, power_law, g3, changed_for(d, ts, td), d, True, True, 5, hash_mode=1)


def test_vertex_relabelling(ctx, er_tiny):
    rng = np.random.Generator(np.random.PCG64(60))
    g2, ts, td = mutate(er_tiny, rng, n_ins=3, n_vrelabel=20)
    for d in (0, 1, 2):
        check(ctx, er_tiny, g2, changed_for(d, ts, td), d, True, True, 6)


def test_random_tiny_updates(ctx):
    rng = np.random.Generator(np.random.PCG64(61))
    for _ in range(120):
        g = graphgen.tiny_random(rng, n_max=40, m_max=120, n_labels=int(rng.integers(1, 4)))
        g2, ts, td = mutate(g, rng, n_ins=int(rng.integers(0, 6)), n_del=int(rng.integers(0, 6)),
                            n_relabel=int(rng.integers(0, 3)), n_vrelabel=int(rng.integers(0, 2)))
        d = int(rng.integers(0, 3))
        check(ctx, g, g2, changed_for(d, ts, td), d, bool(rng.integers(0, 2)), bool(rng.integers(0, 2)),
              int(rng.integers(0, 7)), early_stop=bool(rng.integers(0, 2)), hub_threshold=int(rng.choice([0, 2, 5])))


def test_edge_cases_and_errors(ctx, er_tiny):
    for g in (graphgen.from_edges(1, [0, 0], [0, 0], [1, 2], [5]), graphgen.from_edges(4, [], [], [], [1, 2, 1, 2]),
              graphgen.path_graph(300)):
        rng = np.random.Generator(np.random.PCG64(62))
        g2, ts, td = mutate(g, rng, n_ins=2)
        for d in (0, 1, 2):
            check(ctx, g, g2, changed_for(d, ts, td), d, True, True, 5)
    dg = kb.DeviceGraph.from_numpy(er_tiny, "cuda:0")
    old = ctx.refine(dg, 3, kb.Options()).levels.clone()
    with pytest.raises(kb.KbError):
        ctx.refine_update(dg, old, torch.tensor([er_tiny.n + 3], dtype=torch.int32, device="cuda:0"))
    bad = old.clone()
    bad[2, 7] = er_tiny.n + 1
    with pytest.raises(kb.KbError):
        ctx.refine_update(dg, bad, torch.tensor([1], dtype=torch.int32, device="cuda:0"))
    with pytest.raises(kb.KbError):
        ctx.refine_update(dg, old, torch.tensor([1], dtype=torch.int32, device="cuda:0"),
                          kb.Options(subject=kb.SUBJECT_ALL))
