"""GPU path against the CPU oracle, element by element (exact integers).

Every test calls the library through its C ABI (the ctypes binding) and
compares all levels, block counts and the last refined level with the
oracle on the same seeded graph.
"""
import numpy as np
import pytest

import graphgen
import oracle
from paper_fixture import load, partition

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = kb.Context(0)
    yield c
    c.close()


def gpu_levels(ctx, g, d, vl, el, k, early_stop=True, **kw):
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    res = ctx.refine(dg, k, kb.Options(direction=d, use_vertex_labels=vl, use_edge_labels=el,
                                       early_stop=early_stop, **kw))
    torch.cuda.synchronize()
    return res.levels.cpu().numpy(), res.counts, res.levels_computed


def assert_same(ctx, g, d, vl, el, k, early_stop=True, **kw):
    L, C, lc = oracle.refine_graph(g, d, vl, el, k=k, early_stop=early_stop, subject=kw.get("subject", 0))
    got, gc, glc = gpu_levels(ctx, g, d, vl, el, k, early_stop, **kw)
    for i in range(k + 1):
        if not np.array_equal(got[i], L[i]):
            bad = np.nonzero(got[i] != L[i])[0]
            raise AssertionError("level %d differs at %d vertices, first %s: gpu %s oracle %s (dir %d vl %s el %s %s)"
                                 % (i, bad.size, bad[:5], got[i][bad[:5]], L[i][bad[:5]], d, vl, el, kw))
    assert np.array_equal(gc, C), (gc, C)
    assert glc == lc
    return L, C


# ---------------------------------------------------------------- the paper's example


@pytest.mark.parametrize("table", ["fw", "bw", "sch", "kau"])
def test_paper_tables(ctx, table):
    g, tables = load()
    t = tables[table]
    got, counts, _ = gpu_levels(ctx, g, t["direction"], t["use_vertex_labels"], t["use_edge_labels"], 2,
                                early_stop=False)
    for i, expected in t["levels"].items():
        assert partition(got[i]) == expected
        assert counts[i] == len(expected)


def test_presets_match_definitions(ctx):
    g, tables = load()
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    for name, opts in (("sch", kb.Options.schaetzle(early_stop=False)), ("kau", kb.Options.kaushik(early_stop=False))):
        res = ctx.refine(dg, 2, opts)
        got = res.levels.cpu().numpy()
        for i, expected in tables[name]["levels"].items():
            assert partition(got[i]) == expected


# ---------------------------------------------------------------- configuration 1 (ER, 10k vertices, 50k edges)


@pytest.fixture(scope="module")
def er_tiny():
    return graphgen.make(graphgen.CONFIG_TINY)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("vl,el", [(True, True), (False, True), (True, False), (False, False)])
def test_config_tiny_all_variants(ctx, er_tiny, d, vl, el):
    assert_same(ctx, er_tiny, d, vl, el, 10, early_stop=False)
    assert_same(ctx, er_tiny, d, vl, el, 10, early_stop=True)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_weak_hash_forces_compare_path(ctx, er_tiny, d):
    # hash of the previous block only: every vertex of a block collides, so
    # only the full signature compare separates them
    assert_same(ctx, er_tiny, d, True, True, 6, hash_mode=1)


@pytest.mark.parametrize("thr", [1, 3, 17, 64])
def test_hub_path_equivalent(ctx, er_tiny, thr):
    for d in (0, 1, 2):
        assert_same(ctx, er_tiny, d, True, True, 6, hub_threshold=thr)


@pytest.mark.parametrize("thr", [2, 8])
def test_hub_path_weak_hash(ctx, er_tiny, thr):
    assert_same(ctx, er_tiny, 2, True, True, 5, hub_threshold=thr, hash_mode=1)


@pytest.mark.parametrize("lf", [0.05, 0.5, 0.9])
def test_load_factor_invariance(ctx, er_tiny, lf):
    assert_same(ctx, er_tiny, 0, True, True, 8, load_factor=lf)


# ---------------------------------------------------------------- locality order of the gather


@pytest.mark.parametrize("reorder", [1, 2])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_locality_order(ctx, er_tiny, d, reorder):
    # neighbour ids moved to hotness ranks must not change a single level
    assert_same(ctx, er_tiny, d, True, True, 8, reorder=reorder)
    assert_same(ctx, er_tiny, d, False, True, 6, reorder=reorder, hash_mode=1)
    assert_same(ctx, er_tiny, d, True, False, 6, reorder=reorder, hub_threshold=17)
    assert_same(ctx, er_tiny, d, False, False, 5, early_stop=False, reorder=reorder)


@pytest.fixture(scope="module")
def power_law():
    # a small Chung-Lu graph: skewed in-degrees (a real hot head) and hubs
    return graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.002, seed=21))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_locality_order_power_law(ctx, power_law, d):
    for reorder in (1, 2):
        assert_same(ctx, power_law, d, True, True, 6, reorder=reorder)
        assert_same(ctx, power_law, d, True, True, 4, reorder=reorder, hub_threshold=40, hash_mode=1)


def test_locality_order_resume(ctx, power_law):
    L, C, _ = oracle.refine_graph(power_law, 0, True, True, k=6, early_stop=False)
    dg = kb.DeviceGraph.from_numpy(power_law, "cuda:0")
    for j in (0, 3):
        start = torch.from_numpy(L[j]).to("cuda:0")
        res = ctx.refine_from(dg, start, j, 6, kb.Options(early_stop=False, reorder=2))
        assert np.array_equal(res.levels.cpu().numpy()[j:], L[j:])
        assert np.array_equal(res.counts[j:], C[j:])


# ---------------------------------------------------------------- full bisimulation (fixpoint)


def assert_fixpoint(ctx, g, d, vl, el, max_rounds=None, initial=None, **kw):
    mr = g.n + 1 if max_rounds is None else max_rounds
    L, C, lc = oracle.refine_graph(g, d, vl, el, k=mr, early_stop=True, initial=initial, subject=kw.get("subject", 0))
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    init = torch.from_numpy(initial).to("cuda:0") if initial is not None else None
    final, cnt, rounds, stable = ctx.refine_fixpoint(
        dg, mr, kb.Options(direction=d, use_vertex_labels=vl, use_edge_labels=el, **kw), initial=init)
    assert np.array_equal(final.cpu().numpy(), L[lc])
    assert cnt == C[lc] and rounds == lc
    assert stable == (lc < mr or (lc >= 1 and np.array_equal(L[lc], L[lc - 1])))
    return lc


@pytest.mark.parametrize("d", [0, 1, 2])
def test_fixpoint_matches_oracle(ctx, er_tiny, power_law, d):
    assert_fixpoint(ctx, er_tiny, d, True, True)
    assert_fixpoint(ctx, er_tiny, d, False, False)
    assert_fixpoint(ctx, power_law, d, True, True, reorder=2)
    assert_fixpoint(ctx, power_law, d, False, True, hash_mode=1)


def test_fixpoint_cutoff_and_closed_forms(ctx, er_tiny):
    # a path of n vertices needs n-1 rounds to separate them; a cutoff stops early
    path = graphgen.path_graph(300)
    assert assert_fixpoint(ctx, path, 0, False, False) == 300
    assert assert_fixpoint(ctx, path, 0, False, False, max_rounds=7) == 7
    assert assert_fixpoint(ctx, graphgen.cycle_graph(500), 0, False, False) == 1
    # the coarsest stable refinement of a given partition
    init = (er_tiny.vlabel.astype(np.int64) * 7919 % 5).astype(np.int32)
    assert_fixpoint(ctx, er_tiny, 1, False, False, initial=init)
    assert_fixpoint(ctx, er_tiny, 0, True, True, max_rounds=0)


# ---------------------------------------------------------------- generic CSE rounds


@pytest.mark.parametrize("subject", [kb.SUBJECT_ALL, kb.SUBJECT_LABEL, kb.SUBJECT_ID])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_cse_rounds(ctx, er_tiny, power_law, d, subject):
    # Def. "cse" chained (Def. "chaining-parameterization"): subject T, label or id
    for g in (er_tiny, power_law):
        for vl, el in ((True, True), (False, True), (True, False)):
            assert_same(ctx, g, d, vl, el, 5, early_stop=False, subject=subject)
        assert_same(ctx, g, d, True, True, 8, early_stop=True, subject=subject)  # whole-level stop
    assert_same(ctx, er_tiny, d, True, True, 4, subject=subject, hash_mode=1, hub_threshold=17)
    assert_same(ctx, power_law, d, True, False, 4, subject=subject, reorder=2)


def test_cse_models_of_the_paper(ctx):
    # Eq. (gsm:schaetzle) (T, id, T)^k and Eq. (gsm:kaushik) ((OC, T, OC)^-1)^k
    g, tables = load()
    for name, opts in (("sch", kb.Options(direction=kb.DIR_OUT, use_vertex_labels=False, use_edge_labels=True,
                                          subject=kb.SUBJECT_ALL, early_stop=False)),
                       ("kau", kb.Options(direction=kb.DIR_IN, use_vertex_labels=True, use_edge_labels=False,
                                          subject=kb.SUBJECT_LABEL, early_stop=False))):
        res = ctx.refine(kb.DeviceGraph.from_numpy(g, "cuda:0"), 2, opts)
        got = res.levels.cpu().numpy()
        for i, expected in tables[name]["levels"].items():
            assert partition(got[i]) == expected


def test_cse_fixpoint_and_rejections(ctx, er_tiny):
    for subject in (kb.SUBJECT_ALL, kb.SUBJECT_LABEL):
        assert_fixpoint(ctx, er_tiny, 0, True, True, max_rounds=40, subject=subject)
    # a level-1 merge of differently labelled vertices: levels need not refine
    g = graphgen.from_edges(3, [0, 1], [2, 2], [0, 0], [7, 8, 9])
    assert_same(ctx, g, 0, True, True, 3, subject=kb.SUBJECT_ALL)
    with pytest.raises(kb.KbError):
        gpu_levels(ctx, er_tiny, 0, True, True, 3, subject=4)


# ---------------------------------------------------------------- random small graphs and edge cases


def test_random_tiny_graphs(ctx):
    rng = np.random.Generator(np.random.PCG64(31))
    for _ in range(150):
        g = graphgen.tiny_random(rng, n_max=40, m_max=120, n_labels=int(rng.integers(1, 4)))
        d = int(rng.integers(0, 3))
        assert_same(ctx, g, d, bool(rng.integers(0, 2)), bool(rng.integers(0, 2)), int(rng.integers(0, 7)),
                    hash_mode=int(rng.integers(0, 2)), hub_threshold=int(rng.choice([0, 1, 2, 5])),
                    reorder=int(rng.choice([1, 2])), subject=int(rng.choice([0, 0, 1, 2, 3])))


def test_edge_cases(ctx):
    cases = [
        graphgen.from_edges(1, [], [], [], [5]),
        graphgen.from_edges(1, [0, 0, 0], [0, 0, 0], [1, 1, 2], [5]),  # self loops, parallel edges
        graphgen.from_edges(5, [], [], [], [3, -7, 3, 2147483647, -2147483648]),
        graphgen.path_graph(1000),
        graphgen.cycle_graph(777),
        graphgen.binary_tree(10),
    ]
    for g in cases:
        for d in (0, 1, 2):
            for k in (0, 1, 5):
                assert_same(ctx, g, d, True, True, k)
                assert_same(ctx, g, d, False, False, k, early_stop=False)
                assert_same(ctx, g, d, True, True, k, reorder=2)


def test_extreme_labels(ctx):
    rng = np.random.Generator(np.random.PCG64(3))
    g = graphgen.erdos_renyi(2000, 9000, 3, 3, seed=5)
    g.elabel = rng.choice(np.array([-2147483648, -1, 0, 2147483647], dtype=np.int32), size=g.m)
    g.vlabel = rng.choice(np.array([-2147483648, 7, 2147483647], dtype=np.int32), size=g.n)
    for d in (0, 1, 2):
        assert_same(ctx, g, d, True, True, 6)


def test_hot_slot_and_hubs(ctx):
    # one vertex receives every edge and one vertex sends 100k edges: a hot
    # table slot, a multi-chunk hub with heavy duplicate pairs, and hubs in
    # the in-direction
    n = 50_000
    rng = np.random.Generator(np.random.PCG64(8))
    src = np.concatenate([np.arange(n), np.full(100_000, 17), rng.integers(0, n, 30_000)])
    dst = np.concatenate([np.full(n, 3), rng.integers(0, n, 100_000), rng.integers(0, 100, 30_000)])
    lab = rng.integers(0, 3, size=src.shape[0])
    g = graphgen.from_edges(n, src, dst, lab, rng.integers(0, 4, size=n))
    for d in (0, 1, 2):
        assert_same(ctx, g, d, True, True, 6)
        assert_same(ctx, g, d, False, True, 4, hash_mode=1)


def test_subtile_boundaries(ctx):
    # degrees around the sub-tile split and the default hub threshold (1024):
    # 1023, 1024 (largest non-hub), 1025 (hub), 32/33 (small/medium edge),
    # larger hubs, mixed with zero-degree runs, over several tiles with a
    # ragged last tile
    degs = []
    rng = np.random.Generator(np.random.PCG64(12))
    for t in range(9):
        degs += [1023, 0, 0, 1024, 1, 1025, 0, 32, 33, 2049, 0] + list(rng.integers(0, 9, size=245))
    degs = np.array(degs[: 9 * 256 - 77])
    n = degs.shape[0]
    src = np.repeat(np.arange(n), degs)
    dst = rng.integers(0, n, size=src.shape[0])
    dst[::3] = rng.integers(0, 40, size=dst[::3].shape[0])  # many duplicate pairs
    lab = rng.integers(0, 2, size=src.shape[0])
    g = graphgen.from_edges(n, src, dst, lab, rng.integers(0, 3, size=n))
    for d in (0, 1, 2):
        assert_same(ctx, g, d, True, True, 5)
    assert_same(ctx, g, 0, True, True, 4, hash_mode=1)


# ---------------------------------------------------------------- singleton blocks


def test_singletons_random_tiny(ctx):
    # rounds skip vertices alone in their previous block; re-keying them gives
    # the same levels, and both equal the oracle
    rng = np.random.Generator(np.random.PCG64(33))
    for _ in range(100):
        g = graphgen.tiny_random(rng, n_max=40, m_max=120, n_labels=int(rng.integers(1, 6)))
        d = int(rng.integers(0, 3))
        kw = dict(hash_mode=int(rng.integers(0, 2)), hub_threshold=int(rng.choice([0, 1, 2, 5])))
        k = int(rng.integers(1, 7))
        vl, el = bool(rng.integers(0, 2)), bool(rng.integers(0, 2))
        for rekey in (False, True):
            assert_same(ctx, g, d, vl, el, k, early_stop=bool(rng.integers(0, 2)), rekey_all=rekey, **kw)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_singletons_power_law(ctx, power_law, d):
    # hubs and most vertices of a power-law graph are alone in their block
    # after one or two rounds: the hub, medium and small paths all skip them
    for rekey in (False, True):
        assert_same(ctx, power_law, d, True, True, 6, early_stop=False, rekey_all=rekey)
        assert_same(ctx, power_law, d, True, True, 5, hub_threshold=40, rekey_all=rekey)
        assert_same(ctx, power_law, d, False, True, 5, hub_threshold=8, hash_mode=1, rekey_all=rekey)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_frozen_edgeless_blocks(ctx, d):
    # two thirds of the vertices without out-edges, in a few label classes;
    # edges concentrated on a small head so many vertices also lack in-edges
    rng = np.random.Generator(np.random.PCG64(34 + d))
    n = 30_000
    src = rng.integers(0, n // 3, size=40_000)
    dst = np.minimum(rng.zipf(1.6, size=40_000) - 1, n - 1)
    g = graphgen.from_edges(n, src, dst, rng.integers(0, 3, size=src.shape[0]), rng.integers(0, 5, size=n))
    for rekey in (False, True):
        assert_same(ctx, g, d, True, True, 7, early_stop=False, rekey_all=rekey)
        assert_same(ctx, g, d, False, True, 5, rekey_all=rekey)
    L, C, _ = oracle.refine_graph(g, d, True, True, k=7, early_stop=False)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    for j in (1, 2):
        res = ctx.refine_from(dg, torch.from_numpy(L[j]).to("cuda:0"), j, 7, kb.Options(direction=d, early_stop=False))
        assert np.array_equal(res.levels.cpu().numpy()[j:], L[j:])


@pytest.mark.parametrize("task", [32, 33, 100, 1000])
def test_frozen_blocks_task_sizes(ctx, power_law, task):
    # warp tasks that do not start on a bitmap word: windows of consecutive
    # vertices (round 1) and of refining vertices only (later rounds)
    for d in (0, 2):
        assert_same(ctx, power_law, d, True, True, 6, early_stop=False, small_task_vertices=task)
    assert_same(ctx, power_law, 1, True, True, 5, small_task_vertices=task, hash_mode=1, hub_threshold=40)


def test_singletons_from_start_partition(ctx, er_tiny):
    dg = kb.DeviceGraph.from_numpy(er_tiny, "cuda:0")
    n = er_tiny.n
    # every vertex alone at the start: every later level is the identity
    start = torch.arange(n, dtype=torch.int32, device="cuda:0")
    res = ctx.refine_from(dg, start, 0, 4, kb.Options(early_stop=False))
    assert np.array_equal(res.levels.cpu().numpy(), np.tile(np.arange(n, dtype=np.int32), (5, 1)))
    assert list(res.counts) == [n] * 5
    # half the vertices alone, the rest in three blocks
    init = np.arange(n, dtype=np.int32)
    init[n // 2:] = n + (np.arange(n - n // 2) % 3)
    L, C, _ = oracle.refine_graph(er_tiny, 0, False, True, k=5, early_stop=False, initial=init)
    for rekey in (False, True):
        res = ctx.refine_from(dg, torch.from_numpy(init).to("cuda:0"), 0, 5,
                              kb.Options(early_stop=False, rekey_all=rekey))
        assert np.array_equal(res.levels.cpu().numpy(), L) and np.array_equal(res.counts, C)


# ---------------------------------------------------------------- resume, initial partition, host buffers


def test_refine_from_matches_full_run(ctx, er_tiny):
    for d in (0, 1, 2):
        L, C, _ = oracle.refine_graph(er_tiny, d, True, True, k=8, early_stop=False)
        dg = kb.DeviceGraph.from_numpy(er_tiny, "cuda:0")
        for j in (0, 2, 5):
            start = torch.from_numpy(L[j]).to("cuda:0")
            res = ctx.refine_from(dg, start, j, 8, kb.Options(direction=d, early_stop=False))
            got = res.levels.cpu().numpy()
            assert np.array_equal(got[j:], L[j:])
            assert np.array_equal(res.counts[j:], C[j:])


def test_start_partition_rows_at_any_alignment(ctx):
    # a starting partition passed as a row of a levels array: with n odd its
    # rows start at every 4-byte offset modulo 16 (the level-0 label pass
    # reads 16 bytes at a time only from 16-byte aligned keys)
    g = graphgen.erdos_renyi(3001, 12000, 5, 3, seed=17)
    L, C, _ = oracle.refine_graph(g, 0, True, True, k=6, early_stop=False)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    rows = torch.from_numpy(L).to("cuda:0")
    for j in (0, 1, 2, 3):
        assert (rows[j].data_ptr() - rows.data_ptr()) % 16 == (4 * j * g.n) % 16
        res = ctx.refine_from(dg, rows[j], j, 6, kb.Options(early_stop=False))
        assert np.array_equal(res.levels.cpu().numpy()[j:], L[j:])
        assert np.array_equal(res.counts[j:], C[j:])


def test_initial_partition(ctx, er_tiny):
    init = (er_tiny.vlabel.astype(np.int64) * 1000003 % 7 - 3).astype(np.int32)
    L, C, _ = oracle.refine_graph(er_tiny, 0, False, True, k=6, early_stop=False, initial=init)
    dg = kb.DeviceGraph.from_numpy(er_tiny, "cuda:0")
    res = ctx.refine_from(dg, torch.from_numpy(init).to("cuda:0"), 0, 6, kb.Options(early_stop=False))
    assert np.array_equal(res.levels.cpu().numpy(), L) and np.array_equal(res.counts, C)


def test_host_buffers(ctx, er_tiny):
    # every row reaches the host buffer (rows are copied as they become final,
    # early-stop copies included), whatever the output held before
    for d in (0, 2):
        for early, k in ((True, 10), (False, 6), (True, 0)):
            L, C, lc = oracle.refine_graph(er_tiny, d, True, True, k=k, early_stop=early)
            out = np.full((k + 1, er_tiny.n), -1, dtype=np.int32)
            res = ctx.refine_host(er_tiny.row_offsets, er_tiny.col, er_tiny.elabel, er_tiny.vlabel, k,
                                  kb.Options(direction=d, early_stop=early), out=out)
            assert np.array_equal(out, L) and np.array_equal(res.levels, L), (d, early, k)
            assert np.array_equal(res.counts, C) and res.levels_computed == lc


def test_torch_workspace(er_tiny):
    with kb.Context(0, torch_workspace=True) as c:
        assert_same(c, er_tiny, 1, True, True, 6)
        dg = kb.DeviceGraph.from_numpy(er_tiny, "cuda:0")
        need = c.workspace_size(dg, 6, kb.Options(direction=1))
        assert need > 0


def test_invalid_inputs_rejected(ctx):
    g = graphgen.erdos_renyi(100, 300, 2, 2, seed=1)
    bad = graphgen.Graph(n=g.n, m=g.m, row_offsets=g.row_offsets.copy(), col=g.col.copy(), elabel=g.elabel,
                         vlabel=g.vlabel)
    bad.col[5] = g.n + 3
    with pytest.raises(kb.KbError) as e:
        gpu_levels(ctx, bad, 0, True, True, 3)
    assert e.value.status == 1
    bad2 = graphgen.Graph(n=g.n, m=g.m, row_offsets=g.row_offsets.copy(), col=g.col, elabel=g.elabel,
                          vlabel=g.vlabel)
    bad2.row_offsets[10], bad2.row_offsets[11] = bad2.row_offsets[11] + 1, bad2.row_offsets[10]
    with pytest.raises(kb.KbError):
        gpu_levels(ctx, bad2, 0, True, True, 3)
    with pytest.raises(kb.KbError):
        gpu_levels(ctx, g, 0, True, True, 3, hub_threshold=5000)
    with pytest.raises(kb.KbError):
        gpu_levels(ctx, g, 0, True, True, 3, reorder=3)
    # the context stays usable after errors
    assert_same(ctx, g, 0, True, True, 3)


def _late_split_graphs():
    # graphs whose blocks keep splitting for many rounds while others stay put
    n = 500
    spine = np.arange(n - 1)
    leaves = np.arange(n, 3 * n)
    comb = graphgen.from_edges(3 * n, np.concatenate([spine, (leaves - n) // 2]),
                               np.concatenate([spine + 1, leaves]), None, None)
    paths, _ = graphgen.disjoint_union([graphgen.path_graph(L) for L in range(1, 80)])
    return [graphgen.path_graph(2000), graphgen.binary_tree(11), comb, paths, _path_and_cycles()]


def _path_and_cycles():
    # a labelled path next to 300 directed 10-cycles of another label: the
    # path's block splits every round, the cycles' blocks never do
    parts = [graphgen.path_graph(500)] + [graphgen.cycle_graph(10) for _ in range(300)]
    g, off = graphgen.disjoint_union(parts)
    g.vlabel = np.ones(g.n, dtype=np.int32)
    g.vlabel[:500] = 0
    return g


@pytest.mark.parametrize("d", [0, 1, 2])
def test_clean_blocks(ctx, power_law, d):
    # rounds skip the blocks none of whose members has an edge into a block
    # that the last round split; skipping and re-keying everything give the
    # same levels, and both equal the oracle (locality order on and off,
    # resumed runs included)
    for g in _late_split_graphs() + [power_law]:
        for rekey in (False, True):
            assert_same(ctx, g, d, True, True, 12, early_stop=False, rekey_all=rekey)
        assert_same(ctx, g, d, False, True, 9, reorder=2)
    g = _path_and_cycles()
    L, C, _ = oracle.refine_graph(g, d, True, True, k=12, early_stop=False)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    res = ctx.refine_from(dg, torch.from_numpy(L[3]).to("cuda:0"), 3, 12, kb.Options(direction=d, early_stop=False))
    assert np.array_equal(res.levels.cpu().numpy()[3:], L[3:])


def test_clean_blocks_are_skipped(ctx):
    # the cycles' blocks are clean from the second round on: only the path's
    # vertices (and its edges) are re-keyed after that
    g = _path_and_cycles()
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    ctx.set_timing(2)
    res = ctx.refine(dg, 12, kb.Options(direction=kb.DIR_OUT, early_stop=False))
    ctx.set_timing(0)
    L, _, _ = oracle.refine_graph(g, 0, True, True, k=12, early_stop=False)
    assert np.array_equal(res.levels.cpu().numpy(), L)
    work = ctx.round_work()
    assert len(work) == 12
    keyed = [sum(v for v, _ in w.values()) for w in work]
    assert keyed[0] == g.n
    assert all(v <= 500 for v in keyed[2:]), keyed


@pytest.mark.parametrize("d", [0, 1, 2])
def test_small_label_level0_boundaries(ctx, power_law, d):
    # level 0 over keys in [0, 8192) takes each label's smallest vertex
    # directly; other keys go through the block table.  Moving the labels
    # across the boundary (8191 -> 8192, or below 0) keeps the partition, so
    # every level stays identical, and equal to the oracle's.
    g = graphgen.Graph(n=power_law.n, m=power_law.m, row_offsets=power_law.row_offsets, col=power_law.col,
                       elabel=power_law.elabel, vlabel=power_law.vlabel.copy())
    base = (power_law.vlabel.astype(np.int64) % 3) * 4095  # 0, 4095, 8190
    ref = None
    for shift in (0, 1, 2, -8191):  # 8191 stays inside the range; 8192 and negative keys do not
        g.vlabel = (base + shift).astype(np.int32)
        for rekey in (False, True):
            got, _, _ = gpu_levels(ctx, g, d, True, True, 6, early_stop=False, rekey_all=rekey)
            if ref is None:
                ref = got
                L, _, _ = oracle.refine_graph(g, d, True, True, k=6, early_stop=False)
                assert np.array_equal(got, L)
            assert np.array_equal(got, ref), (shift, rekey)
        assert np.array_equal(gpu_levels(ctx, g, d, True, True, 6, early_stop=False, reorder=2)[0], ref), shift


def test_small_label_level0_single_vertex_labels(ctx, er_tiny):
    # up to 8192 distinct keys (dense), every vertex its own label (keys up
    # to n - 1 > 8192), one label for all; plain and prepared (locality order)
    ids = np.arange(er_tiny.n, dtype=np.int32)
    for lab in (ids % 8192, ids[::-1] % 8192, ids, np.zeros(er_tiny.n, dtype=np.int32),
                np.full(er_tiny.n, 8191, dtype=np.int32)):
        g = graphgen.Graph(n=er_tiny.n, m=er_tiny.m, row_offsets=er_tiny.row_offsets, col=er_tiny.col,
                           elabel=er_tiny.elabel, vlabel=lab)
        assert_same(ctx, g, 0, True, True, 5)
        L, C, _ = oracle.refine_graph(g, 0, True, True, k=5)
        dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
        with ctx.prepare(dg, kb.Options(reorder=2)) as pg:
            res = ctx.refine(pg, 5, kb.Options(reorder=2))
            assert np.array_equal(res.levels.cpu().numpy(), L) and np.array_equal(res.counts, C)
