"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
* the four partition tables the paper prints for its worked example;
* brute-force k-bisimilarity iterated pair by pair from the definitions;
* closed forms (paths, cycles, trees, edgeless graphs, symmetric graphs);
* invariants the paper states (refinement, counts never drop, stop on a
  stable count) and invariance under vertex renumbering.
A last group plants plausible mistakes in a throw-away Python copy of the
signature step and shows that the brute-force pin catches every one.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from oracle import bruteforce
from paper_fixture import canonical_ids, load, load_summary, partition


# ---------------------------------------------------------------- paper tables


@pytest.mark.parametrize("table", ["fw", "bw", "sch", "kau"])
def test_paper_tables_oracle(table):
    g, tables = load()
    t = tables[table]
    L, C, _ = oracle.refine_graph(g, t["direction"], t["use_vertex_labels"], t["use_edge_labels"], k=2,
                                  early_stop=False)
    for i, expected in t["levels"].items():
        assert partition(L[i]) == expected, (table, i)
        assert C[i] == len(expected)


@pytest.mark.parametrize("table", ["fw", "bw", "sch", "kau"])
def test_paper_tables_bruteforce(table):
    g, tables = load()
    t = tables[table]
    src, dst, lab = g.edges()
    ids, Rs = bruteforce.levels(g.n, src, dst, lab, g.vlabel, t["direction"], t["use_vertex_labels"],
                                t["use_edge_labels"], 2)
    for i, expected in t["levels"].items():
        assert bruteforce.is_equivalence(Rs[i])
        assert partition(ids[i]) == expected, (table, i)


def test_generator_matches_fixture():
    g, _ = load()
    h = graphgen.paper_example()
    assert h.n == g.n and h.m == g.m
    assert np.array_equal(h.row_offsets, g.row_offsets)
    assert np.array_equal(h.col, g.col)
    # label ids differ in naming only; the induced partitions must agree
    assert partition(h.vlabel) == partition(g.vlabel)
    assert partition(h.elabel) == partition(g.elabel)


def test_schaetzle_example_stable_at_level_one():
    # Section 3.3: full bisimulation of the example is reached at k = 1
    g, tables = load()
    t = tables["sch"]
    L, C, lc = oracle.refine_graph(g, t["direction"], False, True, k=10, early_stop=True)
    assert lc == 2 and C.tolist() == [1, 3] + [3] * 9
    assert all(np.array_equal(L[i], L[1]) for i in range(1, 11))


# ---------------------------------------------------------------- brute force


def _random_cases(count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(count):
        g = graphgen.tiny_random(rng, n_max=10, m_max=24, n_labels=int(rng.integers(1, 4)))
        d = int(rng.integers(0, 3))
        vl = bool(rng.integers(0, 2))
        el = bool(rng.integers(0, 2))
        k = int(rng.integers(0, 6))
        yield g, d, vl, el, k


def test_oracle_matches_bruteforce_random_tiny():
    for g, d, vl, el, k in _random_cases(400, 11):
        L, C, _ = oracle.refine_graph(g, d, vl, el, k=k, early_stop=False)
        src, dst, lab = g.edges()
        ids, Rs = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, k)
        for i in range(k + 1):
            assert L[i].tolist() == ids[i], (d, vl, el, i)
            assert C[i] == max(ids[i]) + 1


@pytest.mark.slow
def test_oracle_matches_bruteforce_many():
    for g, d, vl, el, k in _random_cases(4000, 12):
        L, _, _ = oracle.refine_graph(g, d, vl, el, k=k, early_stop=False)
        src, dst, lab = g.edges()
        ids, _ = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, k)
        assert [r.tolist() for r in L] == ids


def _stable(g, d, el, ids):
    # Paige-Tarjan stability (Def. "relational coarsest partition problem"):
    # no block holds both a vertex with an edge of some label into some block S
    # and a vertex without one (per processed direction).
    src, dst, lab = g.edges()
    lab = lab if el else np.zeros_like(lab)
    members = {}
    for v, b in enumerate(ids):
        members.setdefault(b, []).append(v)
    for direction in {0: [0], 1: [1], 2: [0, 1]}[d]:
        a, b = (src, dst) if direction == 0 else (dst, src)
        has = set((int(a[i]), int(lab[i]), ids[int(b[i])]) for i in range(len(a)))
        for (v, l, s) in has:
            if any((u, l, s) not in has for u in members[ids[v]]):
                return False
    return True


def test_fixpoint_is_coarsest_stable_refinement():
    # full bisimulation (Sec. "Bisimulation Variants": iterate until no change):
    # the oracle's stable level equals the brute-force relation iterated to
    # its fixpoint, and it is stable in the Paige-Tarjan sense
    for g, d, vl, el, _ in _random_cases(150, 14):
        L, C, lc = oracle.refine_graph(g, d, vl, el, k=g.n + 1, early_stop=True)
        src, dst, lab = g.edges()
        ids, _ = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, g.n + 1)
        assert ids[-1] == ids[-2]  # the relation reached its fixpoint
        assert L[lc].tolist() == ids[-1]
        assert lc <= g.n
        assert _stable(g, d, el, ids[-1])
        if lc >= 2:
            # the level two before the stop was still split by the next round
            assert not _stable(g, d, el, L[lc - 2].tolist())


def test_stability_check_catches_unstable_partition():
    # the path 0 -> 1 -> 2: {0, 1, 2} is unstable (2 has no out-edge)
    g = graphgen.path_graph(3)
    assert not _stable(g, 0, False, [0, 0, 0])
    assert _stable(g, 0, False, [0, 1, 2])


def test_bruteforce_relation_is_equivalence():
    for g, d, vl, el, k in itertools.islice(_random_cases(60, 13), 60):
        src, dst, lab = g.edges()
        _, Rs = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, k)
        assert all(bruteforce.is_equivalence(R) for R in Rs)


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("n", [1, 2, 5, 13])
def test_path_counts(n):
    # directed path, out-edges: vertex v is distinguished by its distance to the
    # sink, capped at i, so level i has min(i+1, n) blocks
    g = graphgen.path_graph(n)
    L, C, _ = oracle.refine_graph(g, 0, False, False, k=15, early_stop=False)
    assert C.tolist() == [min(i + 1, n) for i in range(16)]
    # in-edges: distance from the source instead
    L2, C2, _ = oracle.refine_graph(g, 1, False, False, k=15, early_stop=False)
    assert C2.tolist() == [min(i + 1, n) for i in range(16)]


@pytest.mark.parametrize("n", [1, 3, 8])
def test_cycle_single_block(n):
    g = graphgen.cycle_graph(n)
    for d in (0, 1, 2):
        _, C, _ = oracle.refine_graph(g, d, False, False, k=6, early_stop=False)
        assert C.tolist() == [1] * 7


def test_edgeless_graph_keeps_level0():
    g = graphgen.from_edges(7, [], [], [], [3, 1, 3, 2, 1, 1, 9])
    for d in (0, 1, 2):
        L, C, lc = oracle.refine_graph(g, d, True, True, k=5, early_stop=False)
        assert C.tolist() == [4] * 6
        assert all(np.array_equal(L[i], L[0]) for i in range(6))
        assert L[0].tolist() == [0, 1, 0, 2, 1, 1, 3]


@pytest.mark.parametrize("h", [0, 1, 3, 5])
def test_binary_tree_counts(h):
    # out-edges: blocks are heights (distance to the leaves) capped at i
    g = graphgen.binary_tree(h)
    _, C, _ = oracle.refine_graph(g, 0, False, False, k=8, early_stop=False)
    assert C.tolist() == [min(i + 1, h + 1) for i in range(9)]
    # in-edges: blocks are depths capped at i
    _, C2, _ = oracle.refine_graph(g, 1, False, False, k=8, early_stop=False)
    assert C2.tolist() == [min(i + 1, h + 1) for i in range(9)]


def test_symmetric_graph_directions_agree():
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(30):
        n = int(rng.integers(1, 30))
        m = int(rng.integers(0, 60))
        s = rng.integers(0, n, size=m)
        t = rng.integers(0, n, size=m)
        lab = rng.integers(0, 3, size=m)
        g = graphgen.from_edges(n, np.concatenate([s, t]), np.concatenate([t, s]), np.concatenate([lab, lab]),
                                rng.integers(0, 2, size=n))
        outs = [oracle.refine_graph(g, d, True, True, k=6, early_stop=False)[0] for d in (0, 1, 2)]
        assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


# ---------------------------------------------------------------- invariants


def _tiny_config_graph():
    return graphgen.make(graphgen.CONFIG_TINY)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_invariants_er(d):
    g = _tiny_config_graph()
    L, C, lc = oracle.refine_graph(g, d, True, True, k=10, early_stop=False)
    for i in range(11):
        ids = L[i]
        # canonical: first occurrences of ids appear in order 0,1,2,...
        _, first = np.unique(ids, return_index=True)
        assert np.array_equal(np.sort(first), first)
        assert ids.min() == 0 and ids.max() == C[i] - 1 and C[i] <= g.n
        if i > 0:
            assert C[i] >= C[i - 1]
            # level i refines level i-1: each new block maps to one old block
            pairs = np.unique(np.stack([ids, L[i - 1]], 1), axis=0)
            assert pairs.shape[0] == C[i]


def _degree(g, d):
    out = np.diff(g.row_offsets)
    inn = np.bincount(g.col, minlength=g.n)
    return {0: out, 1: inn, 2: out + inn}[d]


@pytest.mark.parametrize("d", [0, 1, 2])
def test_frozen_blocks_never_change(d):
    # What the GPU rounds skip: with the own previous block in every key (Sec. 3:
    # i-bisimilar requires (i-1)-bisimilar), a vertex alone in its block stays
    # alone, and a block formed by a round (level >= 1) that holds a vertex
    # without edges holds only such vertices and is kept whole at every later
    # level.
    rng = np.random.Generator(np.random.PCG64(70 + d))
    graphs = [graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.0005, seed=23))]
    graphs += [graphgen.tiny_random(rng, n_max=60, m_max=90, n_labels=3) for _ in range(40)]
    checked = 0
    for g in graphs:
        L, _, _ = oracle.refine_graph(g, d, True, True, k=6, early_stop=False)
        edgeless = _degree(g, d) == 0
        for i in range(1, 7):
            prev, cur = L[i - 1], L[i]
            alone = np.bincount(prev)[prev] == 1
            assert np.all(np.bincount(cur)[cur][alone] == 1)
            if i >= 2:
                # blocks of level i-1 holding an edgeless vertex hold only edgeless ones
                mixed = np.zeros(prev.max() + 1, dtype=bool)
                mixed[prev[~edgeless]] = True
                assert not np.any(mixed[prev[edgeless]])
                # and are kept whole: same partition of the edgeless vertices
                pairs = np.unique(np.stack([prev[edgeless], cur[edgeless]], 1), axis=0)
                assert pairs.shape[0] == np.unique(prev[edgeless]).size == np.unique(cur[edgeless]).size
                checked += int(edgeless.sum())
    assert checked > 0


def _smallest_member(level):
    first = np.full(level.max() + 1, level.shape[0], dtype=np.int64)
    np.minimum.at(first, level, np.arange(level.shape[0]))
    return first[level]


def _clean_blocks_keep_members(g, d, L, k):
    """For levels i = 1..k-1: a level-i block none of whose members has an edge
    (in direction d) to a vertex whose smallest block member changed between
    levels i-1 and i must be one block of level i+1.  Returns how many such
    blocks were checked."""
    src, dst, _ = g.edges()
    pairs = []
    if d in (0, 2):
        pairs.append((src, dst))
    if d in (1, 2):
        pairs.append((dst, src))
    checked = 0
    for i in range(1, k):
        prev, cur, nxt = L[i - 1], L[i], L[i + 1]
        moved = _smallest_member(cur) != _smallest_member(prev)
        dirty = np.zeros(g.n, dtype=bool)
        for a, b in pairs:
            dirty[a[moved[b]]] = True
        dirty_block = np.zeros(cur.max() + 1, dtype=bool)
        dirty_block[cur[dirty]] = True
        for blk in np.unique(cur[~dirty_block[cur]]):
            members = np.nonzero(cur == blk)[0]
            assert np.unique(nxt[members]).size == 1, (d, i, blk)
            checked += members.size > 1
    return checked


@pytest.mark.parametrize("d", [0, 1, 2])
def test_clean_blocks_never_split(d):
    # What the GPU rounds also skip.  For a level-i block to split at level
    # i+1, two members with equal signatures over level i-1 must differ over
    # level i, which takes a level-(i-1) block B split into parts C, C' with
    # one member's edge into C and the other's into C' only; one of the parts
    # lacks B's smallest member, so its vertices changed smallest member.
    # Hence a block none of whose members has an edge to such a vertex stays
    # whole.  Checked on the oracle's levels of paths, trees, combs, power-law
    # and random graphs.
    rng = np.random.Generator(np.random.PCG64(90 + d))
    graphs = [graphgen.path_graph(40), graphgen.binary_tree(6),
              graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.0005, seed=29))]
    n = 60
    spine = np.arange(n - 1)
    leaves = np.arange(n, 3 * n)
    graphs.append(graphgen.from_edges(3 * n, np.concatenate([spine, (leaves - n) // 2]),
                                      np.concatenate([spine + 1, leaves]), None, None))
    graphs += [graphgen.tiny_random(rng, n_max=50, m_max=70, n_labels=2) for _ in range(40)]
    checked = 0
    for g in graphs:
        for vl in (True, False):
            L, _, _ = oracle.refine_graph(g, d, vl, True, k=8, early_stop=False)
            checked += _clean_blocks_keep_members(g, d, L, 8)
    assert checked > 100


def test_early_stop_matches_full_run():
    for d in (0, 1, 2):
        g = graphgen.erdos_renyi(300, 400, 2, 2, seed=d)
        A, CA, la = oracle.refine_graph(g, d, True, True, k=30, early_stop=True)
        B, CB, lb = oracle.refine_graph(g, d, True, True, k=30, early_stop=False)
        assert np.array_equal(A, B) and np.array_equal(CA, CB)
        assert lb == 30 and la <= 30
        if la < 30:
            assert CA[la] == CA[la - 1]


def test_vertex_renumbering_invariance():
    g = graphgen.erdos_renyi(500, 2000, 3, 3, seed=9)
    rng = np.random.Generator(np.random.PCG64(2))
    perm = rng.permutation(g.n)  # new id of old vertex v is perm[v]
    src, dst, lab = g.edges()
    vl = np.empty_like(g.vlabel)
    vl[perm] = g.vlabel
    h = graphgen.from_edges(g.n, perm[src], perm[dst], lab, vl)
    for d in (0, 1, 2):
        A, CA, _ = oracle.refine_graph(g, d, True, True, k=6, early_stop=False)
        B, CB, _ = oracle.refine_graph(h, d, True, True, k=6, early_stop=False)
        assert np.array_equal(CA, CB)
        for i in range(7):
            # old vertex v is new vertex perm[v]
            assert partition(A[i]) == partition(B[i][perm])


def test_label_renaming_invariance():
    # labels enter only through equality (Defs. "edge-labeled-fw-bisimulation",
    # "vertex-labeled-bw-bisimulation") and ids are ranks of smallest members,
    # so injective renamings of vertex and edge labels, into large and negative
    # values too, leave every level identical, not just the same partitions
    g = graphgen.erdos_renyi(600, 2400, 6, 4, seed=12)
    rng = np.random.Generator(np.random.PCG64(5))
    vmap = rng.choice(np.array([-2147483648, -7, 0, 8191, 8192, 2147483647], dtype=np.int64), 6, replace=False)
    emap = rng.choice(np.array([-2147483648, -1, 9000, 2147483647], dtype=np.int64), 4, replace=False)
    src, dst, lab = g.edges()
    h = graphgen.from_edges(g.n, src, dst, emap[lab].astype(np.int32), vmap[g.vlabel].astype(np.int32))
    for d in (0, 1, 2):
        A, CA, _ = oracle.refine_graph(g, d, True, True, k=6, early_stop=False)
        B, CB, _ = oracle.refine_graph(h, d, True, True, k=6, early_stop=False)
        assert np.array_equal(A, B) and np.array_equal(CA, CB)
    # a non-injective renaming merges classes: level 0 gets coarser
    merged = graphgen.from_edges(g.n, src, dst, lab, (g.vlabel // 2).astype(np.int32))
    L, C, _ = oracle.refine_graph(merged, 0, True, True, k=1, early_stop=False)
    assert C[0] < len(np.unique(g.vlabel))


def test_initial_partition_equals_label_partition():
    g = graphgen.erdos_renyi(400, 1500, 5, 3, seed=4)
    A, CA, _ = oracle.refine_graph(g, 0, True, True, k=6, early_stop=False)
    B, CB, _ = oracle.refine_graph(g, 0, False, True, k=6, early_stop=False, initial=g.vlabel * 7 - 3)
    assert np.array_equal(A, B) and np.array_equal(CA, CB)


def test_own_block_reading_is_harmless_without_labels():
    # Schaetzle's signature omits the vertex's own block; with P_0 = {V} keeping
    # it changes nothing (P_i refines P_{i-1}).  Compare with a signature-only
    # refinement written here.
    g = graphgen.erdos_renyi(300, 700, 1, 3, seed=8)
    L, _, _ = oracle.refine_graph(g, 0, False, True, k=6, early_stop=False)
    prev = np.zeros(g.n, dtype=np.int64)
    for i in range(1, 7):
        sigs = [oracle.signature(g.row_offsets, g.col, g.elabel, prev, v) for v in range(g.n)]
        ids, cur = {}, np.empty(g.n, dtype=np.int64)
        for v in range(g.n):
            cur[v] = ids.setdefault(sigs[v], len(ids))
        assert np.array_equal(cur, L[i])
        prev = cur


def _in_lists(g):
    src, dst, lab = g.edges()
    lists = {}
    for s, d, l in zip(src.tolist(), dst.tolist(), lab.tolist()):
        lists.setdefault(d, []).append((s, l))
    return lists


@pytest.mark.parametrize("d", [0, 1, 2])
def test_signature_keys_give_the_bruteforce_partition(d):
    # oracle.signature (all three directions, the in-edge branch included):
    # grouping vertices by (own block at level i-1, signature over level i-1)
    # must give the brute-force relation R_i of the definitions.
    rng = np.random.Generator(np.random.PCG64(31 + d))
    for _ in range(60):
        g = graphgen.tiny_random(rng)
        el = bool(rng.integers(0, 2))
        src, dst, lab = g.edges()
        ids, _ = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, True, el, 4)
        inl = _in_lists(g)
        for i in range(1, 5):
            prev = np.array(ids[i - 1])
            keys = [(int(prev[v]), oracle.signature(g.row_offsets, g.col, g.elabel, prev, v, d, el, inl))
                    for v in range(g.n)]
            got = {}
            assert [got.setdefault(key, len(got)) for key in keys] == ids[i], (d, el, i)


def test_in_signature_is_the_reversed_out_signature():
    # the in-direction signature of v in G is the out-direction signature of v
    # in the reversed graph, with the direction bit set; BOTH is their union.
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(40):
        g = graphgen.tiny_random(rng, n_max=15, m_max=40)
        src, dst, lab = g.edges()
        r = graphgen.from_edges(g.n, dst, src, lab, g.vlabel)
        prev = rng.integers(0, 3, size=g.n)
        inl = _in_lists(g)
        for v in range(g.n):
            sin = oracle.signature(g.row_offsets, g.col, g.elabel, prev, v, oracle.DIR_IN, True, inl)
            sout_r = oracle.signature(r.row_offsets, r.col, r.elabel, prev, v, oracle.DIR_OUT, True)
            assert sin == tuple(sorted((1, l, b) for (_, l, b) in sout_r))
            sout = oracle.signature(g.row_offsets, g.col, g.elabel, prev, v, oracle.DIR_OUT, True)
            sboth = oracle.signature(g.row_offsets, g.col, g.elabel, prev, v, oracle.DIR_BOTH, True, inl)
            assert sboth == tuple(sorted(set(sin) | set(sout)))


# ---------------------------------------------------------------- the pins catch planted mistakes


def _mutant_refine(g, d, vl, el, k, mistake):
    """A deliberately simple signature refinement with one planted mistake."""
    n = g.n
    src, dst, lab = g.edges()
    if mistake == "transposed":
        src, dst = dst, src
    labels = g.vlabel if vl else np.zeros(n, dtype=np.int64)
    ids0 = {}
    prev = np.array([ids0.setdefault(int(x), len(ids0)) for x in labels])
    out = [prev]
    for _ in range(k):
        sig = [[] for _ in range(n)]
        for s, t, l in zip(src, dst, lab):
            ll = int(l) if (el and mistake != "drop_label") else 0
            if d in (0, 2):
                sig[s].append((0, ll, int(prev[t])))
            if d in (1, 2):
                sig[t].append((1, ll, int(prev[s])))
        keys = []
        for v in range(n):
            body = tuple(sorted(sig[v])) if mistake == "multiset" else tuple(sorted(set(sig[v])))
            own = 0 if mistake == "drop_own_block" else int(prev[v])
            keys.append((own, body))
        ids = {}
        prev = np.array([ids.setdefault(kk, len(ids)) for kk in keys])
        out.append(prev)
    return out


@pytest.mark.parametrize("mistake", ["drop_own_block", "multiset", "drop_label", "transposed"])
def test_bruteforce_catches_planted_mistakes(mistake):
    caught = False
    for g, d, vl, el, k in _random_cases(300, 21):
        if mistake == "drop_own_block":
            vl = True
        if mistake == "drop_label":
            el = True
        if mistake == "transposed":
            d = 0
        k = max(k, 2)
        src, dst, lab = g.edges()
        ids, _ = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, k)
        got = _mutant_refine(g, d, vl, el, k, mistake)
        if any(list(got[i]) != ids[i] for i in range(k + 1)):
            caught = True
            break
    assert caught, mistake


def test_unmutated_copy_agrees():
    for g, d, vl, el, k in _random_cases(100, 22):
        src, dst, lab = g.edges()
        ids, _ = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, k)
        got = _mutant_refine(g, d, vl, el, k, None)
        assert [list(x) for x in got] == ids


# ---------------------------------------------------------------- summary graph


def test_summary_paper_example():
    # hand-derived summary graphs of the running example (Section 3.4)
    g, tables = load()
    for table, i_src, i_dst, expected in load_summary():
        t = tables[table]
        a = canonical_ids(t["levels"][i_src], g.n)
        b = canonical_ids(t["levels"][i_dst], g.n)
        s, lab, d = oracle.summary(g, t["direction"], t["use_edge_labels"], a, b)
        assert list(zip(s.tolist(), lab.tolist(), d.tolist())) == expected, table


def _first_occurrence(triples):
    # numpy: distinct rows, ordered by the index of their first occurrence
    if len(triples) == 0:
        return np.zeros((0, 3), dtype=np.int64)
    u, first = np.unique(triples, axis=0, return_index=True)
    return u[np.argsort(first, kind="stable")]


def test_summary_identity_and_trivial_partitions():
    for g, d, _, el, _ in itertools.islice(_random_cases(200, 15), 200):
        if d == 2:
            continue
        src, dst, lab = g.edges()
        lab = lab if el else np.zeros_like(lab)
        ident = np.arange(g.n, dtype=np.int32)
        x, y = (src, dst) if d == 0 else (dst, src)
        expect = _first_occurrence(np.stack([x, lab, y], axis=1))
        s, l, t = oracle.summary(g, d, el, ident, ident)
        assert np.array_equal(np.stack([s, l, t], axis=1), expect)
        zero = np.zeros(g.n, dtype=np.int32)
        s, l, t = oracle.summary(g, d, el, zero, zero)
        labs = _first_occurrence(lab.reshape(-1, 1)).reshape(-1)
        assert s.tolist() == [0] * len(labs) and t.tolist() == [0] * len(labs) and l.tolist() == labs.tolist()


def test_summary_edges_hold_for_every_represented_vertex():
    # the paper's description: a summary edge (b, l, c) means every vertex of b
    # has an l-edge into c.  For the layering P_i -> P_{i-1} of a bisimulation
    # refinement that holds, because the vertices of a block of P_i share
    # their signature over P_{i-1}.
    for g, d, vl, el, k in itertools.islice(_random_cases(300, 16), 300):
        if d == 2 or k == 0:
            continue
        L, _, _ = oracle.refine_graph(g, d, vl, el, k=k, early_stop=False)
        src, dst, lab = g.edges()
        lab = lab if el else np.zeros_like(lab)
        x, y = (src, dst) if d == 0 else (dst, src)
        for i in range(1, k + 1):
            s, l, t = oracle.summary(g, d, el, L[i], L[i - 1])
            have = set(zip(x.tolist(), lab.tolist(), L[i - 1][y].tolist()))
            for b, ll, c in zip(s.tolist(), l.tolist(), t.tolist()):
                for v in np.nonzero(L[i] == b)[0].tolist():
                    assert (v, ll, c) in have
            assert len(s) <= g.m


def test_summary_in_direction_reverses_out():
    for g, _, vl, el, k in itertools.islice(_random_cases(100, 17), 100):
        L, _, _ = oracle.refine_graph(g, 0, vl, el, k=k, early_stop=False)
        P = L[k]
        so, lo, do = oracle.summary(g, 0, el, P, P)
        si, li, di = oracle.summary(g, 1, el, P, P)
        assert set(zip(di.tolist(), li.tolist(), si.tolist())) == set(zip(so.tolist(), lo.tolist(), do.tolist()))


def test_summary_follows_block_renaming():
    rng = np.random.Generator(np.random.PCG64(18))
    for g, d, vl, el, k in itertools.islice(_random_cases(60, 19), 60):
        if d == 2:
            continue
        L, _, _ = oracle.refine_graph(g, d, vl, el, k=k, early_stop=False)
        P = L[k]
        perm = rng.permutation(g.n).astype(np.int32) - 5  # any int32 ids, negatives included
        s, l, t = oracle.summary(g, d, el, P, P)
        s2, l2, t2 = oracle.summary(g, d, el, perm[P], perm[P])
        assert np.array_equal(s2, perm[s]) and np.array_equal(l2, l) and np.array_equal(t2, perm[t])


# ---------------------------------------------------------------- generic CSE rounds


def test_cse_matches_bruteforce():
    # Def. "cse": v ~s v', and the (label ~p, object CSE^{i-1}) sets match both ways
    for g, d, vl, el, k in itertools.islice(_random_cases(300, 20), 300):
        src, dst, lab = g.edges()
        for subject in (1, 2, 3):
            L, C, _ = oracle.refine_graph(g, d, vl, el, k=k, early_stop=False, subject=subject)
            ids, _ = bruteforce.levels(g.n, src, dst, lab, g.vlabel, d, vl, el, k, subject)
            assert [r.tolist() for r in L] == ids, (subject, d, vl, el)
            assert C.tolist() == [max(r) + 1 for r in ids]


def test_cse_presets_are_the_paper_models():
    # Eq. (gsm:schaetzle): (T, id, T)^k forward; Eq. (gsm:kaushik): ((OC, T, OC)^-1)^k
    g, tables = load()
    L, _, _ = oracle.refine_graph(g, 0, False, True, k=2, early_stop=False, subject=1)
    for i, expected in tables["sch"]["levels"].items():
        assert partition(L[i]) == expected
    L, _, _ = oracle.refine_graph(g, 1, True, False, k=2, early_stop=False, subject=2)
    for i, expected in tables["kau"]["levels"].items():
        assert partition(L[i]) == expected


def test_cse_levels_need_not_refine():
    # (T, id, OC): subjects are not compared, objects by label at depth 1.  Two
    # differently labelled vertices with an edge to the same vertex share a
    # level-1 block, so level 1 has fewer blocks than level 0.
    g = graphgen.from_edges(3, [0, 1], [2, 2], [0, 0], [7, 8, 9])
    L, C, _ = oracle.refine_graph(g, 0, True, True, k=2, early_stop=False, subject=1)
    assert C.tolist() == [3, 2, 2]
    assert L[1].tolist() == [0, 0, 1]


def test_cse_early_stop_equals_full_run():
    for g, d, vl, el, k in itertools.islice(_random_cases(200, 21), 200):
        for subject in (1, 2, 3):
            A, CA, lc = oracle.refine_graph(g, d, vl, el, k=k, early_stop=True, subject=subject)
            B, CB, _ = oracle.refine_graph(g, d, vl, el, k=k, early_stop=False, subject=subject)
            assert np.array_equal(A, B) and np.array_equal(CA, CB)
