"""The multi-core CPU baseline (cpu_parallel/) against the oracle: every level
and count, all directions and label switches, early stop on and off, and
graphs with hubs, self loops, parallel edges and edgeless vertices."""
import numpy as np
import pytest

import cpu_parallel
import graphgen
import oracle


def _graphs():
    rng = np.random.Generator(np.random.PCG64(31))
    gs = [graphgen.make(graphgen.CONFIG_TINY), graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.001, seed=2))]
    for _ in range(40):
        gs.append(graphgen.tiny_random(rng, n_max=40, m_max=120, n_labels=3))
    n = 500
    src = np.concatenate([np.full(300, 7), rng.integers(0, n, size=800), np.arange(50)])
    dst = np.concatenate([rng.integers(0, n, size=300), rng.integers(0, n, size=800), np.arange(50)])
    gs.append(graphgen.from_edges(n, src, dst, rng.integers(0, 2, size=src.shape[0]), rng.integers(0, 2, size=n)))
    gs.append(graphgen.from_edges(5, [], [], [], [0, 1, 0, 1, 2]))
    return gs


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("vl,el", [(True, True), (False, True), (True, False), (False, False)])
def test_cpu_parallel_equals_oracle(d, vl, el):
    for early in (True, False):
        for g in _graphs():
            L, C, lc = oracle.refine_graph(g, d, vl, el, k=6, early_stop=early)
            P, PC, plc = cpu_parallel.refine_graph(g, d, vl, el, k=6, early_stop=early)
            assert np.array_equal(P, L) and np.array_equal(PC, C) and plc == lc, (g.n, g.m, d, vl, el, early)


def test_cpu_parallel_empty_graph():
    P, C, lc = cpu_parallel.refine(0, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), k=3)
    assert P.shape == (4, 0) and list(C) == [0, 0, 0, 0] and lc == 0
