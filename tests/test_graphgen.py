"""The seeded input generators (graphgen) draw the same graph on every side.

Full-size parity compares the GPU path on a graph drawn on the device with the
oracle's output on the same graph drawn on the host, so the numpy and torch
versions of the power-law generator must agree bit for bit, and the weights
they invert must not depend on the platform's libm.
"""
import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("factor,seed", [(0.002, 1), (0.01, 9)])
def test_numpy_and_torch_draw_the_same_graph(factor, seed):
    c = graphgen.scaled(graphgen.CONFIG_RDF, factor, seed=seed)
    c.pop("kind")
    g = graphgen.chung_lu(**c)
    d = graphgen.chung_lu_torch(device="cpu", **c)
    for name, a in (("row_offsets", g.row_offsets), ("col", g.col), ("elabel", g.elabel), ("vlabel", g.vlabel)):
        assert np.array_equal(a, d[name].numpy()), name
    assert g.row_offsets[-1] == g.m and np.all(np.diff(g.row_offsets) >= 0)
    assert g.col.min() >= 0 and g.col.max() < g.n


def test_counter_streams_agree():
    key = graphgen.stream_key(12345, 3)
    a = graphgen.ctr_bits(key, 1000, 5000).view(np.int64)
    b = graphgen.ctr_bits_torch(key, 1000, 5000, "cpu").numpy()
    assert np.array_equal(a, b)
    u = graphgen.ctr_uniform(key, 0, 1 << 16)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(u, graphgen.ctr_uniform_torch(key, 0, 1 << 16, "cpu").numpy())


def test_det_pow_close_to_pow():
    x = np.concatenate([np.arange(1, 100001, dtype=np.float64), np.array([2.0 ** 30, 3e8, 1.5, 0.75])])
    for a in (-1.0, -1.0 / 1.1, -1.5, -1.2, 0.5):
        rel = np.abs(graphgen.det_pow(x, a) / np.power(x, a) - 1.0)
        assert rel.max() < 1e-13, a
    assert graphgen.det_pow(np.array([1.0]), -0.9)[0] == 1.0


def test_power_law_shape():
    g = graphgen.make(graphgen.scaled(graphgen.CONFIG_RDF, 0.01))
    deg = np.diff(g.row_offsets)
    indeg = np.bincount(g.col, minlength=g.n)
    # heavy tails both ways, literal sinks, Zipf labels with label 0 the most frequent
    assert deg.max() > 50 * deg.mean() and indeg.max() > 50 * indeg.mean()
    assert 0.01 < (deg == 0).mean() < 0.5
    assert np.bincount(g.elabel).argmax() == 0 and np.bincount(g.vlabel).argmax() == 0
