"""The allocation-free round entry point (kb_refine_round_noalloc).

Some callers cannot let a library allocate device memory: an application
that owns all device memory through its own pool, or a latency-critical
thread that must not trigger cudaMalloc's device-wide synchronisation.  For
them the library offers one round of the refinement whose scratch lives in a
fixed static device array.  This file checks, through the C ABI, that two
calls in a row give exactly the levels of the ordinary kb_refine entry point
and of the CPU oracle, so the state a call leaves in the shared array cannot
leak into the next, and that the rejections the header promises happen
without touching the output.  It is named to be collected last.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402


def test_noalloc_round_matches_refine_and_oracle_two_calls_in_a_row():
    g = graphgen.make(graphgen.CONFIG_TINY)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    with kb.Context(0) as ctx:
        res = ctx.refine(dg, 3, kb.Options(early_stop=False))
    torch.cuda.synchronize()
    ref = res.levels
    L, C, _ = oracle.refine_graph(g, oracle.DIR_OUT, True, True, k=3, early_stop=False)
    for i in (1, 2, 3):
        out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda:0")
        count = kb.refine_round_noalloc(dg, ref[i - 1].contiguous(), out, kb.Options())
        torch.cuda.synchronize()
        assert torch.equal(out, ref[i]), "level %d differs from kb_refine" % i
        assert np.array_equal(out.cpu().numpy(), L[i]), "level %d differs from the oracle" % i
        assert count == int(res.counts[i]) == int(C[i])


def test_noalloc_round_with_medium_vertices_and_weak_hash():
    rng = np.random.Generator(np.random.PCG64(4))
    n = 20_000
    deg = rng.integers(0, 40, size=n)
    deg[::97] = rng.integers(33, 1000, size=deg[::97].shape[0])
    src = np.repeat(np.arange(n), deg)
    dst = rng.integers(0, 300, size=src.shape[0])
    g = graphgen.from_edges(n, src, dst, rng.integers(0, 3, size=src.shape[0]), rng.integers(0, 4, size=n))
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    with kb.Context(0) as ctx:
        res = ctx.refine(dg, 2, kb.Options(early_stop=False))
    ref = res.levels
    L, _, _ = oracle.refine_graph(g, oracle.DIR_OUT, True, True, k=2, early_stop=False)
    for mode in (1, 0):
        out = torch.empty(n, dtype=torch.int32, device="cuda:0")
        count = kb.refine_round_noalloc(dg, ref[1].contiguous(), out, kb.Options(hash_mode=mode,
                                                                                  small_task_vertices=64))
        assert torch.equal(out, ref[2]) and count == int(res.counts[2])
        assert np.array_equal(out.cpu().numpy(), L[2])


def _rejected(dg, prev, options):
    out = torch.full((dg.n,), -7, dtype=torch.int32, device="cuda:0")
    with pytest.raises(kb.KbError) as e:
        kb.refine_round_noalloc(dg, prev, out, options)
    assert e.value.status == 1
    assert bool(torch.all(out == -7)), "a rejected call must leave out untouched"


def test_noalloc_rejects_sizes_beyond_the_limit():
    n = kb._capi.NOALLOC_MAX_VERTICES + 1
    row = torch.zeros(n + 1, dtype=torch.int64, device="cuda:0")
    col = torch.zeros(0, dtype=torch.int32, device="cuda:0")
    dg = kb.DeviceGraph(row, col)
    _rejected(dg, torch.zeros(n, dtype=torch.int32, device="cuda:0"), kb.Options())


def test_noalloc_rejects_a_vertex_above_the_hub_threshold_and_bad_prev():
    # vertex 3 has 40 edges: fine at the default threshold, a hub at 32
    n = 100
    src = np.concatenate([np.arange(n), np.full(40, 3)])
    dst = np.concatenate([(np.arange(n) + 1) % n, np.arange(40)])
    g = graphgen.from_edges(n, src, dst)
    dg = kb.DeviceGraph.from_numpy(g, "cuda:0")
    prev = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    out = torch.empty(n, dtype=torch.int32, device="cuda:0")
    assert kb.refine_round_noalloc(dg, prev, out, kb.Options()) >= 1
    _rejected(dg, prev, kb.Options(hub_threshold=32))
    bad = prev.clone()
    bad[17] = n  # a previous id outside [0, n)
    _rejected(dg, bad, kb.Options())
    bad[17] = -1
    _rejected(dg, bad, kb.Options())
    _rejected(dg, prev, kb.Options(small_task_vertices=16))
