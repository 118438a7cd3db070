"""Serving (kb_server_*): requests that arrive while others run are admitted
as slots and memory free up, share every round's kernels, and each result is
exactly the solo oracle result of its graph and options."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2204_05821_gb300 as kb  # noqa: E402


def request_mix(seed, count):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        if i % 3 == 0:
            n = int(rng.integers(50, 4000))
            g = graphgen.chung_lu(n, 5 * n, 2.1, 2.1, n / 3, n / 3, 8, 1.5, 4, 1.2, int(rng.integers(0, 1 << 30)))
        elif i % 3 == 1:
            g = graphgen.erdos_renyi(int(rng.integers(1, 800)), int(rng.integers(0, 3000)), 4, 3,
                                     int(rng.integers(0, 1 << 30)))
        else:
            g = graphgen.tiny_random(rng, n_max=25, m_max=60, n_labels=3)
        opts = kb.Options(direction=int(rng.integers(0, 3)), use_vertex_labels=bool(rng.integers(0, 2)),
                          use_edge_labels=bool(rng.integers(0, 2)), early_stop=bool(rng.integers(0, 2)))
        out.append((g, int(rng.integers(0, 8)), opts))
    return out


def expected(g, k, o):
    return oracle.refine_graph(g, o.direction, o.use_vertex_labels, o.use_edge_labels, k=k, early_stop=o.early_stop)


def drain(server, tickets, results):
    for _ in range(10000):
        running, waiting = server.step()
        for t in list(tickets):
            state = server.poll(t)
            if state == kb.Server.DONE:
                results[t] = server.fetch(t)
                tickets.remove(t)
            elif state == kb.Server.FAILED:
                with pytest.raises(kb.KbError) as e:
                    server.fetch(t)
                results[t] = e.value.status
                tickets.remove(t)
        if not tickets and running == 0 and waiting == 0:
            return
    raise AssertionError("server did not drain")


def check(results, reqs_by_ticket):
    for t, (g, k, o) in reqs_by_ticket.items():
        L, C, lc = expected(g, k, o)
        levels, counts, glc = results[t]
        assert np.array_equal(levels, L), t
        assert np.array_equal(counts, C), t
        assert glc == lc, (t, glc, lc)


def test_serve_mix_equals_solo():
    reqs = request_mix(1, 40)
    with kb.Server(0, max_vertices=1 << 20, max_edges=1 << 22, max_requests=16) as sv:
        tickets, by_ticket, results = [], {}, {}
        # requests keep arriving while earlier ones are on the GPU
        for i, (g, k, o) in enumerate(reqs):
            t = sv.submit_graph(g, k, o)
            tickets.append(t)
            by_ticket[t] = (g, k, o)
            if i % 3 == 2:
                sv.step()
                for tt in list(tickets):
                    if sv.poll(tt) == kb.Server.DONE:
                        results[tt] = sv.fetch(tt)
                        tickets.remove(tt)
        drain(sv, tickets, results)
        st = sv.stats()
    check(results, by_ticket)
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0


def test_serve_small_arena_forces_waiting_and_compaction():
    reqs = request_mix(2, 30)
    big = max(g.n for g, _, _ in reqs)
    bige = max(2 * g.m for g, _, _ in reqs)
    with kb.Server(0, max_vertices=2 * big + 10, max_edges=2 * bige + 10, max_requests=4) as sv:
        tickets, by_ticket, results = [], {}, {}
        for g, k, o in reqs:
            t = sv.submit_graph(g, k, o)
            tickets.append(t)
            by_ticket[t] = (g, k, o)
        drain(sv, tickets, results)
        st = sv.stats()
    check(results, by_ticket)
    assert st["compactions"] > 0


def test_serve_weak_hash_and_hubs():
    reqs = request_mix(3, 20)
    with kb.Server(0, max_vertices=1 << 20, max_edges=1 << 22, max_requests=8, hub_threshold=3,
                   hash_mode=1) as sv:
        tickets, by_ticket, results = [], {}, {}
        for g, k, o in reqs:
            t = sv.submit_graph(g, k, o)
            tickets.append(t)
            by_ticket[t] = (g, k, o)
        drain(sv, tickets, results)
    check(results, by_ticket)


def test_serve_rejects_bad_requests():
    with kb.Server(0, max_vertices=100, max_edges=100, max_requests=2) as sv:
        g = graphgen.erdos_renyi(200, 50, 2, 2, 1)
        with pytest.raises(kb.KbError):
            sv.submit_graph(g, 3)
        g1 = graphgen.erdos_renyi(20, 30, 2, 2, 1)
        g1.row_offsets = g1.row_offsets.copy()
        g1.row_offsets[-1] += 1  # the offsets must end at m: checked at submission
        with pytest.raises(kb.KbError):
            sv.submit_graph(g1, 3)
        # a neighbour id out of range is found on the device at admission: that
        # request fails alone, the one queued behind it completes
        g2 = graphgen.erdos_renyi(20, 30, 2, 2, 1)
        g2.col = g2.col.copy()
        g2.col[3] = 99
        bad = sv.submit_graph(g2, 3)
        g3 = graphgen.erdos_renyi(20, 30, 2, 2, 1)
        t = sv.submit_graph(g3, 2)
        results = {}
        drain(sv, [bad, t], results)
        assert results[bad] == 1  # KB_ERR_INVALID_ARG
        L, C, lc = expected(g3, 2, kb.Options())
        assert np.array_equal(results[t][0], L)
        st = sv.stats()
        assert st["failed"] == 1 and st["completed"] == 1
