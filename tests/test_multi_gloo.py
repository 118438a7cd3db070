"""Multi-rank path on CPU: two gloo ranks shard a batch of independent graphs
(no data-path collective), refine their shares with the CPU oracle standing
in for the device path, and gather results equal to a single-process run."""
import os
import socket

import numpy as np
import pytest

import graphgen
import oracle
from paper_2204_05821_gb300 import multi


def test_shard_graphs_balanced_and_complete():
    rng = np.random.Generator(np.random.PCG64(1))
    sizes = rng.integers(1, 10_000, size=301)
    for world in (1, 2, 3, 8):
        shards = multi.shard_graphs(sizes, world)
        flat = sorted(j for s in shards for j in s)
        assert flat == list(range(len(sizes)))
        loads = [int(sum(sizes[j] for j in s)) for s in shards]
        assert max(loads) - min(loads) <= int(sizes.max())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    graphs, ks = graphgen.batch_workload(G=24, median_m=400, sigma=0.8, m_lo=50, m_hi=3000, k_max=5, seed=9)
    shards = multi.shard_graphs([g.m for g in graphs], world)
    local = {}
    for j in shards[rank]:
        L, C, lc = oracle.refine_graph(graphs[j], 0, True, True, k=int(ks[j]))
        local[j] = (L.tolist(), C.tolist(), lc)
    merged = multi.gather_results(local)
    t = multi.max_over_ranks(float(rank + 1))
    if rank == 0:
        out_q.put((merged, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_a_batch():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.0
    graphs, ks = graphgen.batch_workload(G=24, median_m=400, sigma=0.8, m_lo=50, m_hi=3000, k_max=5, seed=9)
    assert sorted(merged) == list(range(24))
    for j, g in enumerate(graphs):
        L, C, lc = oracle.refine_graph(g, 0, True, True, k=int(ks[j]))
        assert merged[j][0] == L.tolist() and merged[j][1] == C.tolist() and merged[j][2] == lc
