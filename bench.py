"""Benchmark: stratified k-bisimulation edges/s per refinement round on GB300.

Default workload: the large single graph (Chung-Lu power law, exponent 2.0,
200M vertices, 2B edges, 5,000 vertex labels Zipf(1.5), 500 edge labels
Zipf(1.2), out-edges, k = 10).  One step = one kb_refine call (levels 0..10,
early stop on).  value = edges processed per round summed over the rounds of
all timed steps / timed seconds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|rdf|tiny] [--k 10]

With N > 1 (torchrun) every rank refines its own copy of the workload: the
single-graph path does not shard, so ranks are replicas.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402

WORKLOADS = {
    "large": graphgen.CONFIG_LARGE,
    # the same recipe at a tenth of the size: small enough for multi-pass profiling
    "large_tenth": graphgen.scaled(graphgen.CONFIG_LARGE, 0.1),
    "rdf": graphgen.CONFIG_RDF,
    "tiny": graphgen.CONFIG_TINY,
}
METRIC = "k-bisim edges/s per round"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# byte of a kernel, from one ncu capture of it on the large recipe at a tenth
# of the size, where its traffic grows in proportion to its units.  Valid only for the kernel source it was measured
# on: the SHA-1 of the kernel's file followed by the two shared device headers
# must match.
KERNEL_HEADERS = ("paper_2204_05821_gb300/csrc/kb_device.cuh", "paper_2204_05821_gb300/csrc/kb_internal.cuh")
TRAFFIC_PER_ALGO_BYTE = {
    "hub_chunk": ("paper_2204_05821_gb300/csrc/kb_kernels.cu", "9734ccc8cb4fa02be0fff878a6f1f298d83277e3", 2.206),
    "small": ("paper_2204_05821_gb300/csrc/kb_small.cu", "5fe82d2a0a4fa2dc30c2c8474321b9501eb6d7f1", 5.522),
    "medium": ("paper_2204_05821_gb300/csrc/kb_medium.cu", "98941f79c3ef798d184d25adb0e052b61de81aa0", 1.965),
}


def kernel_source_sha(path):
    """SHA-1 of a kernel's source file and the shared device headers, in that order."""
    import hashlib

    h = hashlib.sha1()
    for p in (path,) + KERNEL_HEADERS:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_for(kernel, algo_bytes):
    entry = TRAFFIC_PER_ALGO_BYTE.get(kernel)
    if not entry or entry[1] is None:
        return None
    path, sha, ratio = entry
    try:
        if kernel_source_sha(path) != sha:
            return None
    except OSError:
        return None
    return ratio * algo_bytes


UNIT = "edges/s"


def describe(name, cfg, k, direction):
    d = {"workload": name, "n": cfg["n"], "m": cfg["m"], "k": k, "direction": direction,
         "recipe": cfg["kind"], "seed": cfg["seed"]}
    if cfg["kind"] == "chung_lu":
        d.update(gamma_out=cfg["gamma_out"], gamma_in=cfg["gamma_in"], max_out_deg=cfg["max_out_deg"],
                 vertex_labels="zipf(%g)/%d" % (cfg["zipf_v"], cfg["n_vlabels"]),
                 edge_labels="zipf(%g)/%d" % (cfg["zipf_e"], cfg["n_elabels"]))
    else:
        d.update(vertex_labels="uniform/%d" % cfg["n_vlabels"], edge_labels="uniform/%d" % cfg["n_elabels"])
    return d


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload_gpu(cfg, device):
    import torch

    if cfg["kind"] == "chung_lu" and cfg["m"] >= 50_000_000:
        c = dict(cfg)
        c.pop("kind")
        d = graphgen.chung_lu_torch(device=device, **c)
        torch.cuda.synchronize()
        return d
    g = graphgen.make(cfg)
    return {"n": g.n, "m": g.m, "row_offsets": torch.from_numpy(g.row_offsets).to(device),
            "col": torch.from_numpy(g.col).to(device), "elabel": torch.from_numpy(g.elabel).to(device),
            "vlabel": torch.from_numpy(g.vlabel).to(device)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(cfg, target_s=12.0, max_reps=40):
    """The oracle, as it stands, single-threaded on a scaled-down graph of the
    same recipe: one refinement round (after level 0) per call, repeated until
    about target_s seconds of CPU work have run."""
    import oracle

    factor = 0.005 if cfg["m"] >= 1e9 else (0.05 if cfg["m"] >= 1e8 else 1.0)
    c = graphgen.scaled(cfg, factor) if factor != 1.0 else cfg
    g = graphgen.make(c)
    total, reps = 0.0, 0
    while reps < max_reps and (reps == 0 or total < target_s):
        t0 = time.perf_counter()
        oracle.refine_graph(g, 0, True, True, k=1, early_stop=False)
        total += time.perf_counter() - t0
        reps += 1
    out = {"value": g.m * reps / total, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
           "sample": "oracle (single-threaded C++ map refinement) on the same recipe scaled to n=%d, m=%d: "
                     "%d call(s) of one round after level 0, %.1f s in all" % (g.n, g.m, reps, total)}
    # the multi-core CPU baseline (OpenMP, every host core) on the same sample
    import cpu_parallel

    L, C, _ = oracle.refine_graph(g, 0, True, True, k=1, early_stop=False)
    P, PC, _ = cpu_parallel.refine_graph(g, 0, True, True, k=1, early_stop=False)
    ptotal, preps = 0.0, 0
    while preps < max_reps and (preps == 0 or ptotal < target_s / 3):
        t0 = time.perf_counter()
        cpu_parallel.refine_graph(g, 0, True, True, k=1, early_stop=False)
        ptotal += time.perf_counter() - t0
        preps += 1
    out["parallel"] = {"value": g.m * preps / ptotal, "unit": UNIT, "cores": cpu_parallel.threads(),
                       "kind": "OpenMP signatures + parallel sort (cpu_parallel/)",
                       "equal_to_oracle": bool(np.array_equal(P, L) and np.array_equal(PC, C)),
                       "sample": "the same graph: %d call(s) of one round after level 0, %.1f s in all"
                                 % (preps, ptotal)}
    return out


# ----------------------------------------------------------------------------- reference arm


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle

    cfg = WORKLOADS[args.workload]
    factor = 0.005 if cfg["m"] >= 1e9 else (0.05 if cfg["m"] >= 1e8 else 1.0)
    c = graphgen.scaled(cfg, factor) if factor != 1.0 else cfg
    g = graphgen.make(c)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.refine_graph(g, 0, True, True, k=1, early_stop=False)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = g.m * len(times) / total
    sample = ("each step: one oracle refinement round (plus level 0) on the %s recipe scaled to n=%d, m=%d, "
              "single-threaded" % (args.workload, g.n, g.m))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": describe(args.workload, cfg, args.k, "out"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm


def run_ours(args, rank, world, local):
    import torch

    import paper_2204_05821_gb300 as kb

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    device = "cuda:%d" % local
    cfg = WORKLOADS[args.workload]
    wl = make_workload_gpu(cfg, device)
    dg = kb.DeviceGraph(wl["row_offsets"], wl["col"], wl["elabel"], wl["vlabel"])
    n, m = dg.n, dg.m
    k = args.k
    opts = kb.Options(direction=kb.DIR_OUT, hub_threshold=args.hub_threshold)
    ctx = kb.Context(local)
    levels = torch.empty((k + 1, n), dtype=torch.int32, device=device)
    stream = ctx.stream
    # The per-graph part of a call (validation, degree classes, hub plan,
    # edgeless bits, locality order) is built once (kb_graph_prepare) and timed
    # on its own; every step is one kb_refine_prepared call.
    ctx.prepare(dg, opts).release()  # first-touch of the library's buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pg = ctx.prepare(dg, opts)
    torch.cuda.synchronize()
    prepare_ms = 1000 * (time.perf_counter() - t0)
    prepared_info = pg.info()

    def step():
        return ctx.refine(pg, k, opts, out=levels)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ctx.set_timing(True)
    fam_ms, fam_n = {}, {}
    rounds = 0
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        r = step()
        rounds += r.levels_computed
        round_ms, fam = ctx.timing()
        for name, (ms, cnt) in fam.items():
            fam_ms[name] = fam_ms.get(name, 0.0) + ms
            fam_n[name] = fam_n.get(name, 0) + cnt
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ctx.set_timing(False)
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    if dist:
        t = torch.tensor([elapsed], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        rt = torch.tensor([rounds], device=device, dtype=torch.float64)
        dist.all_reduce(rt)
        total_edge_rounds = float(rt.item()) * m
    else:
        total_edge_rounds = float(rounds) * m
    value = total_edge_rounds / elapsed
    counts_last = [int(x) for x in r.counts]
    del r

    # roofline of the dominant kernel family (algorithmic bytes per launch).
    # A round skips the blocks that cannot change (frozen blocks), so a
    # launch's units are the vertices and edges the round re-keyed, which the
    # library counts when asked to (one more call, outside the timed region).
    ctx.set_timing(2)
    ctx.refine(pg, k, opts, out=levels)
    work = ctx.round_work()
    ctx.set_timing(0)
    # the same calls without preparation (kb_refine: the per-graph part every call)
    ctx.refine(dg, k, opts, out=levels)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(3):
        ctx.refine(dg, k, opts, out=levels)
    ev1.record(stream)
    torch.cuda.synchronize()
    unprepared_ms = ev0.elapsed_time(ev1) / 3
    hub_thr, small_max = (args.hub_threshold or 1024), 32
    deg = (wl["row_offsets"][1:] - wl["row_offsets"][:-1])
    cls_small = deg <= small_max
    cls_hub = deg > hub_thr
    cls_med = ~cls_small & ~cls_hub
    vertex_classes = {"small_le32": [int(cls_small.sum().item()), int(deg[cls_small].sum().item())],
                      "medium": [int(cls_med.sum().item()), int(deg[cls_med].sum().item())],
                      "hub_gt%d" % hub_thr: [int(cls_hub.sum().item()), int(deg[cls_hub].sum().item())]}
    del deg, cls_small, cls_hub, cls_med
    lc = max(1, len(work))
    units = {"small_edges": sum(w["small"][1] for w in work), "med_edges": sum(w["medium"][1] for w in work),
             "hub_edges": sum(w["hub"][1] for w in work), "n_small": sum(w["small"][0] for w in work),
             "n_med": sum(w["medium"][0] for w in work), "n_hubs": sum(w["hub"][0] for w in work)}
    keyed = [[sum(f[0] for f in w.values()), sum(f[1] for f in w.values())] for w in work]
    # per step, then per launch of each family (the medium and hub kernels are
    # launched only in rounds where some of their vertices refine)
    step_bytes = {
        # 12 B per edge (neighbour id 4, edge label 4, gathered block 4) and per
        # vertex 24 B (row offset 8, own block 4, slot write 4, table entry 8)
        "small": 12 * units["small_edges"] + 24 * units["n_small"],
        "medium": 12 * units["med_edges"] + 28 * units["n_med"],
        "hub_chunk": 12 * units["hub_edges"],
        "hub_final": 24 * units["n_hubs"],
        # per vertex: slot 4, table entry 8, level write 4; bitmap read twice
        "renumber": lc * (16 * n + n // 4),
        "other": lc * (n // 8),
    }
    algo_bytes = {kname: step_bytes[kname] / max(1.0, fam_n.get(kname, 0) / args.steps) for kname in step_bytes}
    units = {key: val / lc for key, val in units.items()}
    dom = max(fam_ms, key=lambda kname: fam_ms[kname])
    peak, peak_kind = peaks()
    per_launch_ms = fam_ms[dom] / max(1, fam_n[dom])
    achieved = algo_bytes.get(dom, 0) / (per_launch_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_for(dom, algo_bytes.get(dom, 0)), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": algo_bytes.get(dom, 0),
                "kernel_share": {kname: fam_ms[kname] / sum(fam_ms.values()) for kname in fam_ms},
                "per_launch_ms": {kname: fam_ms[kname] / max(1, fam_n[kname]) for kname in fam_ms}}
    # our kernels per family event: the medium family is a warp kernel and a
    # CTA kernel, the hub-chunk family clears the refining hubs' sets first,
    # renumbering is the 3-kernel rank scan, the stable-round copy, the
    # assignment, the moved count, the dirty, freeze and frozen-count passes
    # and the refining count; "other" is memsets only; per call add level 0
    # over the small labels (label minima, minima marks, rank scan, label ids,
    # assignment, freeze, frozen count, refining count); the setup kernels
    # ran once, in kb_graph_prepare
    per_event = {"small": 1, "medium": 2, "hub_chunk": 2, "hub_final": 1, "renumber": 10, "other": 0}
    launches = int(sum(per_event.get(kname, 1) * cnt for kname, cnt in fam_n.items())) + 10 * args.steps
    # Round 1 is the one round that keys every vertex and every edge (nothing
    # is frozen before it): the full-work figure, with the whole round's
    # algorithmic bytes taken as 12 B per edge (neighbour id, edge label,
    # gathered block) and 40 B per vertex (row offset 8, own block 4, hash 8,
    # table probe and minimum 8, bitmap and scan 8, level write 4).
    r1_ms = round_ms[0] if round_ms else float("nan")
    round1 = {"ms": r1_ms, "edges_per_s": m / (r1_ms / 1000.0),
              "algorithmic_bytes": 12 * m + 40 * n,
              "achieved_gbs": (12 * m + 40 * n) / (r1_ms / 1000.0) / 1e9,
              "frac": (12 * m + 40 * n) / (r1_ms / 1000.0) / 1e9 / peak,
              "peak": peak, "peak_source": peak_kind}

    # end to end through the host-buffer entry point, pinned host memory
    e2e = None
    if not args.no_e2e:
        hrow = wl["row_offsets"].cpu().pin_memory()
        hcol = wl["col"].cpu().pin_memory()
        hel = wl["elabel"].cpu().pin_memory()
        hvl = wl["vlabel"].cpu().pin_memory()
        hout = torch.empty((k + 1, n), dtype=torch.int32).pin_memory()
        np_row, np_col, np_el, np_vl, np_out = (hrow.numpy(), hcol.numpy(), hel.numpy(), hvl.numpy(), hout.numpy())
        ctx.refine_host(np_row, np_col, np_el, np_vl, k, opts, out=np_out)  # warm
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e_rounds = 0
        e_steps = max(1, min(args.steps, 3))
        for _ in range(e_steps):
            rr = ctx.refine_host(np_row, np_col, np_el, np_vl, k, opts, out=np_out)
            e_rounds += rr.levels_computed
            del rr
        et = time.perf_counter() - t0
        if dist:
            t = torch.tensor([et], device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            et = float(t.item())
        h2d = hrow.numel() * 8 + (hcol.numel() + hel.numel()) * 4 + hvl.numel() * 4
        d2h = hout.numel() * 4
        e2e = {"value": e_rounds * m * world / et, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e_steps}
        del hrow, hcol, hel, hvl, hout, np_row, np_col, np_el, np_vl, np_out

    # the next rows: full bisimulation to a fixpoint, and the summary graph of
    # the last two levels (the paper's layer of summary edges) on this graph
    next_rows = None
    if world == 1 and not args.no_summary:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        final, fcount, frounds, fstable = ctx.refine_fixpoint(dg, 64, opts)
        tf = time.perf_counter() - t0
        lc = int(round(rounds / args.steps))
        src_lv, dst_lv = levels[lc], levels[lc - 1]
        ctx.summary(dg, src_lv, dst_lv)  # warm
        t0 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            s_src, s_lab, s_dst = ctx.summary(dg, src_lv, dst_lv)
        ts = (time.perf_counter() - t0) / reps
        # incremental refinement: 1,000 edges relabelled, against the full refinement's time
        gen = torch.Generator(device=device)
        gen.manual_seed(7)
        eidx = torch.randint(0, m, (1000,), generator=gen, device=device)
        el2 = wl["elabel"].clone()
        el2[eidx] = el2[eidx] + 1
        row = wl["row_offsets"]
        src = torch.searchsorted(row, eidx, right=True) - 1
        changed = src.to(torch.int32)
        dg2 = kb.DeviceGraph(row, wl["col"], el2, wl["vlabel"])
        upd_levels = levels.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ures, uwork = ctx.refine_update(dg2, upd_levels, changed, opts)
        torch.cuda.synchronize()
        tu = time.perf_counter() - t0
        # the alternative: a full kb_refine of the changed graph (same clock)
        t0 = time.perf_counter()
        full = ctx.refine(dg2, k, opts)
        torch.cuda.synchronize()
        tfull = time.perf_counter() - t0
        same = bool(torch.equal(full.levels, ures.levels))
        del full, upd_levels, el2, dg2, ures
        next_rows = {
            "fixpoint": {"rounds": frounds, "stable": fstable, "blocks": fcount, "ms": 1000 * tf,
                         "same_as_stratified": bool(torch.equal(final, levels[lc]))},
            "update": {"change": "1,000 random edges relabelled", "ms": 1000 * tu,
                       "full_refine_ms": 1000 * tfull,
                       "timing": "host clock around each synchronous call; full_refine_ms is kb_refine of "
                                 "the changed graph",
                       "rekeyed_vertices_per_level": [int(x) for x in uwork], "same_as_full_refine": same},
            "summary": {"layer": "P_%d -> P_%d, out-edges, edge labels" % (lc, lc - 1),
                        "summary_edges": int(s_src.numel()), "ms": 1000 * ts, "edges_per_s": m / ts,
                        "timing": "host clock around the synchronous call (validation, table, ranking, output)"}}
        del final, s_src, s_lab, s_dst, src_lv, dst_lv
        torch.cuda.empty_cache()

    pg.release()
    del pg
    batch_info = serve_info = None
    if world == 1 and not args.no_batch:
        del wl, dg, levels
        ctx.close()
        torch.cuda.empty_cache()
        ctx = kb.Context(local)
        batch_info = bench_batch(ctx, device)
        torch.cuda.empty_cache()
    if world == 1 and not args.no_serve:
        serve_info = bench_serve(device)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": dict(describe(args.workload, cfg, k, "out"),
                               vertex_classes=vertex_classes,
                               units_per_round=units,
                               counts_last_step=counts_last,
                               l2="inputs larger than L2 (CSR %.1f GB); no flush" % ((8 * (n + 1) + 8 * m) / 1e9),
                               parallelism="replicas" if world > 1 else "single GPU",
                               path="kb_refine_prepared on a graph prepared once (kb_graph_prepare, timed "
                                    "apart as prepare_ms)",
                               rounds_per_step=rounds / args.steps,
                               keyed_vertices_edges_per_round=keyed,
                               kernel_ms_per_round_last_step=[round(x, 2) for x in round_ms]),
                "prepare_ms": prepare_ms,
                "prepared": {key: prepared_info[key] for key in ("reorder", "device_bytes", "n_hubs", "n_medium")},
                "unprepared_ms_per_step": unprepared_ms,
                "round1": round1, "round1_edges_per_s": round1["edges_per_s"], "round1_frac": round1["frac"],
                "roofline": roofline, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
                "batch": batch_info, "serve": serve_info, "next_rows": next_rows}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(cfg)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()



# ----------------------------------------------------------------------------- batching and serving


def bench_batch(ctx, device, steps=3):
    """The batching workload (4,096 uneven graphs) through kb_refine_batch with
    the library defaults, then with the autotuner's choice for this batch (the
    tuning is cached in the context under the batch's size class, and
    kb_refine_batch picks it up), against one kb_refine launch per graph on
    the same GPU."""
    import torch

    import paper_2204_05821_gb300 as kb

    union, voff, ks = graphgen.batch_union_torch(device=device)
    dg = kb.DeviceGraph(union["row_offsets"], union["col"], union["elabel"], union["vlabel"])
    opts = kb.Options()
    G = len(ks)

    def time_batch():
        ctx.refine_batch(dg, voff, ks, opts)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            _, counts, lc = ctx.refine_batch(dg, voff, ks, opts)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps, lc

    ctx.clear_tuning()
    td, lc = time_batch()
    t_tune = time.perf_counter()
    tuning = ctx.autotune(dg, opts, vertex_offsets=voff, ks=ks)
    t_tune = time.perf_counter() - t_tune
    tb, lc = time_batch()
    # plain path: one kb_refine per graph (single-graph calls keep the defaults:
    # the batch's tuning is cached under a batch size class)
    row, col, el, vl = union["row_offsets"], union["col"], union["elabel"], union["vlabel"]
    singles = []
    for j in range(G):
        a, b = int(voff[j]), int(voff[j + 1])
        e0, e1 = int(row[a].item()), int(row[b].item())
        singles.append(kb.DeviceGraph((row[a:b + 1] - e0).contiguous(), (col[e0:e1] - a).contiguous(),
                                      el[e0:e1].contiguous(), vl[a:b].contiguous()))
    for j in range(4):
        ctx.refine(singles[j], int(ks[j]), opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(G):
        ctx.refine(singles[j], int(ks[j]), opts)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    edge_rounds = float(np.sum(lc.astype(np.float64) * np.diff([int(row[int(x)].item()) for x in voff])))
    del singles
    ctx.clear_tuning()
    return {"workload": "4096 ER graphs, edges lognormal(median 5e4, sigma 1.25) in [1e3, 2e6], n=m/5, "
                        "16 vertex / 8 edge labels uniform, k uniform 1..10, seed 3",
            "graphs": G, "edges": int(union["m"]), "vertices": int(union["n"]),
            "graphs_per_s": G / tb, "ms_per_batch": 1000 * tb, "edge_rounds_per_s": edge_rounds / tb,
            "default_graphs_per_s": G / td, "default_ms_per_batch": 1000 * td,
            "tuned": {k: tuning[k] for k in ("load_factor", "hub_threshold", "small_task_vertices",
                                             "hub_chunk_edges", "medium_split", "small_max_degree")},
            "autotune_s": t_tune, "autotune_ms_tuned": tuning["ms"], "autotune_ms_default": tuning["default_ms"],
            "plain_graphs_per_s": G / tp, "plain_ms": 1000 * tp, "speedup_vs_plain": tp / tb}


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(np.ceil(q * len(xs))) - 1))] if xs else None


def bench_serve(device, duration_s=8.0, rate=200.0, seed=4, sat_requests=600):
    """A Poisson stream of summarisation requests through kb_server_*, and the
    same requests through the plain path (one kb_refine_host per request, in
    arrival order): at the nominal rate (p50 / p99 latency from arrival to
    completion, both arms) and at saturation (every request queued at once:
    requests per second, both arms).  Graphs come from a pre-drawn pool
    spanning the size distribution (each request takes the pool graph closest
    to its drawn size), since drawing hundreds of million-edge graphs per
    second on the host is not possible."""
    import threading as th

    import torch

    import paper_2204_05821_gb300 as kb

    stream = graphgen.serve_workload(duration_s=duration_s, rate=rate, seed=seed)
    sizes = np.array([r[1] for r in stream])
    qs = np.unique(np.quantile(sizes, np.linspace(0, 1, 24)).astype(np.int64))
    pool = []
    for i, mm in enumerate(qs):
        n = max(1, int(mm) // 5)
        c = dict(n=n, m=int(mm), gamma_out=2.1, gamma_in=2.1, max_out_deg=max(1.0, mm / 10),
                 max_in_deg=max(1.0, mm / 10), n_vlabels=64, zipf_v=1.5, n_elabels=32, zipf_e=1.2, seed=1000 + i)
        d = graphgen.chung_lu_torch(device=device, **c)
        pool.append(tuple(d[kx].cpu().numpy() for kx in ("row_offsets", "col", "elabel", "vlabel")))
        del d
    torch.cuda.synchronize()
    reqs = [(ta, pool[int(np.argmin(np.abs(qs - mm)))], k) for (ta, mm, k, _) in stream]
    opts = kb.Options()
    # Every request gets its own output array, allocated and touched before
    # any timing, for both arms: the measurement is of the refinement and the
    # copies, not of the host allocator faulting in fresh pages.
    outs = [np.zeros((k + 1, g[0].shape[0] - 1), dtype=np.int32) for _, g, k in reqs]
    for o in outs:
        o.fill(0)
    dev = int(str(device).split(":")[-1]) if ":" in str(device) else 0

    def serve(batch, arrivals):
        """Run requests through a server; arrivals: submit at their times
        (else all at once).  Returns (seconds, stats, latencies_ms)."""
        with kb.Server(dev, max_vertices=1 << 26, max_edges=1 << 28, max_requests=256) as sv:
            for _, (r, c, e, v), k in batch[:4]:  # warm
                sv.submit(r, c, e, v, k, opts)
            while sv.step() != (0, 0):
                pass
            for t in list(sv._meta):
                sv.fetch(t)
            lock = th.Lock()
            tickets, done_at, sub_at = [], {}, {}
            t_start = time.perf_counter()

            def producer():
                for i, (ta, (r, c, e, v), k) in enumerate(batch):
                    if arrivals:
                        dt = t_start + ta - time.perf_counter()
                        if dt > 0:
                            time.sleep(dt)
                    t = sv.submit(r, c, e, v, k, opts, out=outs[i])
                    with lock:
                        tickets.append(t)
                        sub_at[t] = (t_start + ta) if arrivals else t_start

            prod = th.Thread(target=producer)
            prod.start()
            while True:
                running, waiting = sv.step()
                now = time.perf_counter()
                with lock:
                    pending = list(tickets)
                for t in pending:
                    if sv.poll(t) == kb.Server.DONE:
                        sv.fetch(t)
                        done_at[t] = now
                        with lock:
                            tickets.remove(t)
                if not prod.is_alive() and running == 0 and waiting == 0:
                    with lock:
                        if not tickets:
                            break
                if running == 0 and waiting == 0:
                    time.sleep(0.0002)
            prod.join()
            elapsed = time.perf_counter() - t_start
            st = sv.stats()
        lat = [1000 * (done_at[t] - sub_at[t]) for t in done_at]
        return elapsed, st, lat

    def plain(batch, arrivals):
        """One kb_refine_host per request, in arrival order (a FIFO queue)."""
        ctx = kb.Context(dev)
        for _, (r, c, e, v), k in batch[:4]:
            ctx.refine_host(r, c, e, v, k, opts)
        lat = []
        t_start = time.perf_counter()
        for i, (ta, (r, c, e, v), k) in enumerate(batch):
            if arrivals:
                dt = t_start + ta - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            ctx.refine_host(r, c, e, v, k, opts, out=outs[i])
            lat.append(1000 * (time.perf_counter() - (t_start + (ta if arrivals else 0.0))))
        elapsed = time.perf_counter() - t_start
        ctx.close()
        return elapsed, lat

    sv_t, sv_st, sv_lat = serve(reqs, True)
    pl_t, pl_lat = plain(reqs, True)
    sat = reqs[:sat_requests]
    sat_sv_t, _, _ = serve(sat, False)
    sat_pl_t, _ = plain(sat, False)
    return {"workload": "Poisson arrivals %.0f/s for %.0f s; edges lognormal(median 7e5, sigma 1.4) in [1e4, 5e7], "
                        "Chung-Lu exponent 2.1, 64 vertex / 32 edge labels Zipf, k uniform 1..10, seed %d; graphs "
                        "from a pool of %d pre-drawn graphs at the size quantiles" % (rate, duration_s, seed, len(qs)),
            "requests": len(reqs), "completed": int(sv_st["completed"]),
            "nominal_rate": {"server_p50_ms": _pct(sv_lat, 0.5), "server_p99_ms": _pct(sv_lat, 0.99),
                             "plain_p50_ms": _pct(pl_lat, 0.5), "plain_p99_ms": _pct(pl_lat, 0.99),
                             "server_requests_per_s": len(reqs) / sv_t, "plain_requests_per_s": len(reqs) / pl_t,
                             "server_steps": int(sv_st["steps"]), "server_compactions": int(sv_st["compactions"]),
                             "plain": "one kb_refine_host per request, FIFO in arrival order"},
            "saturation": {"requests": len(sat), "server_requests_per_s": len(sat) / sat_sv_t,
                           "plain_requests_per_s": len(sat) / sat_pl_t,
                           "server_vs_plain": sat_pl_t / sat_sv_t,
                           "how": "every request queued at once; plain: back to back"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--hub-threshold", type=int, default=0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-summary", action="store_true", help="skip the fixpoint and summary-graph measurements")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
