"""Benchmark: per-vertex directed k-motif counting on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--k 3|4]

A step is one vdmc_count over the whole graph (every root, every BFS
structure), with the graph already resident in HBM.  Prints ONE JSON line.

value      connected k-sets counted per second (instances/s), device time
           measured with CUDA events on the launching stream.  config splits
           the sets into those enumerated one by one and those the
           root-per-CTA kernel accounts for by signature (vdmc_count_stats).
e2e        the same metric through the public API with HOST buffers: each
           step builds the graph from pinned host arcs (H2D inside), counts,
           and copies the uint64 counts back to pinned host memory.
roofline   HBM roofline of one count: algorithmic bytes (vdmc_work_model:
           N(r), N(a) per depth-1 vertex, N(b) per distinct depth-2 vertex,
           output) / device time against the measured copy peak.
cpu_baseline  the CPU oracle on a bounded root sample of the same graph.

--impl reference times the CPU oracle alone (the reference arm of this
benchmark), on the host cores, on a bounded sample of the same workload.
N > 1 (torchrun): one graph, its roots split into N rank ranges of equal
estimated work (Lemma 1), one count of its range per GPU and one uint64
sum-reduce of the per-vertex counts (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "chunglu_n1M_m10M_a2.3_r0.2"
METRIC = "k=%d per-vertex motif instances/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--k", type=int, default=4)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target oracle sample time")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--batch-graphs", type=int, default=50_000)
    p.add_argument("--batch-compare", type=int, default=2_000,
                   help="graphs of the batch also counted one launch per graph")
    p.add_argument("--no-sub", action="store_true", help="skip the 4M-vertex ER and G(100, 0.08) sub-benchmarks")
    p.add_argument("--serve-requests", type=int, default=2000, help="requests per offered-load point")
    p.add_argument("--serve-n-hi", type=int, default=50_000)
    p.add_argument("--serve-loads", default="0.25,0.5,0.75,0.9", help="offered loads (fractions of capacity)")
    p.add_argument("--no-tuned", action="store_true", help="keep the library's default schedule")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_hash():
    """Hash of the root-per-CTA kernel's sources (the kernel the traffic record covers)."""
    h = hashlib.sha256()
    for name in ("hub.cu", "device_common.cuh", "vdmc_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2201_11655_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_traffic(k):
    """The committed one-launch ncu record of the root-per-CTA kernel on a smaller
    graph of the same shape (profiles/traffic_small_case.json), if it was taken
    on the current kernel sources.  Its DRAM bytes are not scaled to the full
    workload: the ratio to the algorithmic bytes grows with the graph (the
    scratch of all slots outgrows L2), so `traffic` stays null and the record is
    reported beside it."""
    path = os.path.join(ROOT, "profiles", "traffic_small_case.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        e = rec.get("k%d" % k)
        if e and e.get("kernel_hash") == kernel_source_hash():
            return dict(e, ratio_to_algorithmic=e["dram_bytes_per_launch"] / e["algorithmic_bytes_of_count"])
    except Exception:
        pass
    return None


def load_traffic_full(k):
    """The committed one-launch ncu record of the root-per-CTA kernel on the
    full-size workload itself (profiles/traffic_full_size.json: DRAM bytes read
    + written, a one-pass capture), if it was taken on the current kernel
    sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic_full_size.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        e = rec.get("k%d" % k)
        if e and e.get("kernel_hash") == kernel_source_hash():
            return dict(e, ratio_to_algorithmic=e["dram_bytes_per_launch"] / e["algorithmic_bytes_of_count"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", "vdmc_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def oracle_sample(n, s, d, k, target_s, threads=None):
    """Time the oracle on a contiguous range of root ranks, grown until it takes ~target_s.

    Returns dict(value=instances/s, instances, seconds, sample=str, cores)."""
    from oracle import oracle as O
    threads = threads or O.default_threads()
    rank = O.degree_rank(n, s, d)
    # graph build cost of one oracle call (empty root range), subtracted
    t0 = time.perf_counter()
    O.count_roots(n, s, d, k, rank, 0, 0, threads=threads)
    build_s = time.perf_counter() - t0
    lo = min(n - 1, max(0, n // 100))
    w = 64
    while True:
        hi = min(n, lo + w)
        t0 = time.perf_counter()
        _, found = O.count_roots(n, s, d, k, rank, lo, hi, threads=threads)
        el = time.perf_counter() - t0 - build_s
        if el >= target_s or hi >= n or w > n:
            break
        w = int(w * max(2.0, min(8.0, target_s / max(el, 1e-3))))
    return {"value": found / max(el, 1e-9), "instances": int(found), "seconds": el, "cores": threads,
            "sample": "oracle (ESU + k! canonicalisation, %d threads) on the roots of degree rank [%d, %d) "
                      "of the same graph: %d connected %d-sets in %.2f s (its own graph build, %.2f s, "
                      "subtracted)" % (threads, lo, hi, found, k, el, build_s), "lo": lo, "hi": hi}


_WORKLOADS = {}


def workload(name):
    """synth.workload(name), drawn once per process (the sub-benchmarks reuse graphs)."""
    from paper_2201_11655_b300 import synth
    if name not in _WORKLOADS:
        _WORKLOADS[name] = synth.workload(name)
    return _WORKLOADS[name]


def timed_ms(fn, reps=3, stream=None):
    """Best of `reps` device times (CUDA events on the launching stream) after one untimed call."""
    import torch
    stream = stream or torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def launches_per_count(g, schedule):
    """Kernels one vdmc_count launches: the warp-per-task kernel, the
    root-per-CTA kernel, the split-root finish and the un-relabel pass."""
    info = g.info()
    n_split = min(schedule["hub_split_roots"], info["num_hub_roots"]) if schedule["hub_split"] > 1 else 0
    return (1 if info["num_tasks"] > 0 else 0) + (1 if info["num_hub_roots"] > 0 else 0) + \
        (1 if n_split > 0 else 0) + (1 if info["n"] > 0 else 0)


def rates(stats, ms):
    sec = ms / 1e3
    return {"instances_enumerated": stats["sets_enumerated"], "instances_by_signature": stats["sets_by_signature"],
            "enumerated_per_s": stats["sets_enumerated"] / sec,
            "by_signature_per_s": stats["sets_by_signature"] / sec,
            "stats": stats}


def roofline_of(model, ms, peak, peak_kind, kernel, traffic=None, traffic_src=None):
    achieved = model["bytes"] / (ms / 1e3) / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
         "traffic": traffic, "kernel": kernel, "algorithmic_bytes_per_launch": model["bytes"],
         "peak_kind": "%s hbm_gbs (copy)" % peak_kind,
         "per_use_model": {"bytes": model["bytes_per_use"],
                           "frac": model["bytes_per_use"] / (ms / 1e3) / 1e9 / peak},
         "model": model}
    if traffic_src:
        r["traffic_small_case"] = traffic_src
    return r


def bench_single(name, k, peak, peak_kind, base_schedule, tuned=True, override=None, reps=3):
    """One named single-graph workload: device time per count, instances/s
    (enumerated / by signature), algorithmic-byte roofline.  The schedule is
    the library default (base_schedule), then the tuned entry of the graph's
    size bucket if any, then `override`."""
    import torch
    from paper_2201_11655_b300 import autotune, synth, vdmc
    n, s, d = workload(name)
    saved = vdmc.get_schedule()
    vdmc.set_schedule(**base_schedule)
    sched = autotune.apply_tuned(k, n, len(s)) if tuned else None
    if override:
        vdmc.set_schedule(**override)
    g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    try:
        out = torch.empty((n, vdmc.num_classes(k)), dtype=torch.uint64, device="cuda")
        ms = timed_ms(lambda: vdmc.count(g, k, out), reps=reps)
        torch.cuda.synchronize()
        if g.device_status() != 0:
            raise RuntimeError("device status error in %s" % name)
        total = int(out.view(torch.int64).sum().item())
        if total % k:
            raise RuntimeError("sum of per-vertex counts is not a multiple of k")
        inst = total // k
        stats = g.count_stats()
        if stats["sets_enumerated"] + stats["sets_by_signature"] != inst:
            raise RuntimeError("set counters disagree with the counts")
        model = g.work_model(k)
        res = {"workload": name, "k": k, "n": n, "arcs": int(len(s)), "ms_per_count": ms,
               "instances": inst, "instances_per_s": inst / (ms / 1e3),
               "schedule": vdmc.get_schedule(),
               "schedule_source": ("tuned" if sched else "default") + ("+%s" % override if override else ""),
               "roofline": roofline_of(model, ms, peak, peak_kind, "vdmc_count (all kernels of one count)")}
        res.update(rates(stats, ms))
        return res
    finally:
        g.close()
        vdmc.set_schedule(**saved)


def bench_variant(name, k, peak, peak_kind, base_schedule, undirected=False, per_edge=False, tuned=True, reps=3):
    """The undirected variant and the per-edge counts on a named workload:
    device time per count, sets/s (from the count's set counters), byte
    roofline (per-edge: the output is one row per edge of G_U)."""
    import torch
    from paper_2201_11655_b300 import autotune, synth, vdmc
    n, s, d = workload(name)
    saved = vdmc.get_schedule()
    vdmc.set_schedule(**base_schedule)
    sched = autotune.apply_tuned(k, n, len(s)) if tuned else None
    g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), undirected=undirected)
    try:
        C = g.num_classes(k)
        ne = g.info()["edges_u"]
        out = torch.empty((ne if per_edge else n, C), dtype=torch.uint64, device="cuda")
        fn = (lambda: vdmc.count_edges(g, k, out)) if per_edge else (lambda: vdmc.count(g, k, out))
        ms = timed_ms(fn, reps=reps)
        torch.cuda.synchronize()
        if g.device_status() != 0:
            raise RuntimeError("device status error in %s" % name)
        st = g.count_stats()
        inst = st["sets_enumerated"] + st["sets_by_signature"]
        if not per_edge and int(out.view(torch.int64).sum().item()) != k * inst:
            raise RuntimeError("set counters disagree with the counts")
        model = g.work_model(k)
        if per_edge:  # the output is one row per edge instead of per vertex
            model = dict(model)
            out_b = 8 * ne * C + 4 * n
            for key in ("bytes", "bytes_per_use"):
                model[key] = model[key] - model["output_bytes"] + out_b
            model["output_bytes"] = out_b
        res = {"workload": name, "k": k, "undirected": undirected, "per_edge": per_edge, "n": n,
               "edges_u": ne, "columns": C, "ms_per_count": ms, "instances": inst,
               "instances_per_s": inst / (ms / 1e3), "schedule": vdmc.get_schedule(),
               "schedule_source": "tuned" if sched else "default",
               "roofline": roofline_of(model, ms, peak, peak_kind, "vdmc_count_edges" if per_edge else "vdmc_count")}
        res.update(rates(st, ms))
        return res
    finally:
        g.close()
        vdmc.set_schedule(**saved)


def bench_batch(args, ks=(3, 4)):
    """Batched graphs/s: many small uneven graphs (n log-uniform in [10, 500],
    half G(n,p), half Chung-Lu, p ~ U[0.02, 0.2]) counted in one launch over
    their concatenated CSR, against one vdmc_count launch per graph on a
    subset (same pre-built graphs; builds excluded from both), and against
    vdmc_count_batch (cached plan, CUDA-graph replay) on that subset."""
    import torch
    from paper_2201_11655_b300 import autotune, synth, vdmc
    t0 = time.perf_counter()
    graphs = synth.batch(args.batch_graphs, 4)
    gen_s = time.perf_counter() - t0
    res = {"workload": "%d graphs, n log-uniform [10,500], G(n,p) / Chung-Lu 2.5, p~U[0.02,0.2]" % len(graphs),
           "generate_s": gen_s}
    for k in ks:
        C = vdmc.num_classes(k)
        saved = vdmc.get_schedule()
        vdmc.set_schedule(**getattr(args, "base_schedule", saved))
        tuned = None if args.no_tuned else autotune.apply_tuned(k, sum(g[0] for g in graphs),
                                                                sum(len(g[1]) for g in graphs))
        try:
            t0 = time.perf_counter()
            U = vdmc.graph_create_batch(graphs)
            build_s = time.perf_counter() - t0
            out = torch.empty((U.n, C), dtype=torch.uint64, device="cuda")
            ms_union = timed_ms(lambda: vdmc.count(U, k, out))
            inst = int(out.view(torch.int64).sum().item()) // k
            stats = U.count_stats()
            U.close()
            sub = graphs[:args.batch_compare]
            gs = [vdmc.graph_create(n, s, d) for n, s, d in sub]
            outs = [torch.empty((g.n, C), dtype=torch.uint64, device="cuda") for g in gs]
            ms_each = timed_ms(lambda: [vdmc.count(g, k, o) for g, o in zip(gs, outs)], reps=1)
            ms_plan = timed_ms(lambda: vdmc.count_batch(gs, k, outs=outs))
            Us = vdmc.graph_create_batch(sub)
            outs_u = torch.empty((Us.n, C), dtype=torch.uint64, device="cuda")
            ms_union_sub = timed_ms(lambda: vdmc.count(Us, k, outs_u))
            # identical results: union rows == per-graph counts
            vdmc.count(Us, k, outs_u)
            [vdmc.count(g, k, o) for g, o in zip(gs, outs)]
            torch.cuda.synchronize()
            same = all(torch.equal(outs_u[Us.offsets[i]:Us.offsets[i + 1]].view(torch.int64),
                                   outs[i].view(torch.int64)) for i in range(len(gs)))
            Us.close()
            for g in gs:
                g.close()
            r = {"k": k, "schedule": tuned or saved, "schedule_source": "tuned" if tuned else "default",
                 "graphs_per_s": len(graphs) / (ms_union / 1e3), "ms_per_batch": ms_union,
                 "instances_per_s": inst / (ms_union / 1e3), "instances": inst, "union_build_s": build_s,
                 "subset": {"graphs": len(sub), "one_launch_per_graph_graphs_per_s": len(sub) / (ms_each / 1e3),
                            "count_batch_replay_graphs_per_s": len(sub) / (ms_plan / 1e3),
                            "union_graphs_per_s": len(sub) / (ms_union_sub / 1e3),
                            "identical_results": bool(same)}}
            r.update(rates(stats, ms_union))
            res["k%d" % k] = r
        finally:
            vdmc.set_schedule(**saved)
    return res


def bench_serve(args):
    """Served requests (see paper_2201_11655_b300.serve.sweep): Poisson
    arrivals swept over offered load, against one plain launch per request."""
    from paper_2201_11655_b300 import serve
    return serve.sweep(num=args.serve_requests, n_hi=args.serve_n_hi, loads=args.serve_loads, seed=5)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_2201_11655_b300 import synth
    from oracle import oracle as O
    n, s, d = synth.workload(args.workload)
    O.build()
    threads = O.default_threads()
    probe = oracle_sample(n, s, d, args.k, max(2.0, args.cpu_seconds / 3))
    lo, hi = probe["lo"], probe["hi"]
    rk = O.degree_rank(n, s, d)
    times, found = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, found = O.count_roots(n, s, d, args.k, rk, lo, hi, threads=threads)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
    sec = sum(times) / len(times)
    val = found / sec
    unit = "instances/s"
    print(json.dumps({
        "impl": "reference", "metric": METRIC % args.k, "value": val, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "k": args.k, "n": n, "arcs": int(s.size)},
        "cpu_baseline": {"value": val, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": "each step: oracle on the roots of degree rank [%d, %d) (%d connected %d-sets, "
                                   "graph build included)" % (lo, hi, found, args.k)},
        "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch

    from paper_2201_11655_b300 import build, synth, vdmc

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build.build()
    vdmc.load()
    base_schedule = vdmc.get_schedule()  # the library default, before any tuned entry
    k = args.k
    C = vdmc.num_classes(k)
    n, s, d = workload(args.workload)
    m = int(s.size)
    tuned = None
    if not args.no_tuned:
        from paper_2201_11655_b300 import autotune
        tuned = autotune.apply_tuned(k, n, m)
    stream = torch.cuda.current_stream()
    src_dev = torch.from_numpy(s).cuda()
    dst_dev = torch.from_numpy(d).cuda()
    g = vdmc.graph_create(n, src_dev, dst_dev)
    info = g.info()
    del src_dev, dst_dev
    sharded = world > 1
    if sharded:
        # one graph, its roots split into `world` ranges of equal estimated
        # work (Lemma 1); one uint64 sum-reduce of the partial counts
        from paper_2201_11655_b300 import shard
        bounds = shard.partition(g, k, world)
        count_fn = lambda: shard.count_sharded(g, k, out, bounds, rank, dist)
    else:
        count_fn = lambda: vdmc.count(g, k, out)
    out = torch.empty((n, C), dtype=torch.uint64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > L2 (126 MB)

    for _ in range(args.warmup):
        count_fn()
    torch.cuda.synchronize()
    if g.device_status() != 0:
        raise RuntimeError("device status error after warm-up")
    ref = out.view(torch.int64).clone()
    total = int(ref.sum().item())
    if total % k:
        raise RuntimeError("sum of per-vertex counts is not a multiple of k")
    instances = total // k

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local_rank) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()  # evict L2 between timed launches
            evs[i][0].record(stream)
            count_fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    # the timed counts are checked too: status word clean, output unchanged
    if g.device_status() != 0:
        raise RuntimeError("device status error in the timed region")
    if not torch.equal(out.view(torch.int64), ref):
        raise RuntimeError("timed counts differ from the warm-up counts")
    del ref
    stats = g.count_stats()
    if not sharded and stats["sets_enumerated"] + stats["sets_by_signature"] != instances:
        raise RuntimeError("set counters disagree with the counts")
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # sharded: every rank counts a share of the one graph's sets
    value = (instances if sharded else world * instances) / (ms / 1e3)

    # e2e through the public API with host buffers
    e2e = None
    if not args.no_e2e and not sharded:
        src_h = torch.from_numpy(s).pin_memory()
        dst_h = torch.from_numpy(d).pin_memory()
        out_h = torch.empty((n, C), dtype=torch.int64).pin_memory()
        e2e_steps = max(1, min(args.steps, 3))
        tt = []
        for i in range(1 + e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with vdmc.graph_create(n, src_h, dst_h) as g2:
                vdmc.count(g2, k, out)
                out_h.copy_(out.view(torch.int64), non_blocking=True)
                torch.cuda.synchronize()
            el = time.perf_counter() - t0
            if i > 0:
                tt.append(el)
        e2e_s = sum(tt) / len(tt)
        e2e = {"value": world * instances / e2e_s, "unit": "instances/s", "ms_per_step": e2e_s * 1e3,
               "h2d_bytes_per_step": 8 * m, "d2h_bytes_per_step": 8 * n * C,
               "path": "vdmc_graph_create(host arcs) + vdmc_count + D2H of counts"}

    peak, peak_kind = load_peaks()
    model = g.work_model(k)
    roofline = roofline_of(model, ms, peak, peak_kind,
                           "vdmc_count: hub_kernel<%d, %s warps> (root-per-CTA) overlapped with count_kernel<%d> "
                           "(warp-per-task), timed together" % (k, vdmc.get_schedule()["hub_warps"] or "16 or 32", k),
                           None, load_traffic(k))
    # traffic: DRAM bytes of one root-per-CTA launch of this very workload and
    # schedule, when the committed full-size record matches the kernel sources
    # (else null)
    full = load_traffic_full(k) if args.workload == DEFAULT_WORKLOAD and not args.no_tuned else None
    if full:
        roofline["traffic"] = full["dram_bytes_per_launch"]
        roofline["traffic_full_size"] = full

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            smp = oracle_sample(n, s, d, k, args.cpu_seconds)
            cpu = {"value": smp["value"], "unit": "instances/s", "cores": smp["cores"], "kind": "oracle",
                   "sample": smp["sample"]}
        except Exception as ex:  # the oracle is a baseline only
            cpu = {"value": None, "unit": "instances/s", "cores": None, "kind": "oracle", "sample": "failed: %s" % ex}

    launches = launches_per_count(g, vdmc.get_schedule()) * args.steps
    g.close()
    extra = {}
    if rank == 0 and world == 1 and not args.no_sub:
        # the 4M-vertex ER graph: the paper's enumeration alone (every root
        # to the warp-per-task kernel), and with roots of >= 16 higher-rank
        # neighbours sent to the root-per-CTA kernel
        extra["er4m"] = bench_single("er_n4M_m32M", 4, peak, peak_kind, base_schedule, tuned=not args.no_tuned,
                                     override={"hub_min_l": 0})
        extra["er4m_hub16"] = bench_single("er_n4M_m32M", 4, peak, peak_kind, base_schedule, tuned=False,
                                           override={"hub_min_l": 16})
        # the same power-law graph at the other k
        other = 3 if k == 4 else 4
        extra["%s_k%d" % (args.workload, other)] = bench_single(args.workload, other, peak, peak_kind, base_schedule,
                                                               tuned=not args.no_tuned)
        # the variants of the Discussion / Tables 1-2: undirected motifs of the
        # same power-law graph, per-edge counts of the 1M ER graph (the per-edge
        # path enumerates every set, so not the hub-heavy graph)
        extra["undirected"] = bench_variant(args.workload, k, peak, peak_kind, base_schedule, undirected=True,
                                            tuned=not args.no_tuned)
        extra["per_edge"] = bench_variant("er_n1M_m8M", 4, peak, peak_kind, base_schedule, per_edge=True,
                                          tuned=False)
        extra["gnp100"] = {"k3": bench_single("gnp_n100_p0.08", 3, peak, peak_kind, base_schedule, tuned=False),
                           "k4": bench_single("gnp_n100_p0.08", 4, peak, peak_kind, base_schedule, tuned=False)}
    if rank == 0 and world == 1 and not args.no_batch:
        args.base_schedule = base_schedule
        extra["batch"] = bench_batch(args)
    if rank == 0 and world == 1 and not args.no_serve:
        extra["serve"] = bench_serve(args)
    if rank == 0:
        cfg = {"workload": args.workload, "k": k, "n": n, "arcs": m, "edges_u": info["edges_u"],
               "max_degree": info["max_degree"], "instances_per_step": instances,
               "l2": "256 MB buffer written between timed launches (L2 flush)",
               "parallelism": ("root-range shards x%d + uint64 all-reduce" % world) if sharded else "single",
               "schedule": vdmc.get_schedule()}
        if not sharded:
            cfg.update(rates(stats, ms))
        line = {
            "metric": METRIC % k, "value": value, "unit": "instances/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu, "step_ms": step_ms, "schedule_source": "tuned" if tuned else "default",
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
