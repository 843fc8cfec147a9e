"""Autotuner for the launch schedule (vdmc_schedule_t).

Knobs (results never depend on them; they are checked bit for bit in the
tests):
  hub_min_l          roots with at least this many higher-rank neighbours go
                     to the root-per-CTA kernel (the split between the two
                     kernels)
  hub_blocks_per_sm  CTAs per SM of the root-per-CTA kernel (one scratch
                     slot each)
  a_chunk            depth-1 neighbours per task of the warp-per-task kernel
                     (work-queue granularity)
  warps_per_block    warps per CTA of the warp-per-task kernel (its shared
                     memory -- per-warp credit histograms -- grows with it)
  hub_split,         the largest hub_split_roots roots are each counted by
  hub_split_roots    hub_split CTAs (the critical path of fat-tailed graphs)
  hub_warps          warps per CTA of the root-per-CTA kernel (16 or 32)

The search is staged: the two root-per-CTA knobs first (they dominate on
fat-tailed graphs), then the two warp-kernel knobs with the best of the
first stage, then the root split.  Each candidate is timed with CUDA events after a warm-up
count.  Results are stored per (k, size bucket) in ``tuned_schedules.json``
next to this file; ``apply_tuned`` loads the entry for a graph's bucket.

Command line (on a GPU):
    python -m paper_2201_11655_b300.autotune --workload chunglu_n1M_m10M_a2.3_r0.2 --k 4
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNED_PATH = os.path.join(HERE, "tuned_schedules.json")

STAGE1 = ([{"hub_min_l": h, "hub_blocks_per_sm": b} for h in (1, 2, 4, 8, 16, 32, 64, 128, 256, 1024) for b in (1, 2)] +
          [{"hub_min_l": 0, "hub_blocks_per_sm": 1}])
STAGE2 = [{"a_chunk": a, "warps_per_block": w} for a in (4, 16, 64) for w in (4, 8)]
STAGE3 = ([{"hub_split": 1, "hub_split_roots": 0, "hub_warps": w} for w in (16, 32)] +
          [{"hub_split": s, "hub_split_roots": r, "hub_warps": w} for s, r in ((2, 32), (2, 64), (4, 16), (8, 12))
           for w in (16, 32)])


def bucket(n: int, m: int) -> str:
    """Size bucket: log2 of the vertex count and of the mean degree."""
    d = 2.0 * m / max(n, 1)
    return "n2^%d_d2^%d" % (int(math.log2(max(n, 1))), int(math.log2(max(d, 1.0))))


def time_count(g, k, reps=1):
    import torch
    from . import vdmc
    out = torch.empty((g.n, vdmc.num_classes(k)), dtype=torch.uint64, device="cuda")
    vdmc.count(g, k, out)  # warm-up (rebuilds tasks / scratch for the schedule)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vdmc.count(g, k, out)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune(g, k, stage1=STAGE1, stage2=STAGE2, stage3=STAGE3, reps=1, log=print):
    """Staged search on graph g; returns (best schedule dict, {str(candidate): ms})."""
    from . import vdmc
    base = vdmc.get_schedule()
    timings = {}
    best, best_ms = dict(base), float("inf")
    try:
        for name, stage in (("stage1", stage1), ("stage2", stage2), ("stage3", stage3)):
            base_s = dict(best) if best_ms < float("inf") else dict(base)
            for cand in stage:
                sch = dict(base_s, **cand)
                vdmc.set_schedule(**sch)
                ms = time_count(g, k, reps)
                timings[json.dumps(cand, sort_keys=True)] = ms
                log("%s %s: %.2f ms" % (name, cand, ms))
                if ms < best_ms:
                    best, best_ms = sch, ms
    finally:
        vdmc.set_schedule(**base)
    return best, best_ms, timings


def load_tuned(path=TUNED_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_tuned(key: str, sched: dict, ms: float, meta: dict, path=TUNED_PATH):
    db = load_tuned(path)
    db[key] = {"schedule": sched, "ms": ms, **meta}
    with open(path, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)


def apply_tuned(k: int, n: int, m: int, path=TUNED_PATH) -> dict | None:
    """Set the stored schedule for (k, bucket(n, m)) if there is one; return it."""
    from . import vdmc
    e = load_tuned(path).get("k%d/%s" % (k, bucket(n, m)))
    if e:
        vdmc.set_schedule(**e["schedule"])
        return e["schedule"]
    return None


def main():
    import numpy as np
    import torch
    from . import synth, vdmc
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="chunglu_n1M_m10M_a2.3_r0.2")
    p.add_argument("--k", type=int, default=4)
    p.add_argument("--batch", type=int, default=0, help="tune on a union of N small graphs instead")
    p.add_argument("--reps", type=int, default=1)
    p.add_argument("--out", default=TUNED_PATH)
    p.add_argument("--hub-min-l", default=None, help="comma list: restrict stage 1 to these values")
    p.add_argument("--skip-stage2", action="store_true", help="skip the warp-kernel knobs (stage 2)")
    p.add_argument("--skip-stage3", action="store_true", help="skip the root split and CTA size (stage 3)")
    a = p.parse_args()
    vdmc.load()
    if a.batch:
        graphs = synth.batch(a.batch, 4)
        g = vdmc.graph_create_batch(graphs)
        n, m, name = g.n, sum(len(x[1]) for x in graphs), "batch%d" % a.batch
    else:
        n, s, d = synth.workload(a.workload)
        g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
        m, name = len(s), a.workload
    t0 = time.time()
    stage1 = STAGE1
    if a.hub_min_l:
        keep = {int(x) for x in a.hub_min_l.split(",")}
        stage1 = [c for c in STAGE1 if c["hub_min_l"] in keep]
    best, ms, timings = tune(g, a.k, stage1=stage1, stage2=[] if a.skip_stage2 else STAGE2,
                             stage3=[] if a.skip_stage3 else STAGE3, reps=a.reps)
    key = "k%d/%s" % (a.k, bucket(n, m))
    save_tuned(key, best, ms, {"workload": name, "n": n, "m": m, "timings_ms": timings,
                               "tuned_seconds": round(time.time() - t0, 1)}, a.out)
    print(json.dumps({"key": key, "best": best, "ms": ms}))
    g.close()


if __name__ == "__main__":
    main()
