"""Autotuner for the counting kernel's source split (warp per source vs block per source).

For R-MAT and uniform graphs of increasing size it builds each graph once per candidate threshold, times the count
(CUDA events, median of several launches), keeps the fastest threshold per graph, and writes a size-class table
(class bounds at the geometric midpoints of the graphs' edge counts) to tuning.json, keyed by device name and SM
count.  It then times both counting kernels — the fused traversal and segmented intersection — on uniform graphs of
several sizes and mean degrees and on the R-MAT series, and keeps the wedges-per-edge threshold below which
tc_count takes the intersection kernel that minimises the summed time relative to each graph's faster kernel.
The binding installs the table through tc_set_tuning when the device matches.  Counts do not depend on the
table; only speed does.

It also times the build paths (the compact build with one host synchronisation, and the build that reads each size as
it becomes known) on graphs of increasing size and keeps the largest size at which the compact build still wins
(compact_max_pairs), and likewise for the one-launch build against the compact build on the graphs within its bounds
(tiny_max_pairs); and it times the count with long hop-2 rows
staged through shared memory against plain loads on graphs too large for L2, keeping the smallest CSR size from which
staging wins (stage_min_csr_bytes; 0 if it never does).

    python -m paper_1909_02127_gb300.tune [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CANDIDATES = [1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 20, 1 << 40]


def time_count(tc, g, d_total, reps):
    import torch
    s = torch.cuda.current_stream()
    tc.tc_count_device(g, d_total, s)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(s)
        tc.tc_count_device(g, d_total, s)
        b.record(s)
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    return ms[len(ms) // 2]


def time_build(tc, ds, dd, n, reps):
    """Median time (ms, CUDA events) of tc_load_edges + tc_build from device-resident edges."""
    import torch
    s = torch.cuda.current_stream()
    out = []
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g = tc.tc_load_edges(ds, dd, n, stream=s)
        tc.tc_build(g, s)
        e1.record(s)
        torch.cuda.synchronize()
        tc.tc_free(g)
        out.append(e0.elapsed_time(e1))
    out = sorted(out[1:])
    return out[len(out) // 2]


def largest_winning(rows, fast, slow):
    """The largest pair count up to which the `fast` path is not slower than `slow` on every measured graph (0 if
    it loses on the smallest)."""
    best = 0
    for r in sorted(rows, key=lambda r: r["pairs"]):
        if r[fast] <= r[slow] * 1.01:
            best = r["pairs"]
        else:
            break
    return best


def tune_build_paths(tc, graphgen, quick):
    """Build times of the compact build against the one that reads sizes as known (compact_max_pairs), and on the
    graphs small enough for it, of the one-launch build against the compact build (tiny_max_pairs)."""
    import torch
    names = ["rmat10", "er4096", "rmat12", "rmat13", "rmat14_ef15", "rmat16", "rmat18", "rmat20"] + (
        [] if quick else ["rmat21", "rmat22"])
    rows = []
    base = (tc.tc_get_compact_max_pairs(), tc.tc_get_tiny_max_pairs())
    try:
        for name in names:
            # R-MAT 14 with edge factor 15: 245,760 pairs, near the one-launch build's bound of 2^18 - 1
            spec = graphgen.rmat(14, 15, graphgen.BASE_SEED + 114) if name == "rmat14_ef15" else graphgen.config(name)
            ds, dd = spec.edges(device="cuda")
            row = {"graph": name, "pairs": spec.num_edges, "n": spec.n}
            paths = [("compact_ms", 1 << 40, 0), ("sync_ms", 0, 0)]
            if spec.n <= tc.TINY_MAX_VERTICES and spec.num_edges <= tc.TINY_MAX_PAIRS:
                paths.append(("tiny_ms", 0, tc.TINY_MAX_PAIRS))
            for path, cmp, tiny in paths:
                tc.tc_set_tuning(tc.tc_get_tuning(), compact_max_pairs=cmp, tiny_max_pairs=tiny)
                row[path] = round(time_build(tc, ds, dd, spec.n, 3 if quick else 7), 4)
            rows.append(row)
            print(row, flush=True)
            del ds, dd
            torch.cuda.empty_cache()
    finally:
        tc.tc_set_tuning(tc.tc_get_tuning(), compact_max_pairs=base[0], tiny_max_pairs=base[1])
    tiny_rows = [r for r in rows if "tiny_ms" in r]
    return rows, largest_winning(rows, "compact_ms", "sync_ms"), largest_winning(tiny_rows, "tiny_ms", "compact_ms")


def tune_staging(tc, graphgen, quick):
    import torch
    names = ["rmat22", "rmat24"] + ([] if quick else ["rmat26"])
    rows = []
    base = (tc.tc_get_stage_min_csr_bytes(), tc.tc_get_isect_max_wedges_milli())
    d_total = torch.zeros(1, dtype=torch.int64, device="cuda")
    try:
        tc.tc_set_tuning(tc.tc_get_tuning(), isect_max_wedges_milli=0)  # the fused kernel, whose loads are staged
        for name in names:
            spec = graphgen.config(name)
            ds, dd = spec.edges(device="cuda")
            g = tc.tc_load_edges(ds, dd, spec.n)
            try:
                tc.tc_build(g)
                del ds, dd
                torch.cuda.empty_cache()
                info = tc.tc_graph_get_info(g)
                row = {"graph": name, "csr_bytes": 8 * (info["num_vertices"] + 1) + 4 * info["csr_entries"]}
                for key, thr in (("plain_ms", 0), ("staged_ms", 1)):
                    tc.tc_set_tuning(tc.tc_get_tuning(), stage_min_csr_bytes=thr)
                    row[key] = round(time_count(tc, g, d_total, 3), 3)
            finally:
                tc.tc_free(g)
            rows.append(row)
            print(row, flush=True)
            torch.cuda.empty_cache()
    finally:
        tc.tc_set_tuning(tc.tc_get_tuning(), stage_min_csr_bytes=base[0], isect_max_wedges_milli=base[1])
    wins = [r for r in sorted(rows, key=lambda r: r["csr_bytes"]) if r["staged_ms"] < r["plain_ms"]]
    if not wins:
        return rows, 0
    first = wins[0]
    below = [r for r in rows if r["csr_bytes"] < first["csr_bytes"]]
    # between the largest losing size and the smallest winning one (geometric midpoint)
    thr = int(math.sqrt(max(r["csr_bytes"] for r in below) * first["csr_bytes"])) if below else first["csr_bytes"]
    return rows, thr


def main():
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build

    p = argparse.ArgumentParser()
    p.add_argument("--quick", action="store_true")
    p.add_argument("--out", default=tc.TUNING_FILE)
    args = p.parse_args()
    build.build()
    tc.load_library()
    scales = [14, 17, 20, 22] if args.quick else [12, 14, 16, 18, 20, 21, 22, 23, 24]
    specs = [graphgen.rmat(sc, 16, graphgen.BASE_SEED + 500 + sc, name=f"rmat{sc}") for sc in scales]
    specs += [graphgen.gnp(1 << 20, 16.0 / ((1 << 20) - 1), graphgen.BASE_SEED + 600, name="G(n=2^20, p=16/(n-1))")]
    reps = 3 if args.quick else 5
    d_total = torch.zeros(1, dtype=torch.int64, device="cuda")
    results = []
    for spec in specs:
        ds, dd = spec.edges(device="cuda")
        row = {"graph": spec.name, "times_ms": {}}
        count = None
        for cand in CANDIDATES:
            tc.tc_set_tuning([(1 << 62, cand)], isect_max_wedges_milli=0)
            g = tc.tc_load_edges(ds, dd, spec.n)
            try:
                tc.tc_build(g)
                row["m"] = tc.tc_graph_get_info(g)["num_edges"]
                row["times_ms"][str(cand)] = time_count(tc, g, d_total, reps)
                c = int(d_total.item())
                if count is not None and c != count:
                    raise RuntimeError("count changed with the tuning")
                count = c
            finally:
                tc.tc_free(g)
        row["best"] = int(min(row["times_ms"], key=row["times_ms"].get))
        results.append(row)
        print(row["graph"], row["m"], row["best"], {k: round(v, 3) for k, v in row["times_ms"].items()}, flush=True)
        del ds, dd
        torch.cuda.empty_cache()
    # size classes from the skewed (R-MAT) series, where the split matters; a graph keeps the previous class's
    # threshold when that is within 2% of its best, so measurement noise does not split classes
    series = sorted((r for r in results if r["graph"].startswith("rmat")), key=lambda r: r["m"])
    classes = []
    for i, r in enumerate(series):
        bound = int(math.sqrt(r["m"] * series[i + 1]["m"])) if i + 1 < len(series) else 1 << 62
        t = r["times_ms"]
        choice = r["best"]
        if classes and str(classes[-1][1]) in t and t[str(classes[-1][1])] <= 1.02 * t[str(choice)]:
            choice = classes[-1][1]
        if classes and classes[-1][1] == choice:
            classes[-1][0] = bound
        else:
            classes.append([bound, choice])
    # batches: how large a graph may be and still run all its sources one warp each (timed on the batch mix)
    tc.tc_set_tuning([tuple(c) for c in classes])
    mix = graphgen.batch_mix(512 if args.quick else 1024)
    handles = []
    for sp in mix:
        s_, d_ = sp.edges(device="cuda")
        handles.append(tc.tc_load_edges(s_, d_, sp.n))
        tc.tc_build(handles[-1])
    batch_times = {}
    ref = None
    for cand in (0, 1 << 20, 1 << 22, 1 << 25, 1 << 62):
        tc.tc_set_tuning([tuple(c) for c in classes], batch_warp_max_edges=cand)
        got = tc.tc_count_batch(handles)
        torch.cuda.synchronize()
        if ref is not None and not (got == ref).all():
            raise RuntimeError("batch counts changed with the tuning")
        ref = got
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tc.tc_count_batch(handles)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        batch_times[str(cand)] = sorted(ts)[len(ts) // 2]
    for h in handles:
        tc.tc_free(h)
    batch_warp = int(min(batch_times, key=batch_times.get))
    print("batch", {k: round(v, 3) for k, v in batch_times.items()}, flush=True)
    # the per-graph choice of kernel: time both on every graph, then pick the threshold on W/m
    method_specs = [graphgen.gnp(1 << lg, deg / ((1 << lg) - 1), graphgen.BASE_SEED + 700 + 10 * lg + deg,
                                 name=f"G(n=2^{lg}, p={deg}/(n-1))")
                    for lg in ((16, 20, 22) if args.quick else (16, 18, 20, 22)) for deg in (4, 8, 16)]
    method_specs += [graphgen.rmat(sc, 16, graphgen.BASE_SEED + 500 + sc, name=f"rmat{sc}")
                     for sc in ((14, 18) if args.quick else (12, 16, 20))]
    method_rows = []
    for spec in method_specs:
        ds, dd = spec.edges(device="cuda")
        g = tc.tc_load_edges(ds, dd, spec.n)
        try:
            tc.tc_build(g)
            info = tc.tc_graph_get_info(g)
            row = {"graph": spec.name, "m": info["num_edges"],
                   "wedges_milli": (1000 * info["num_wedges"] + max(info["num_edges"], 1) - 1) // max(info["num_edges"], 1)}
            counts = set()
            for name, ratio in (("fused", 0), ("intersect", 1 << 62)):
                tc.tc_set_tuning([tuple(c) for c in classes], batch_warp_max_edges=batch_warp,
                                 isect_max_wedges_milli=ratio)
                row[name + "_ms"] = time_count(tc, g, d_total, reps)
                counts.add(int(d_total.item()))
            if len(counts) != 1:
                raise RuntimeError("the two kernels disagree")
        finally:
            tc.tc_free(g)
        method_rows.append(row)
        print(row, flush=True)
        del ds, dd
        torch.cuda.empty_cache()

    def cost(t):
        return sum((r["intersect_ms"] if 0 < r["wedges_milli"] <= t else r["fused_ms"])
                   / min(r["intersect_ms"], r["fused_ms"]) for r in method_rows)

    cands = [0] + sorted({r["wedges_milli"] for r in method_rows})
    isect_ratio = min(cands, key=lambda t: (cost(t), t))
    print("isect_max_wedges_milli", isect_ratio, {t: round(cost(t), 3) for t in cands}, flush=True)
    # the table chosen so far is installed before the build and staging sweeps (the method sweep leaves the last
    # kernel it timed selected)
    tc.tc_set_tuning([tuple(c) for c in classes], batch_warp_max_edges=batch_warp, isect_max_wedges_milli=isect_ratio)
    build_rows, compact_pairs, tiny_pairs = tune_build_paths(tc, graphgen, args.quick)
    print("compact_max_pairs", compact_pairs, "tiny_max_pairs", tiny_pairs, flush=True)
    stage_rows, stage_bytes = tune_staging(tc, graphgen, args.quick)
    print("stage_min_csr_bytes", stage_bytes, flush=True)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    out = {"device": props.name, "sms": props.multi_processor_count, "cc": f"{props.major}.{props.minor}",
           "classes": classes, "batch_warp_max_edges": batch_warp, "batch_times_ms": batch_times,
           "isect_max_wedges_milli": isect_ratio, "method_measurements": method_rows,
           "bucket_max_pairs": tc.tc_get_bucket_max_pairs(), "measurements": results,
           "compact_max_pairs": compact_pairs, "tiny_max_pairs": tiny_pairs, "build_measurements": build_rows,
           "stage_min_csr_bytes": stage_bytes, "staging_measurements": stage_rows}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    tc.tc_set_tuning([tuple(c) for c in classes], batch_warp_max_edges=batch_warp,
                     isect_max_wedges_milli=isect_ratio, compact_max_pairs=compact_pairs,
                     stage_min_csr_bytes=stage_bytes, tiny_max_pairs=tiny_pairs)
    print(json.dumps({"classes": classes, "batch_warp_max_edges": batch_warp, "isect_max_wedges_milli": isect_ratio,
                      "compact_max_pairs": compact_pairs, "stage_min_csr_bytes": stage_bytes,
                      "tiny_max_pairs": tiny_pairs}))


if __name__ == "__main__":
    main()
