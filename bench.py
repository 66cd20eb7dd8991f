"""Benchmark of the GB300 triangle counter.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload rmat20|rmat26|er4096|batch]

A step is one pass of the whole hot path over one synthetic graph: ingest (validate + pack the edge list), CSR
build (sort, dedup, degree, orientation, offsets, bins) and the fused count.  `value` is GTEPS = m / t_step with the
edge list already resident in HBM (m = distinct undirected edges); `e2e` repeats the step through the C ABI from
pinned host buffers, the host->device copy of the edge list and the device->host read of the count included.
Per-phase times, count-only GTEPS and the dominant kernel's roofline are reported beside it.

Under torchrun (N > 1) every rank counts its own graph (same workload, seed + rank): independent problems, weak
scaling, no collective on the data path; the barrier and the max over ranks are for timing only.

--impl reference times the CPU oracle (test infrastructure, never tuned) on the host cores for the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="rmat20",
                   help="rmat20 | rmat26 | er4096 | batch | serve | unfused | prune | list | rmat<scale> (R-MAT, edge factor 16)")
    p.add_argument("--graph", default="rmat20", help="unfused, list: the graph")
    p.add_argument("--unfused-chunk-bytes", type=int, default=0,
                   help="unfused: bytes one hop-2 pass may hold (0: the largest pass)")
    p.add_argument("--batch-graphs", type=int, default=4096)
    p.add_argument("--rate", type=float, default=2000.0, help="serve: mean request arrivals per second")
    p.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    p.add_argument("--serve-pool", type=int, default=1024, help="serve: distinct request graphs")
    p.add_argument("--build-workers", type=int, default=6, help="serve: concurrent CSR builders")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--allocator", default="library", choices=["library", "torch"],
                   help="device memory for graphs: the library's pool, or torch's caching allocator")
    return p.parse_args()


# ------------------------------------------------------------------------------------------------------------
# Distributed plumbing (timing only)
# ------------------------------------------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")

    def _reduce(self, x, op):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(local_units: float, local_seconds: float, dist: Dist):
    """Whole-job rate: units summed over ranks / the slowest rank's time."""
    units = dist.sum(local_units)
    secs = dist.max(local_seconds)
    return units, secs


# ------------------------------------------------------------------------------------------------------------
# Clocks during the timed region
# ------------------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------------------
# Roofline helpers
# ------------------------------------------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def count_kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("tc_count.cuh", "tc_count.cu", "tc_internal.cuh", "tc_prims.cuh"):
        with open(os.path.join(ROOT, "paper_1909_02127_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the count kernel from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"k_count_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != count_kernel_source_hash():
        return None
    return float(m_tr.group(1))


def algorithmic_bytes(info: dict, grid_ctas: int) -> float:
    """Bytes the two-hop method must read once per use: offsets of every source (8(n+1)), its row N+(u) (4m), the
    offset pair of every hop-1 target (16m), the row N+(v) of every hop-1 target — 4 bytes per id for rows read
    as id lists (4(W - W_dense)) and 16 bytes per 128-id quad for rows read as bitmaps (16 Q_dense) — and one
    8-byte atomic per CTA."""
    n, m, W = info["num_vertices"], info["num_edges"], info["num_wedges"]
    Wd, Qd = info.get("dense_wedges", 0), info.get("dense_quads", 0)
    return 8.0 * (n + 1) + 4.0 * m + 16.0 * m + 4.0 * (W - Wd) + 16.0 * Qd + 8.0 * grid_ctas


def count_grid(info: dict) -> int:
    want = info["bin_block"] + (info["bin_warp"] + 15) // 16 + (info.get("bin_thread", 0) + 511) // 512
    return int(max(1, min(want, 2 * 152)))


# ------------------------------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------------------------------
def run_single(args, dist: Dist):
    import numpy as np
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    base = graphgen.config(args.workload)
    spec = dataclasses.replace(base, seed=base.seed + dist.rank)
    stream = torch.cuda.current_stream()
    ds, dd = spec.edges(device=dev)
    torch.cuda.synchronize()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    d_total = torch.zeros(1, dtype=torch.int64, device=dev)
    alloc = "torch" if args.allocator == "torch" else None

    def step(events=None):
        if events:
            events[0].record(stream)
        g = tc.tc_load_edges(ds, dd, spec.n, stream=stream, allocator=alloc)
        tc.tc_build(g, stream)
        if events:
            events[1].record(stream)
        tc.tc_count_device(g, d_total, stream)
        if events:
            events[2].record(stream)
        return g

    # warm-up (also fixes the graph's sizes)
    info = None
    T_ref = None
    for _ in range(args.warmup):
        g = step()
        info = tc.tc_graph_get_info(g)
        torch.cuda.synchronize()
        T_now = int(d_total.item())
        if T_ref is not None and T_now != T_ref:
            raise RuntimeError("count changed between warm-up steps")
        T_ref = T_now
        tc.tc_free(g)
    if info is None:
        g = step()
        info = tc.tc_graph_get_info(g)
        torch.cuda.synchronize()
        T_ref = int(d_total.item())
        tc.tc_free(g)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(dist.local)
    launches0 = tc.tc_kernel_launches()
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k)  # L2 flush between timed steps (outside the events)
        g = step(evs[k])
        tc.tc_free(g)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clock_info = clocks.stop()
    dist.barrier()
    launches = tc.tc_kernel_launches() - launches0
    if int(d_total.item()) != T_ref:
        raise RuntimeError("count changed in the timed region")
    step_ms = [evs[k][0].elapsed_time(evs[k][2]) for k in range(args.steps)]
    build_ms = [evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)]
    count_ms = [evs[k][1].elapsed_time(evs[k][2]) for k in range(args.steps)]
    local_s = sum(step_ms) / 1e3
    m = info["num_edges"]
    units, secs = aggregate(m * args.steps, local_s, dist)
    value = units / secs / 1e9

    # end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        hs = ds.cpu().pin_memory()
        hd = dd.cpu().pin_memory()
        for _ in range(max(1, min(args.warmup, 2))):
            g = tc.tc_load_edges(hs, hd, spec.n, stream=stream, allocator=alloc)
            tc.tc_build(g, stream)
            tc.tc_count(g, stream)
            tc.tc_free(g)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g = tc.tc_load_edges(hs, hd, spec.n, stream=stream, allocator=alloc)
            tc.tc_build(g, stream)
            T_e2e = tc.tc_count(g, stream)
            tc.tc_free(g)
            if T_e2e != T_ref:
                raise RuntimeError("end-to-end count differs")
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        u2, s2 = aggregate(m * args.steps, e2e_s, dist)
        e2e = {"value": round(u2 / s2 / 1e9, 4), "unit": "GTEPS", "h2d_bytes_per_step": int(spec.num_edges * 8),
               "d2h_bytes_per_step": 8}

    peak, peak_kind = measured_peaks()
    grid = count_grid(info)
    b_alg = algorithmic_bytes(info, grid)
    mean_count_s = statistics.mean(count_ms) / 1e3
    achieved = b_alg / mean_count_s / 1e9
    ratio = tc.tc_get_isect_max_wedges_milli()
    isect = ratio > 0 and m > 0 and 1000 * info["num_wedges"] <= ratio * m  # the kernel tc_count picks
    traffic = None if isect else profiled_traffic(args.workload)
    roofline = {"bound": "hbm", "kernel": "k_count_isect" if isect else "k_count", "achieved": round(achieved, 1),
                "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "algorithmic_bytes": b_alg}

    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, ds, dd, T_ref)

    out = {
        "metric": "triangle-count GTEPS (R-MAT 20/26; ingest+build+count per step)",
        "value": round(value, 4), "unit": "GTEPS", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": workload_config(spec, "2x L2 buffer written between timed steps; edge list (8 B/pair) exceeds L2",
                                  dist.world),
        "m": m, "wedges": info["num_wedges"], "triangles": T_ref, "allocator": args.allocator,
        "phases_ms": {"build": round(statistics.mean(build_ms), 4), "count": round(statistics.mean(count_ms), 4)},
        "count_gteps": round(m / mean_count_s / 1e9, 4),
        "triangles_per_s": round(T_ref / mean_count_s, 1),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clock_info,
        "wall_s_timed": round(wall, 4),
    }
    return out


# Graphs above this many generated pairs are sampled for the CPU legs: the oracle takes minutes on them.
CPU_WHOLE_MAX_PAIRS = 1 << 25


def workload_config(spec, l2, world):
    """The workload's identity, the same on both arms."""
    return {"workload": spec.name, "n": spec.n, "generated_pairs": spec.num_edges, "seed": spec.seed, "l2": l2,
            "parallelism": f"replicas x{world}"}


def cpu_sample(spec, scale):
    """The graph the CPU legs time: the workload itself when it is small enough, else an R-MAT graph of the same
    recipe (edge factor, noise, seed, id permutation) at a smaller scale; the rate per edge is the reported unit."""
    import graphgen
    if spec.num_edges <= CPU_WHOLE_MAX_PAIRS:
        return spec, f"whole {spec.name} graph"
    small = graphgen.rmat(scale, 16, spec.seed, permute=True, name=f"R-MAT scale {scale} ef 16 (permuted ids)")
    return small, f"{small.name}, same recipe and seed as {spec.name}"


def cpu_baseline(spec, ds, dd, T_expect):
    """The oracle as it stands, on all host cores: the same graph when small enough, else a smaller graph of the
    same recipe (build + count)."""
    import oracle
    sample, what = cpu_sample(spec, 22)
    if sample is spec:
        hs, hd = ds.cpu().numpy(), dd.cpu().numpy()
    else:
        hs, hd = sample.edges()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    T, m = oracle.count(hs, hd, sample.n, threads=cores)
    t = time.perf_counter() - t0
    if sample is spec and T != T_expect:
        raise RuntimeError(f"oracle {T} != GPU {T_expect}")
    return {"value": round(m / t / 1e9, 5), "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": f"{what} (sort+CSR+merge count), m = {m}, {t:.2f} s"}


def run_unfused(args, dist: Dist):
    """The ablation of Algorithm 1's unfused loop: the same graph counted by tc_count_unfused (frontiers written to
    memory and compacted each round) and by the fused kernel, both timed with CUDA events on one stream."""
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    base = graphgen.config(args.graph)
    spec = dataclasses.replace(base, seed=base.seed + dist.rank)
    stream = torch.cuda.current_stream()
    ds, dd = spec.edges(device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    d_total = torch.zeros(1, dtype=torch.int64, device=dev)
    g = tc.tc_load_edges(ds, dd, spec.n, stream=stream)
    tc.tc_build(g, stream)
    info = tc.tc_graph_get_info(g)
    T = tc.tc_count(g, stream)
    stats = None
    for _ in range(max(1, args.warmup)):
        T_u, stats = tc.tc_count_unfused(g, args.unfused_chunk_bytes, stream)
        tc.tc_count_device(g, d_total, stream)
        if T_u != T:
            raise RuntimeError(f"unfused count {T_u} != fused {T}")
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(dist.local)
    launches0 = tc.tc_kernel_launches()
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k)
        evs[k][0].record(stream)
        T_u, _ = tc.tc_count_unfused(g, args.unfused_chunk_bytes, stream)
        evs[k][1].record(stream)
        flush.fill_(k + 1)
        evs[k][2].record(stream)
        tc.tc_count_device(g, d_total, stream)
        evs[k][3].record(stream)
        if T_u != T:
            raise RuntimeError("unfused count changed in the timed region")
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    dist.barrier()
    launches = tc.tc_kernel_launches() - launches0
    if int(d_total.item()) != T:
        raise RuntimeError("fused count changed in the timed region")
    tc.tc_free(g)
    unf_ms = [e[0].elapsed_time(e[1]) for e in evs]
    fused_ms = [e[2].elapsed_time(e[3]) for e in evs]
    m = info["num_edges"]
    units, secs = aggregate(m * args.steps, sum(unf_ms) / 1e3, dist)
    t_unf = statistics.mean(unf_ms) / 1e3
    peak, peak_kind = measured_peaks()
    # hop-2 frontier bytes: per slot the column read, the keep-flag write, the scan's read and write of it and
    # the compaction's read (5 x 4 B)
    frontier_bytes = 20 * stats["frontier2"]
    return {
        "metric": "unfused-loop count GTEPS (Algorithm 1 frontiers materialised) vs the fused kernel",
        "value": round(units / secs / 1e9, 4), "unit": "GTEPS", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(unf_ms), 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": workload_config(spec, "2x L2 buffer written before each timed count", dist.world),
        "m": m, "triangles": T, "wedges_padded": info["num_wedges"],
        "unfused": {"ms": round(statistics.mean(unf_ms), 3), **stats,
                    "chunk_bytes": args.unfused_chunk_bytes},
        "fused": {"ms": round(statistics.mean(fused_ms), 4), "intermediate_bytes": 0,
                  "gteps": round(m / (statistics.mean(fused_ms) / 1e3) / 1e9, 4)},
        "slowdown_unfused_vs_fused": round(statistics.mean(unf_ms) / statistics.mean(fused_ms), 2),
        "roofline": {"bound": "hbm", "kernel": "unfused loop (all of its kernels)",
                     "achieved": round(frontier_bytes / t_unf / 1e9, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(frontier_bytes / t_unf / 1e9 / peak, 4), "traffic": None,
                     "algorithmic_bytes": frontier_bytes},
        "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clock_info,
    }


def run_list(args, dist: Dist):
    """Triangle listing: every triangle of the graph written as ascending original-id triples into device memory
    (tc_list_triangles), timed with CUDA events; the count kernel on the same graph beside it."""
    import ctypes

    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    base = graphgen.config(args.graph)
    spec = dataclasses.replace(base, seed=base.seed + dist.rank)
    stream = torch.cuda.current_stream()
    ds, dd = spec.edges(device=dev)
    g = tc.tc_load_edges(ds, dd, spec.n, stream=stream)
    tc.tc_build(g, stream)
    info = tc.tc_graph_get_info(g)
    T = tc.tc_count(g, stream)
    out = torch.empty((max(T, 1), 3), dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    lib = tc.load_library()
    found = ctypes.c_uint64()
    sp = ctypes.c_void_p(stream.cuda_stream)

    def list_all():
        st = lib.tc_list_triangles(g, 0, spec.n, out.data_ptr(), T, ctypes.byref(found), tc.TC_PTR_DEVICE, sp)
        if st != tc.TC_OK or found.value != T:
            raise RuntimeError(f"listing: status {st}, found {found.value} of {T}")

    for _ in range(max(1, args.warmup)):
        list_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(dist.local)
    launches0 = tc.tc_kernel_launches()
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        list_all()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    dist.barrier()
    launches = tc.tc_kernel_launches() - launches0
    # spot check: a sample of the listed triples are triangles of the input (sorted, distinct, adjacent)
    sample = out[torch.randint(0, max(T, 1), (4096,), device=dev)].cpu().numpy() if T else None
    if sample is not None:
        import numpy as np
        hs, hd = ds.cpu().numpy().astype(np.int64), dd.cpu().numpy().astype(np.int64)
        edges = np.unique(np.minimum(hs, hd) * spec.n + np.maximum(hs, hd))
        t = sample.astype(np.int64)

        def present(x):
            i = np.minimum(np.searchsorted(edges, x), edges.size - 1)
            return edges[i] == x

        ok = (t[:, 0] < t[:, 1]) & (t[:, 1] < t[:, 2])
        ok &= present(t[:, 0] * spec.n + t[:, 1]) & present(t[:, 1] * spec.n + t[:, 2])
        ok &= present(t[:, 0] * spec.n + t[:, 2])
        if not ok.all():
            raise RuntimeError(f"listing: {int((~ok).sum())} sampled triples are not triangles")
    count_ms = []
    d_total = torch.zeros(1, dtype=torch.int64, device=dev)
    for k in range(args.steps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tc.tc_count_device(g, d_total, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        count_ms.append(e0.elapsed_time(e1))
    tc.tc_free(g)
    list_ms = [a.elapsed_time(b) for a, b in ev]
    units, secs = aggregate(T * args.steps, sum(list_ms) / 1e3, dist)
    out_bytes = 12 * T
    t_list = statistics.mean(list_ms) / 1e3
    peak, peak_kind = measured_peaks()
    # what listing must move: one traversal (the counting pass's bytes, dense rows as bitmaps) and per triangle its
    # 12-byte triple and the 4-byte rank -> id lookup of its third vertex.  The second traversal of the two-pass
    # design (per-source counts, then the triples) is not counted: it shows as a lower fraction.
    list_bytes = algorithmic_bytes(info, 2 * 152) + 16.0 * T
    return {
        "metric": "triangles listed per second (ascending original-id triples into device memory)",
        "value": round(units / secs, 1), "unit": "triangles/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(list_ms), 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": workload_config(spec, "2x L2 buffer written before each timed listing", dist.world),
        "m": info["num_edges"], "triangles": T, "output_bytes": out_bytes,
        "count_ms": round(statistics.mean(count_ms), 4),
        "roofline": {"bound": "hbm", "kernel": "k_list (counting and listing passes)",
                     "achieved": round(list_bytes / t_list / 1e9, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(list_bytes / t_list / 1e9 / peak, 4), "traffic": None,
                     "algorithmic_bytes": list_bytes},
        "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clock_info,
    }


def run_batch(args, dist: Dist):
    import numpy as np
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    specs = graphgen.batch_mix(args.batch_graphs, graphgen.BASE_SEED + graphgen.BATCH_SEED_OFFSET
                               + dist.rank * 1000003)
    handles = []
    for sp in specs:
        s, d = sp.edges(device=dev)
        h = tc.tc_load_edges(s, d, sp.n, stream=stream)
        tc.tc_build(h, stream)
        handles.append(h)
    torch.cuda.synchronize()
    solo = np.array([tc.tc_count(h, stream) for h in handles], dtype=np.uint64)
    if not np.array_equal(tc.tc_count_batch(handles, stream), solo):
        raise RuntimeError("batched counts differ from one-by-one counts")
    plan = tc.tc_batch_plan_create(handles, stream)  # the launch sequence, captured once as a CUDA graph
    got = np.zeros(len(handles), dtype=np.uint64)
    for _ in range(args.warmup):
        tc.tc_batch_plan_run(plan, len(handles), stream, got)
        if not np.array_equal(got, solo):
            raise RuntimeError("batched counts differ from one-by-one counts")
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    l0 = tc.tc_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tc.tc_batch_plan_run(plan, len(handles), stream, got)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    launches = tc.tc_kernel_launches() - l0
    clock_info = clocks.stop()
    if not np.array_equal(got, solo):
        raise RuntimeError("batched counts differ")
    # one graph per launch, same graphs and counts
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        for h in handles:
            tc.tc_count(h, stream)
    t_solo = (time.perf_counter() - t0) / max(1, args.steps // 2)
    units, secs = aggregate(len(handles) * args.steps, t_batch, dist)
    u1, s1 = aggregate(len(handles), t_solo, dist)
    tc.tc_batch_plan_free(plan)
    for h in handles:
        tc.tc_free(h)
    return {
        "metric": "batched graphs/s (4096-graph mix, one persistent launch replayed from a CUDA graph) vs one graph "
                  "per launch",
        "value": round(units / secs, 2), "unit": "graphs/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_batch / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": {"workload": f"batch of {len(handles)} graphs (ER/R-MAT mix, n log-uniform [64, 65536])",
                   "total_triangles": int(solo.sum()), "parallelism": f"replicas x{dist.world}"},
        "one_by_one_graphs_per_s": round(u1 / s1, 2),
        "speedup_vs_one_by_one": round((units / secs) / (u1 / s1), 3),
        "e2e": None, "gpu_launches": int(launches), "clocks": clock_info,
    }


def run_prune(args, dist: Dist):
    """Does the NE filter to a fixpoint (2-core peeling) pay for itself on the batch mix?  The same graphs are
    loaded and built plainly and pruned, and counted with one batch plan each; build and count are timed apart."""
    import numpy as np
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    specs = graphgen.batch_mix(args.batch_graphs, graphgen.BASE_SEED + graphgen.BATCH_SEED_OFFSET
                               + dist.rank * 1000003)
    edges = [sp.edges(device=dev) for sp in specs]
    torch.cuda.synchronize()

    def build_all(pruned):
        hs, removed, kept = [], 0, 0
        t0 = time.perf_counter()
        for sp, (s, d) in zip(specs, edges):
            h = tc.tc_load_edges(s, d, sp.n, stream=stream)
            if pruned:
                removed += tc.tc_build_pruned(h, 0, stream)["edges_removed"]
            else:
                tc.tc_build(h, stream)
            hs.append(h)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        kept = sum(tc.tc_graph_get_info(h)["num_edges"] for h in hs)
        return hs, t, removed, kept

    def count_all(hs):
        plan = tc.tc_batch_plan_create(hs, stream)
        got = np.zeros(len(hs), dtype=np.uint64)
        for _ in range(args.warmup):
            tc.tc_batch_plan_run(plan, len(hs), stream, got)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tc.tc_batch_plan_run(plan, len(hs), stream, got)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / args.steps
        tc.tc_batch_plan_free(plan)
        return got.copy(), t

    out = {}
    counts = {}
    clocks = ClockSampler(dist.local)
    dist.barrier()
    clocks.start()
    l0 = tc.tc_kernel_launches()
    for name, pruned in (("plain", False), ("pruned", True)):
        for h in build_all(pruned)[0]:  # warm-up build (pool growth, first-call setup)
            tc.tc_free(h)
        hs, t_build, removed, kept = build_all(pruned)
        counts[name], t_count = count_all(hs)
        for h in hs:
            tc.tc_free(h)
        out[name] = {"build_s": round(t_build, 4), "count_ms": round(t_count * 1e3, 3), "edges_kept": kept,
                     "edges_removed": removed}
    launches = tc.tc_kernel_launches() - l0
    clock_info = clocks.stop()
    if not np.array_equal(counts["plain"], counts["pruned"]):
        raise RuntimeError("pruned counts differ")
    total = {k: v["build_s"] + v["count_ms"] / 1e3 for k, v in out.items()}
    units, secs = aggregate(len(specs), total["pruned"], dist)
    return {
        "metric": "batch mix: build + one batched count, with the NE filter to a fixpoint (2-core) vs without",
        "value": round(units / secs, 2), "unit": "graphs/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total["pruned"] * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": {"workload": f"batch of {len(specs)} graphs (ER/R-MAT mix, n log-uniform [64, 65536])",
                   "parallelism": f"replicas x{dist.world}"},
        **out, "pays": total["pruned"] < total["plain"],
        "plain_graphs_per_s": round(len(specs) / total["plain"], 2),
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clock_info,
    }


def run_serve(args, dist: Dist):
    """Replay one Poisson arrival trace against the serving loop twice: continuous batching, then one graph per
    launch.  Every result is checked against the graph's solo count."""
    import threading

    import numpy as np
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    pool = graphgen.serve_pool(args.serve_pool, graphgen.BASE_SEED + graphgen.SERVE_SEED_OFFSET + dist.rank * 7919)
    gen = [sp.edges(device=dev) for sp in pool]
    sizes = np.array([int(s.numel()) for s, _ in gen], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    total = int(offs[-1])
    host = torch.empty(2 * total, dtype=torch.int32).pin_memory()
    for i, (s, d) in enumerate(gen):
        host[offs[i]:offs[i + 1]].copy_(s)
        host[total + offs[i]:total + offs[i + 1]].copy_(d)
    torch.cuda.synchronize()
    del gen
    base = host.data_ptr()
    src_ptr = [base + 4 * int(offs[i]) for i in range(len(pool))]
    dst_ptr = [base + 4 * (total + int(offs[i])) for i in range(len(pool))]
    solo = []
    for i, sp in enumerate(pool):
        g = tc.tc_load_edges(host[offs[i]:offs[i + 1]], host[total + offs[i]:total + offs[i + 1]], sp.n)
        tc.tc_build(g)
        solo.append(tc.tc_count(g))
        tc.tc_free(g)
    arrivals = graphgen.poisson_arrivals(args.rate, args.duration)
    key = graphgen.stream_key(graphgen.BASE_SEED + graphgen.SERVE_SEED_OFFSET - 2, graphgen.STREAM_PARAMS)
    half = len(pool) // 2
    pick = [2 * (graphgen.draw(key, j) % half) + (j % 2) for j in range(len(arrivals))]

    def replay(batching: bool):
        srv = tc.tc_server_create(batching=batching, build_workers=args.build_workers)
        results = []
        done = threading.Event()
        expected = len(arrivals)

        def poller():
            while len(results) < expected and not done.is_set():
                results.extend(tc.tc_server_poll(srv, 8192, 20))

        th = threading.Thread(target=poller)
        th.start()
        owner = {}
        t0 = time.perf_counter()
        for j, ta in enumerate(arrivals):
            wait = t0 + ta - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            k = pick[j]
            owner[tc.tc_server_submit(srv, src_ptr[k], dst_ptr[k], int(sizes[k]), pool[k].n)] = k
        th.join(timeout=args.duration * 20 + 600)
        done.set()
        stats = tc.tc_server_get_stats(srv)
        tc.tc_server_destroy(srv)
        if len(results) != expected:
            raise RuntimeError(f"serve: {len(results)} of {expected} requests finished")
        bad = [r for r in results if r["status"] != 0 or r["triangles"] != solo[owner[r["id"]]]]
        if bad:
            raise RuntimeError(f"serve: {len(bad)} results differ from their solo counts")
        lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in results])
        span = (max(r["t_done_ns"] for r in results) - min(r["t_submit_ns"] for r in results)) / 1e9
        return {"graphs_per_s": round(expected / span, 2), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
                "launches": stats["launches"], "max_batch": stats["max_batch_seen"],
                "mean_batch": round(stats["completed"] / max(1, stats["launches"]), 2),
                "peak_held_gb": round(stats["peak_held_bytes"] / 1e9, 3), "requests": expected,
                "span_s": round(span, 3)}

    clocks = ClockSampler(dist.local)
    dist.barrier()
    clocks.start()
    l0 = tc.tc_kernel_launches()
    batched = replay(True)
    launches = tc.tc_kernel_launches() - l0
    clock_info = clocks.stop()
    single = replay(False)
    units, secs = aggregate(batched["requests"], batched["span_s"], dist)
    return {
        "metric": "served graphs/s with p50/p99 latency (Poisson arrivals, continuous batching) vs one graph per launch",
        "value": round(units / secs, 2), "unit": "graphs/s", "n_gpus": dist.world, "steps": 1, "warmup": 0,
        "ms_per_step": round(batched["span_s"] * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": {"workload": f"Poisson {args.rate:g} req/s for {args.duration:g} s over {len(pool)} R-MAT/ER "
                               f"graphs, pairs log-uniform [1e3, 4e6]",
                   "pool_pairs": total, "build_workers": args.build_workers, "parallelism": f"replicas x{dist.world}"},
        "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"], "batched": batched, "one_by_one": single,
        "speedup_vs_one_by_one": round(batched["graphs_per_s"] / single["graphs_per_s"], 3),
        "e2e": {"value": round(units / secs, 2), "unit": "graphs/s",
                "h2d_bytes_per_step": int(8 * sum(sizes[k] for k in pick)), "d2h_bytes_per_step": 8 * len(pick)},
        "gpu_launches": int(launches), "clocks": clock_info,
    }


# ------------------------------------------------------------------------------------------------------------
# Reference arm: the CPU oracle
# ------------------------------------------------------------------------------------------------------------
def run_reference(args, dist: Dist):
    import graphgen
    import oracle
    if dist.rank != 0:
        return None
    if args.workload in ("batch", "serve", "unfused", "prune", "list"):
        return {"impl": "reference", "unavailable": "the oracle arm is defined for the single-graph workloads"}
    spec = graphgen.config(args.workload)
    sample, what = cpu_sample(spec, 21)
    hs, hd = sample.edges()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.count(hs, hd, sample.n, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        T, m = oracle.count(hs, hd, sample.n, threads=cores)
        times.append(time.perf_counter() - t0)
    value = m * len(times) / sum(times) / 1e9
    return {
        "impl": "reference", "metric": "triangle-count GTEPS (R-MAT 20/26; ingest+build+count per step)",
        "value": round(value, 5), "unit": "GTEPS", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(times) * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": workload_config(spec, "CPU arm: no device cache to flush", dist.world),
        "sample_m": m, "sample_triangles": T,
        "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                         "sample": f"{what} per step (sort+CSR+merge count), m = {m}"},
        "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        dist.init("gloo")
        out = run_reference(args, dist)
        dist.close()
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    tc.load_library()
    dist.init("nccl")
    if args.workload == "batch":
        out = run_batch(args, dist)
    elif args.workload == "serve":
        out = run_serve(args, dist)
    elif args.workload == "unfused":
        out = run_unfused(args, dist)
    elif args.workload == "prune":
        out = run_prune(args, dist)
    elif args.workload == "list":
        out = run_list(args, dist)
    else:
        out = run_single(args, dist)
    dist.close()
    if dist.rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
