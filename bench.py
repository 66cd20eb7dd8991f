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
    p.add_argument("--serve-rates", default="2000,5000,6000,7000,8000,10000",
                   help="serve: offered rates (req/s) of the capacity sweep, comma-separated ('' for none)")
    p.add_argument("--sweep-duration", type=float, default=2.0, help="serve: seconds of arrivals per swept rate")
    p.add_argument("--no-extras", action="store_true",
                   help="rmat20: leave out the R-MAT 26, per-vertex/listing, batch and serving sub-records")
    p.add_argument("--rmat26-launches", type=int, default=5, help="R-MAT 26 sub-record: timed count launches")
    p.add_argument("--extra-serve-duration", type=float, default=10.0,
                   help="serving sub-record: seconds of arrivals at --rate")
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
class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, clock-event reasons); None if unavailable."""
    SM = 1  # NVML_CLOCK_SM
    # clock-event reason bits (nvml.h): software power cap, hardware slowdown, software / hardware thermal
    # slowdown, hardware power brake (reported as a hardware slowdown)
    REASONS = ((0x4, "sw_power_cap"), (0x8, "hw_slowdown"), (0x20, "sw_thermal_slowdown"),
               (0x40, "hw_thermal_slowdown"), (0x80, "hw_slowdown"))

    def __init__(self, lib, handle):
        import ctypes
        self.lib, self.handle, self._u = lib, handle, ctypes.c_uint
        self._reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)

    @classmethod
    def open(cls, uuid: str = None, index: int = 0):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if uuid and lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0:
                return cls(lib, h)
            if lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(h)) == 0:
                return cls(lib, h)
        except (OSError, AttributeError):
            pass
        return None

    def sample(self):
        """(sm_mhz, sm_max_mhz, [reason names]) or None."""
        import ctypes
        cur, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.handle, self.SM, ctypes.byref(cur)) != 0:
            return None
        if self.lib.nvmlDeviceGetMaxClockInfo(self.handle, self.SM, ctypes.byref(mx)) != 0:
            return None
        names = []
        if self._reasons is not None and self._reasons(self.handle, ctypes.byref(rs)) == 0:
            names = sorted({name for bit, name in self.REASONS if rs.value & bit})
        return float(cur.value), float(mx.value), names


def summarize_clocks(samples, source):
    """samples: [(sm_mhz, sm_max_mhz, reasons)] -> the bench line's clocks record."""
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [f"{source}: no samples"], "samples": 0,
                "source": source}
    reasons = sorted({r for _, _, rs in samples for r in rs})
    return {"sm_mhz": statistics.median(x[0] for x in samples), "sm_max_mhz": max(x[1] for x in samples),
            "reasons": reasons, "samples": len(samples), "source": source}


class ClockSampler:
    """SM clocks and throttle reasons during a timed region: NVML read every 5 ms in a thread, else nvidia-smi
    every 50 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_s: float = 0.005):
        self.gpu = gpu_index
        self.period = period_s
        self.proc = None
        self.path = None
        self.nvml = None
        self.thread = None
        self.samples = []
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(gpu_index).uuid)
        except Exception:
            uuid = None
        self.nvml = _Nvml.open(uuid, gpu_index)

    def start(self):
        import threading
        self.samples = []
        if self.nvml is not None:
            self._stop = threading.Event()

            def loop():
                while True:
                    x = self.nvml.sample()
                    if x is not None:
                        self.samples.append(x)
                    if self._stop.wait(self.period):
                        return

            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            return
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
        if self.thread is not None:
            self._stop.set()
            self.thread.join(timeout=5)
            self.thread = None
            x = self.nvml.sample()  # at least one sample, taken as the region ends
            if x is not None:
                self.samples.append(x)
            return summarize_clocks(self.samples, "nvml 5 ms")
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        samples = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm, smax = float(parts[1]), float(parts[2])
                except ValueError:
                    continue
                samples.append((sm, smax, [n for n, v in zip(names, parts[5:9]) if v.lower().startswith("active")]))
        os.unlink(self.path)
        return summarize_clocks(samples, "nvidia-smi 50 ms")


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


def algorithmic_bytes_ids(info: dict, grid_ctas: int) -> float:
    """The same reads with every hop-2 row counted as an id list (4 bytes per candidate 2-path, 4W), as if no row
    were read as a bitmap."""
    n, m, W = info["num_vertices"], info["num_edges"], info["num_wedges"]
    return 8.0 * (n + 1) + 4.0 * m + 16.0 * m + 4.0 * W + 8.0 * grid_ctas


def count_grid(info: dict) -> int:
    """CTAs of the counting kernel's launch, as the library reports it (tc_graph_info.count_ctas)."""
    return int(max(1, info["count_ctas"]))


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
    csr_bytes = 8 * (info["num_vertices"] + 1) + 4 * info["csr_entries"]
    l2_resident = csr_bytes <= L2_BYTES
    roofline = {"bound": "l2" if l2_resident else "hbm", "kernel": "k_count_isect" if isect else "k_count",
                "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "algorithmic_bytes": b_alg,
                "dram_frac": round(traffic / mean_count_s / 1e9 / peak, 4) if traffic else None,
                "csr_bytes": csr_bytes}
    if l2_resident:
        roofline["note"] = ("the CSR fits in the 129 MB L2, so the kernel reads it from L2 (DRAM traffic is "
                            "dram_frac of the HBM peak): issue- and L2-latency-bound; frac = algorithmic bytes / "
                            "time against the HBM copy peak")

    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, ds, dd, T_ref)
        if args.workload == "rmat20":
            cpu["single_thread"] = cpu_single_thread()
    extras = {}
    if args.workload == "rmat20" and dist.world == 1 and not args.no_extras:
        extras = run_extras(args, dist, dev, stream, flush)

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
        **extras,
    }
    return out


GOLDEN_RMAT26 = os.path.join(ROOT, "tests", "golden", "rmat26_oracle.json")


def stored_oracle(path: str):
    """A stored oracle result (written by a committed script that calls only the oracle), or None."""
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def sub_rmat26(args, dev, stream, flush) -> dict:
    """R-MAT scale 26 (2^30 pairs, permuted ids): ingest + build timed once after a warm-up build, then the counting
    pass timed over several launches with CUDA events on its stream (the 5 GB CSR is 40x the L2, so the L2 flush
    between launches changes little).  The count is compared with the oracle's stored T."""
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    spec = graphgen.config("rmat26")
    ds, dd = spec.edges(device=dev)
    torch.cuda.synchronize()
    build_ms = []
    g = None
    for _ in range(2):
        if g is not None:
            tc.tc_free(g)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = tc.tc_load_edges(ds, dd, spec.n, stream=stream)
        tc.tc_build(g, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        build_ms.append(e0.elapsed_time(e1))
    del ds, dd
    try:
        info = tc.tc_graph_get_info(g)
        d_total = torch.zeros(1, dtype=torch.int64, device=dev)
        T = tc.tc_count(g, stream)
        tc.tc_count_device(g, d_total, stream)  # second warm-up launch
        count_ms = []
        launches0 = tc.tc_kernel_launches()
        for k in range(args.rmat26_launches):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tc.tc_count_device(g, d_total, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            count_ms.append(e0.elapsed_time(e1))
            if int(d_total.item()) != T:
                raise RuntimeError("R-MAT 26 count changed between launches")
        launches = tc.tc_kernel_launches() - launches0
    finally:
        tc.tc_free(g)
    torch.cuda.empty_cache()
    peak, peak_kind = measured_peaks()
    grid = count_grid(info)
    t = statistics.mean(count_ms) / 1e3
    b_kernel = algorithmic_bytes(info, grid)
    b_ids = algorithmic_bytes_ids(info, grid)
    m = info["num_edges"]
    gold = stored_oracle(GOLDEN_RMAT26)
    return {
        "workload": spec.name, "n": spec.n, "generated_pairs": spec.num_edges, "m": m, "triangles": T,
        "oracle_T": gold["T"] if gold else None, "matches_oracle": (gold["T"] == T and gold["m"] == m) if gold else None,
        "wedges": info["num_wedges"], "dense_wedges": info["dense_wedges"],
        "build_ms": round(build_ms[-1], 2), "count_ms": round(statistics.mean(count_ms), 3),
        "count_ms_all": [round(x, 3) for x in count_ms], "count_gteps": round(m / t / 1e9, 4),
        "step_gteps": round(m / (t + build_ms[-1] / 1e3) / 1e9, 4), "triangles_per_s": round(T / t, 1),
        "roofline": {"bound": "hbm", "kernel": "k_count", "achieved": round(b_kernel / t / 1e9, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(b_kernel / t / 1e9 / peak, 4),
                     "frac_of_nominal_8tbs": round(b_kernel / t / 8e12, 4), "algorithmic_bytes": b_kernel,
                     "traffic": None,
                     "traffic_note": "DRAM counters are taken only on small captures; the CSR (5 GB) is 40x the L2, "
                                     "so DRAM bytes track the algorithmic bytes less L2 reuse of hub rows"},
        "roofline_id_lists": {"achieved": round(b_ids / t / 1e9, 1), "frac": round(b_ids / t / 1e9 / peak, 4),
                              "algorithmic_bytes": b_ids,
                              "note": "every hop-2 row counted as 4 B per candidate 2-path (4W)"},
        "gpu_launches": int(launches),
    }


def sub_serve(args, dist: Dist) -> dict:
    """The serving workload on a shorter trace (--extra-serve-duration s at --rate) in both modes, then the
    offered-rate sweep."""
    pool = ServePool(args, dist)
    arrivals, pick = pool.trace(args.rate, args.extra_serve_duration)
    out = {"workload": f"Poisson {args.rate:g} req/s for {args.extra_serve_duration:g} s (a shorter trace than the "
                       f"60 s config) over {len(pool.specs)} G(n,p)/R-MAT graphs, sizes log-uniform [1e3, 4e6]",
           "pool_pairs": pool.total_pairs}
    for mode, batching in SERVE_MODES:
        out[mode] = serve_replay(args, pool, arrivals, pick, batching, args.extra_serve_duration * 20 + 300)
    if args.serve_rates:
        out["capacity"] = serve_capacity(args, pool, [float(x) for x in args.serve_rates.split(",")],
                                         args.sweep_duration)
    del pool
    return out


def run_extras(args, dist: Dist, dev, stream, flush) -> dict:
    """The sub-records of the default line: R-MAT 26, per-vertex counts and listing on R-MAT 20, the 4096-graph batch,
    serving.  A failure is reported in its record (and raised again when it is a count mismatch)."""
    import torch
    out = {}
    for name, fn in (("rmat26", lambda: sub_rmat26(args, dev, stream, flush)),
                     ("modes", lambda: sub_modes(args, dev, stream, flush)),
                     ("batch", lambda: batch_measure(args, dist, 10, 3)),
                     ("serve", lambda: sub_serve(args, dist))):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except RuntimeError as e:
            if "differ" in str(e) or "changed" in str(e):
                raise
            out[name] = {"error": str(e)[:300]}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()
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


def cpu_single_thread() -> list:
    """The oracle on one host thread: the ER-4096 graph whole, and R-MAT scale 17 of the R-MAT 20 recipe (edge
    factor 16, noise; one sixteenth of R-MAT 20's merge work), so that the row stays within seconds."""
    import graphgen
    import oracle
    rows = []
    for spec, what in ((graphgen.config("er4096"), "whole ER-4096 graph"),
                       (graphgen.rmat(17, 16, graphgen.BASE_SEED + 1, name="R-MAT scale 17 ef 16"),
                        "R-MAT scale 17 ef 16, the R-MAT 20 recipe at 1/8 of the vertices")):
        hs, hd = spec.edges()
        times = []
        for _ in range(3 if spec.num_edges < (1 << 20) else 1):
            t0 = time.perf_counter()
            T, m = oracle.count(hs, hd, spec.n, threads=1)
            times.append(time.perf_counter() - t0)
        t = min(times)
        rows.append({"value": round(m / t / 1e9, 6), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                     "sample": f"{what} (sort+CSR+merge count), m = {m}, {t:.3f} s"})
    return rows


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


def check_listed(out, T: int, ds, dd, n: int, samples: int = 4096) -> None:
    """Spot check of a listing: a sample of the listed triples are triangles of the input (ascending, distinct,
    every pair an input edge)."""
    import numpy as np
    import torch
    if T == 0:
        return
    sample = out[torch.randint(0, T, (samples,), device=out.device)].cpu().numpy()
    hs, hd = ds.cpu().numpy().astype(np.int64), dd.cpu().numpy().astype(np.int64)
    edges = np.unique(np.minimum(hs, hd) * n + np.maximum(hs, hd))
    t = sample.astype(np.int64)

    def present(x):
        i = np.minimum(np.searchsorted(edges, x), edges.size - 1)
        return edges[i] == x

    ok = (t[:, 0] < t[:, 1]) & (t[:, 1] < t[:, 2])
    ok &= present(t[:, 0] * n + t[:, 1]) & present(t[:, 1] * n + t[:, 2])
    ok &= present(t[:, 0] * n + t[:, 2])
    if not ok.all():
        raise RuntimeError(f"listing differs: {int((~ok).sum())} sampled triples are not triangles")


def sub_modes(args, dev, stream, flush, reps: int = 10) -> dict:
    """The two other outputs of the traversal on the headline graph (R-MAT 20), built once: per-vertex counts t(x)
    (tc_count_per_vertex into device memory; the sum of t must be 3T) and the listing of every triangle
    (tc_list_triangles into device memory; the number found must be T, and sampled triples must be triangles),
    each timed with CUDA events over `reps` calls after one untimed call, the L2 flushed before each."""
    import ctypes

    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    spec = graphgen.config("rmat20")
    ds, dd = spec.edges(device=dev)
    g = tc.tc_load_edges(ds, dd, spec.n, stream=stream)
    try:
        tc.tc_build(g, stream)
        T = tc.tc_count(g, stream)
        pv = torch.empty(spec.n, dtype=torch.int64, device=dev)

        def timed(fn):
            fn()
            ms = []
            for k in range(reps):
                flush.fill_(k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return statistics.median(ms)

        def per_vertex():
            T2, _ = tc.tc_count_per_vertex(g, pv, stream)
            if T2 != T:
                raise RuntimeError(f"per-vertex total {T2} differs from the count {T}")

        pv_ms = timed(per_vertex)
        if int(pv.sum().item()) != 3 * T:
            raise RuntimeError("per-vertex counts differ: their sum is not 3T")
        del pv
        out = torch.empty((max(T, 1), 3), dtype=torch.int32, device=dev)
        lib = tc.load_library()
        found = ctypes.c_uint64()
        sp = ctypes.c_void_p(stream.cuda_stream)

        def list_all():
            st = lib.tc_list_triangles(g, 0, spec.n, out.data_ptr(), T, ctypes.byref(found), tc.TC_PTR_DEVICE, sp)
            if st != tc.TC_OK:
                raise RuntimeError(f"listing: status {st}")
            if found.value != T:
                raise RuntimeError(f"listing differs: found {found.value} of {T}")

        list_ms = timed(list_all)
        check_listed(out, T, ds, dd, spec.n)
        del out
    finally:
        tc.tc_free(g)
    return {"workload": spec.name, "triangles": T, "reps": reps, "per_vertex_ms": round(pv_ms, 4),
            "list_ms": round(list_ms, 4), "list_triangles_per_s": round(T / (list_ms / 1e3), 1),
            "list_output_bytes": 12 * T,
            "note": "per-vertex: tc_count_per_vertex into device memory; listing: both passes of tc_list_triangles "
                    "(ascending original-id triples into device memory); CUDA events, median, L2 flushed before "
                    "each call"}


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
    check_listed(out, T, ds, dd, spec.n)
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
    list_bytes = algorithmic_bytes(info, count_grid(info)) + 16.0 * T
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


def batch_measure(args, dist: Dist, steps: int, warmup: int, clocks=None) -> dict:
    """The 4096-graph mix: every graph built once (CSRs resident), then one step = one replay of the batch plan (one
    persistent launch captured as a CUDA graph) against one graph per launch (tc_count per graph) on the same
    graphs, at identical counts."""
    import numpy as np
    import torch

    import graphgen
    import paper_1909_02127_gb300 as tc

    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream()
    specs = graphgen.batch_mix(args.batch_graphs, graphgen.BASE_SEED + graphgen.BATCH_SEED_OFFSET
                               + dist.rank * 1000003)
    handles = []
    edges = []
    try:
        for sp in specs:
            s, d = sp.edges(device=dev)
            edges.append((s, d, sp.n))
            h = tc.tc_load_edges(s, d, sp.n, stream=stream)
            handles.append(h)
            tc.tc_build(h, stream)
        torch.cuda.synchronize()
        m_total = sum(tc.tc_graph_get_info(h)["num_edges"] for h in handles)
        solo = np.array([tc.tc_count(h, stream) for h in handles], dtype=np.uint64)
        if not np.array_equal(tc.tc_count_batch(handles, stream), solo):
            raise RuntimeError("batched counts differ from one-by-one counts")
        plan = tc.tc_batch_plan_create(handles, stream)  # the launch sequence, captured once as a CUDA graph
        try:
            got = np.zeros(len(handles), dtype=np.uint64)
            for _ in range(warmup):
                tc.tc_batch_plan_run(plan, len(handles), stream, got)
                if not np.array_equal(got, solo):
                    raise RuntimeError("batched counts differ from one-by-one counts")
            dist.barrier()
            torch.cuda.synchronize()
            if clocks:
                clocks.start()
            l0 = tc.tc_kernel_launches()
            t0 = time.perf_counter()
            for _ in range(steps):
                tc.tc_batch_plan_run(plan, len(handles), stream, got)
            torch.cuda.synchronize()
            t_batch = time.perf_counter() - t0
            launches = tc.tc_kernel_launches() - l0
            clock_info = clocks.stop() if clocks else None
            if not np.array_equal(got, solo):
                raise RuntimeError("batched counts differ")
        finally:
            tc.tc_batch_plan_free(plan)
        # one graph per launch, same graphs and counts
        reps = max(1, steps // 2)
        t0 = time.perf_counter()
        for _ in range(reps):
            for h, c in zip(handles, solo):
                if tc.tc_count(h, stream) != int(c):
                    raise RuntimeError("one-by-one count changed")
        t_solo = (time.perf_counter() - t0) / reps
    finally:
        for h in handles:
            tc.tc_free(h)
    pipe = pipeline_measure(edges, solo, stream, max(1, steps // 5))
    del edges
    units, secs = aggregate(len(handles) * steps, t_batch, dist)
    u1, s1 = aggregate(len(handles), t_solo, dist)
    return {"graphs": len(handles), "graphs_per_s": round(units / secs, 2),
            "ms_per_replay": round(t_batch / steps * 1e3, 4), "one_by_one_graphs_per_s": round(u1 / s1, 2),
            "one_by_one_ms": round(t_solo * 1e3, 3), "speedup_vs_one_by_one": round((units / secs) / (u1 / s1), 3),
            "edges": int(m_total), "total_triangles": int(solo.sum()), "steps": steps, "gpu_launches": int(launches),
            "clocks": clock_info, "whole_path": pipe}


def pipeline_measure(edges, solo, stream, reps: int) -> dict:
    """The whole path (ingest + build + count) of every graph from device-resident edges: batched by tc_count_many
    in chunks of at most the compact build's pair limit (each chunk one disjoint union), against one graph at a time
    (tc_load_edges, tc_build, tc_count, tc_free), at identical counts."""
    import numpy as np
    import torch

    import paper_1909_02127_gb300 as tc
    cap = max(1, tc.tc_get_compact_max_pairs())
    chunks, cur, pairs = [], [], 0
    for i, (s, d, n) in enumerate(edges):
        if cur and pairs + s.numel() > cap:
            chunks.append(cur)
            cur, pairs = [], 0
        cur.append(i)
        pairs += s.numel()
    if cur:
        chunks.append(cur)

    def batched():
        return np.concatenate([tc.tc_count_many([edges[i] for i in c], stream) for c in chunks])

    if not np.array_equal(batched(), solo):
        raise RuntimeError("tc_count_many counts differ from one-by-one counts")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        got = batched()
    torch.cuda.synchronize()
    t_many = (time.perf_counter() - t0) / reps
    if not np.array_equal(got, solo):
        raise RuntimeError("tc_count_many counts differ from one-by-one counts")
    t0 = time.perf_counter()
    for (s, d, n), c in zip(edges, solo):
        g = tc.tc_load_edges(s, d, n, stream=stream)
        tc.tc_build(g, stream)
        if tc.tc_count(g, stream) != int(c):
            raise RuntimeError("one-by-one count changed")
        tc.tc_free(g)
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    k = len(edges)
    return {"what": "ingest + build + count of every graph from device-resident edges",
            "batched_graphs_per_s": round(k / t_many, 1), "batched_calls": len(chunks),
            "one_by_one_graphs_per_s": round(k / t_one, 1), "speedup_vs_one_by_one": round(t_one / t_many, 3),
            "reps": reps}


def run_batch(args, dist: Dist):
    import torch
    torch.cuda.set_device(torch.device("cuda", dist.local))
    b = batch_measure(args, dist, args.steps, args.warmup, ClockSampler(dist.local))
    return {
        "metric": "batched graphs/s (4096-graph mix, one persistent launch replayed from a CUDA graph) vs one graph "
                  "per launch",
        "value": b["graphs_per_s"], "unit": "graphs/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_replay"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": {"workload": f"batch of {b['graphs']} graphs (G(n,p)/R-MAT mix, n log-uniform [64, 65536])",
                   "total_triangles": b["total_triangles"], "parallelism": f"replicas x{dist.world}"},
        "one_by_one_graphs_per_s": b["one_by_one_graphs_per_s"],
        "speedup_vs_one_by_one": b["speedup_vs_one_by_one"],
        "e2e": None, "gpu_launches": b["gpu_launches"], "clocks": b["clocks"],
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


class ServePool:
    """The serving workload's request graphs in one page-locked host buffer, with each graph's solo count."""

    def __init__(self, args, dist: Dist):
        import numpy as np
        import torch

        import graphgen
        import paper_1909_02127_gb300 as tc

        dev = torch.device("cuda", dist.local)
        self.specs = graphgen.serve_pool(args.serve_pool,
                                         graphgen.BASE_SEED + graphgen.SERVE_SEED_OFFSET + dist.rank * 7919)
        sizes = []
        chunks = []
        for sp in self.specs:
            s, d = sp.edges(device=dev)
            sizes.append(int(s.numel()))
            chunks.append((s.cpu(), d.cpu()))
        self.sizes = np.array(sizes, dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(self.sizes)])
        total = int(offs[-1])
        self.host = torch.empty(2 * total, dtype=torch.int32).pin_memory()
        for i, (s, d) in enumerate(chunks):
            self.host[offs[i]:offs[i + 1]].copy_(s)
            self.host[total + offs[i]:total + offs[i + 1]].copy_(d)
        del chunks
        base = self.host.data_ptr()
        self.src_ptr = [base + 4 * int(offs[i]) for i in range(len(self.specs))]
        self.dst_ptr = [base + 4 * (total + int(offs[i])) for i in range(len(self.specs))]
        self.total_pairs = total
        self.solo = []
        for i, sp in enumerate(self.specs):
            g = tc.tc_load_edges(self.host[offs[i]:offs[i + 1]], self.host[total + offs[i]:total + offs[i + 1]], sp.n)
            tc.tc_build(g)
            self.solo.append(tc.tc_count(g))
            tc.tc_free(g)

    def trace(self, rate: float, duration: float, seed_offset: int = 0):
        """Poisson arrivals and the pool graph each one requests (even / odd requests alternate kinds)."""
        import graphgen
        arrivals = graphgen.poisson_arrivals(rate, duration, graphgen.BASE_SEED + graphgen.SERVE_SEED_OFFSET - 1
                                             + seed_offset)
        key = graphgen.stream_key(graphgen.BASE_SEED + graphgen.SERVE_SEED_OFFSET - 2 + seed_offset,
                                  graphgen.STREAM_PARAMS)
        half = len(self.specs) // 2
        pick = [2 * (graphgen.draw(key, j) % half) + (j % 2) for j in range(len(arrivals))]
        return arrivals, pick


def serve_replay(args, pool: ServePool, arrivals, pick, batching, deadline_s: float) -> dict:
    """Replay one arrival trace against a server; every result is checked against its graph's solo count.  Latency
    = finish - submission, the host-to-device copy inside it."""
    import threading

    import numpy as np

    import paper_1909_02127_gb300 as tc

    srv = tc.tc_server_create(batching=batching, build_workers=args.build_workers)
    # warm-up before the timed trace (pool growth, first launches of each kernel): every pool graph once, spread
    # over the workers, all results awaited
    warm = list(range(min(len(pool.specs), 256)))
    for k in warm:
        tc.tc_server_submit(srv, pool.src_ptr[k], pool.dst_ptr[k], int(pool.sizes[k]), pool.specs[k].n)
    got = 0
    t_end = time.perf_counter() + 300
    while got < len(warm) and time.perf_counter() < t_end:
        got += len(tc.tc_server_poll(srv, 8192, 50))
    if got < len(warm):
        raise RuntimeError("serve: warm-up requests did not finish")
    stats0 = tc.tc_server_get_stats(srv)
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
        owner[tc.tc_server_submit(srv, pool.src_ptr[k], pool.dst_ptr[k], int(pool.sizes[k]), pool.specs[k].n)] = k
    th.join(timeout=deadline_s)
    done.set()
    th.join()
    stats = tc.tc_server_get_stats(srv)
    tc.tc_server_destroy(srv)
    if len(results) != expected:
        raise RuntimeError(f"serve: {len(results)} of {expected} requests finished")
    bad = [r for r in results if r["status"] != 0 or r["triangles"] != pool.solo[owner[r["id"]]]]
    if bad:
        raise RuntimeError(f"serve: {len(bad)} results differ from their solo counts")
    lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in results])
    span = (max(r["t_done_ns"] for r in results) - min(r["t_submit_ns"] for r in results)) / 1e9
    launches = stats["launches"] - stats0["launches"]
    return {"graphs_per_s": round(expected / span, 2), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "p999_ms": round(float(np.percentile(lat, 99.9)), 3),
            "mean_ms": round(float(lat.mean()), 3), "launches": launches, "max_batch": stats["max_batch_seen"],
            "mean_batch": round((stats["completed"] - stats0["completed"]) / max(1, launches), 2),
            "peak_held_gb": round(stats["peak_held_bytes"] / 1e9, 3), "requests": expected,
            "span_s": round(span, 3)}


# The serving modes compared: the whole path batched (each batch of pending requests ingested, built and counted
# as one disjoint union), the count alone batched, and one graph per launch.
SERVE_MODES = (("batched", "pipeline"), ("count_batched", True), ("one_by_one", False))

# A mode keeps up with an offered rate when it serves at least this share of it and its p99 stays below the cap.
KEEP_UP_SHARE = 0.95
KEEP_UP_P99_MS = 50.0


def serve_capacity(args, pool: ServePool, rates, duration: float) -> dict:
    """The offered-rate sweep: for each rate, the same trace against both modes; the highest rate each mode keeps
    up with."""
    out = {"rates": list(rates), "duration_s": duration, "keep_up": {"share": KEEP_UP_SHARE, "p99_ms": KEEP_UP_P99_MS},
           **{mode: [] for mode, _ in SERVE_MODES}}
    for i, rate in enumerate(rates):
        arrivals, pick = pool.trace(rate, duration, seed_offset=100 + i)
        for mode, batching in SERVE_MODES:
            r = serve_replay(args, pool, arrivals, pick, batching, duration * 20 + 300)
            out[mode].append({"rate": rate, "graphs_per_s": r["graphs_per_s"], "p50_ms": r["p50_ms"],
                              "p99_ms": r["p99_ms"], "mean_batch": r["mean_batch"]})
    for mode, _ in SERVE_MODES:
        ok = [x["rate"] for x in out[mode]
              if x["graphs_per_s"] >= KEEP_UP_SHARE * x["rate"] and x["p99_ms"] <= KEEP_UP_P99_MS]
        out[f"{mode}_max_rate"] = max(ok) if ok else None
    return out


def run_serve(args, dist: Dist):
    """Replay one Poisson arrival trace against the serving loop twice: continuous batching, then one graph per
    launch.  Every result is checked against the graph's solo count."""
    import torch

    import paper_1909_02127_gb300 as tc

    torch.cuda.set_device(torch.device("cuda", dist.local))
    pool = ServePool(args, dist)
    arrivals, pick = pool.trace(args.rate, args.duration)
    clocks = ClockSampler(dist.local, period_s=0.05)
    dist.barrier()
    clocks.start()
    l0 = tc.tc_kernel_launches()
    batched = serve_replay(args, pool, arrivals, pick, "pipeline", args.duration * 20 + 600)
    launches = tc.tc_kernel_launches() - l0
    clock_info = clocks.stop()
    count_batched = serve_replay(args, pool, arrivals, pick, True, args.duration * 20 + 600)
    single = serve_replay(args, pool, arrivals, pick, False, args.duration * 20 + 600)
    units, secs = aggregate(batched["requests"], batched["span_s"], dist)
    out = {
        "metric": "served graphs/s with p50/p99 latency (Poisson arrivals, continuous batching) vs one graph per launch",
        "value": round(units / secs, 2), "unit": "graphs/s", "n_gpus": dist.world, "steps": 1, "warmup": 0,
        "ms_per_step": round(batched["span_s"] * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32/uint64 (exact integer)", "data": "synthetic",
        "config": {"workload": f"Poisson {args.rate:g} req/s for {args.duration:g} s over {len(pool.specs)} "
                               f"G(n,p)/R-MAT graphs, sizes log-uniform [1e3, 4e6]",
                   "pool_pairs": pool.total_pairs, "build_workers": args.build_workers,
                   "parallelism": f"replicas x{dist.world}"},
        "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"], "batched": batched,
        "count_batched": count_batched, "one_by_one": single,
        "speedup_vs_one_by_one": round(batched["graphs_per_s"] / single["graphs_per_s"], 3),
        "e2e": {"value": round(units / secs, 2), "unit": "graphs/s",
                "h2d_bytes_per_step": int(8 * sum(int(pool.sizes[k]) for k in pick)),
                "d2h_bytes_per_step": 8 * len(pick)},
        "gpu_launches": int(launches), "clocks": clock_info,
    }
    if args.serve_rates:
        out["capacity"] = serve_capacity(args, pool, [float(x) for x in args.serve_rates.split(",")],
                                         args.sweep_duration)
    return out


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
