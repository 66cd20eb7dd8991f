"""bench.py's host-side arithmetic on CPU: the algorithmic bytes of one counting pass, the counting grid, the clock
record, and the rule that ncu traffic is reported only when the summary was taken on the current count-kernel
source."""
import pytest

import bench


def test_algorithmic_bytes_of_one_triangle():
    """K3 oriented 0->1, 0->2, 1->2: n = 3, m = 3 and one candidate 2-path (0->1->2), on one CTA: offsets of every
    source 8(n+1), the rows N+(u) 4m, an offset pair per hop-1 target 16m, the hop-2 ids 4W, one 8-byte atomic."""
    info = {"num_vertices": 3, "num_edges": 3, "num_wedges": 1}
    assert bench.algorithmic_bytes(info, 1) == 8 * 4 + 4 * 3 + 16 * 3 + 4 * 1 + 8


def test_dense_rows_trade_their_ids_for_quads():
    """2-paths through dense rows are read as 16-byte quads instead of 4-byte ids."""
    info = {"num_vertices": 10, "num_edges": 20, "num_wedges": 1000, "dense_wedges": 600, "dense_quads": 7}
    plain = bench.algorithmic_bytes({**info, "dense_wedges": 0, "dense_quads": 0}, 4)
    assert plain - bench.algorithmic_bytes(info, 4) == 4 * 600 - 16 * 7


def test_count_grid_is_the_library_s():
    """The counting grid comes from tc_graph_info.count_ctas (the launch the library makes), not from a copy of its
    arithmetic."""
    assert bench.count_grid({"count_ctas": 7, "bin_block": 10 ** 6}) == 7
    assert bench.count_grid({"count_ctas": 0}) == 1


def test_id_list_bytes_count_every_2path_as_an_id():
    info = {"num_vertices": 10, "num_edges": 20, "num_wedges": 1000, "dense_wedges": 600, "dense_quads": 7}
    assert bench.algorithmic_bytes_ids(info, 4) == bench.algorithmic_bytes(
        {**info, "dense_wedges": 0, "dense_quads": 0}, 4)


def test_clock_summary():
    s = bench.summarize_clocks([(2070.0, 2070.0, []), (1995.0, 2070.0, ["sw_power_cap"]), (2070.0, 2070.0, [])],
                               "test")
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.summarize_clocks([], "test")["samples"] == 0


def test_nvml_reason_bits():
    """The clock-event reason bits of nvml.h map to the names the bench line reports."""
    names = dict(bench._Nvml.REASONS)
    assert names[0x4] == "sw_power_cap" and names[0x8] == "hw_slowdown"
    assert names[0x20] == "sw_thermal_slowdown" and names[0x40] == "hw_thermal_slowdown"


def test_profiled_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1909_02127_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("tc_count.cuh", "tc_count.cu", "tc_internal.cuh", "tc_prims.cuh"):
        (csrc / f).write_text(f"// {f}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.count_kernel_source_hash()
    assert len(sha) == 16
    (tmp_path / "profiles" / "k_count_x.md").write_text(f"source_sha: {sha}\n\ndram_bytes_per_launch: 1.5e+09\n")
    assert bench.profiled_traffic("x") == 1.5e9
    assert bench.profiled_traffic("y") is None  # no summary
    (csrc / "tc_prims.cuh").write_text("// changed\n")
    assert bench.profiled_traffic("x") is None  # taken on another source


def test_listing_spot_check():
    """check_listed accepts the triangles of K4 and rejects a listed triple that is not a triangle of the input."""
    import pytest
    import torch
    src = torch.tensor([0, 0, 0, 1, 1, 2], dtype=torch.int32)
    dst = torch.tensor([1, 2, 3, 2, 3, 3], dtype=torch.int32)
    tri = torch.tensor([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]], dtype=torch.int32)
    bench.check_listed(tri, 4, src, dst, 4, samples=64)
    bench.check_listed(tri[:0], 0, src, dst, 4)
    keep = src != 0
    with pytest.raises(RuntimeError, match="differs"):  # K4 without vertex 0's edges: only (1, 2, 3) remains
        bench.check_listed(tri, 4, src[keep], dst[keep], 4, samples=64)


def test_serving_keep_up_rule(monkeypatch):
    """The capacity sweep's rule: a mode keeps up with a rate when it serves at least 95% of it with p99 at most
    50 ms; its capacity is the highest such rate (None if none).  Replays are faked on the host."""
    import types
    served = {  # (mode's batching, rate) -> (graphs/s, p99 ms)
        ("pipeline", 1000.0): (1000.0, 3.0), ("pipeline", 2000.0): (1990.0, 49.0), ("pipeline", 4000.0): (3000.0, 900.0),
        (True, 1000.0): (999.0, 2.0), (True, 2000.0): (1800.0, 10.0), (True, 4000.0): (2000.0, 10.0),
        (False, 1000.0): (1000.0, 51.0), (False, 2000.0): (2000.0, 60.0), (False, 4000.0): (2100.0, 80.0)}

    class Pool:
        def trace(self, rate, duration, seed_offset=0):
            return [rate], None

    def replay(args, pool, arrivals, pick, batching, timeout):
        gps, p99 = served[(batching, arrivals[0])]
        return {"graphs_per_s": gps, "p50_ms": 1.0, "p99_ms": p99, "mean_batch": 1.0}

    monkeypatch.setattr(bench, "serve_replay", replay)
    out = bench.serve_capacity(types.SimpleNamespace(), Pool(), [1000.0, 2000.0, 4000.0], 2.0)
    assert out["batched_max_rate"] == 2000.0        # 1990/2000 >= 0.95 and p99 49 <= 50; 4000 fails both
    assert out["count_batched_max_rate"] == 1000.0  # 1800/2000 < 0.95
    assert out["one_by_one_max_rate"] is None       # p99 above 50 ms at every rate
    assert [x["rate"] for x in out["batched"]] == [1000.0, 2000.0, 4000.0]


def test_profiled_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The DRAM traffic of a committed count-kernel profile is used only while its recorded source hash is the
    current kernel source's; otherwise the bench reports none."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_count_demo.md").write_text(
        "# demo\n\nsource_sha: 0123456789abcdef\n\ndram_bytes_per_launch: 7.5e+07\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "count_kernel_source_hash", lambda: "0123456789abcdef")
    assert bench.profiled_traffic("demo") == 7.5e7
    monkeypatch.setattr(bench, "count_kernel_source_hash", lambda: "fedcba9876543210")
    assert bench.profiled_traffic("demo") is None
    assert bench.profiled_traffic("absent") is None
