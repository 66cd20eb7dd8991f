"""bench.py's host-side arithmetic on CPU: the algorithmic bytes of one counting pass, the counting grid, and the
rule that ncu traffic is reported only when the summary was taken on the current count-kernel source."""
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


@pytest.mark.parametrize("bins,grid", [({"bin_block": 0, "bin_warp": 0}, 1),
                                       ({"bin_block": 3, "bin_warp": 17, "bin_thread": 513}, 3 + 2 + 2),
                                       ({"bin_block": 10 ** 6, "bin_warp": 0}, 2 * 152)])
def test_count_grid(bins, grid):
    """One CTA per block-bin source, one per 16 warp-bin sources and one per 512 thread-bin sources, at most two
    per SM."""
    assert bench.count_grid(bins) == grid


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
