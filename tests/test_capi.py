"""The C-ABI library loads and exports every symbol include/tc.h declares; host-side argument checks (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    with open(os.path.join(ROOT, "include", "tc.h")) as f:
        text = f.read()
    for m in re.finditer(r"TC_API\s+[\w\s\*]+?\b(tc_\w+)\s*\(", text):
        names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1909_02127_gb300 import build
    build.build()
    import paper_1909_02127_gb300 as tc
    return tc.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tc_load_edges", "tc_build", "tc_count", "tc_count_per_vertex", "tc_count_batch", "tc_free"):
        assert required in names


def test_exports_every_declared_symbol(lib):
    import paper_1909_02127_gb300 as tc
    for name in _declared_functions():
        assert hasattr(lib, name), f"libtc.so does not export {name}"
    assert set(_declared_functions()) <= set(tc.EXPORTED)


def test_library_is_built_for_sm103a():
    # the build flags name exactly one target: sm_103a
    from paper_1909_02127_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_argument_errors_without_gpu(lib):
    import paper_1909_02127_gb300 as tc
    out = ctypes.c_void_p()
    # NULL out
    assert lib.tc_load_edges(None, None, 0, 0, tc.TC_PTR_HOST, None, None, None) == tc.TC_ERR_INVALID_ARG
    assert "out is NULL" in tc.tc_last_error()
    # negative sizes
    assert lib.tc_load_edges(None, None, -1, 3, tc.TC_PTR_HOST, None, None, ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_load_edges(None, None, 0, -3, tc.TC_PTR_HOST, None, None, ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    # too many vertices / edges
    assert lib.tc_load_edges(None, None, 0, 1 << 31, tc.TC_PTR_HOST, None, None,
                             ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_load_edges(None, None, (1 << 32) - 1, 5, tc.TC_PTR_HOST, None, None,
                             ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    # bad flags
    assert lib.tc_load_edges(None, None, 0, 3, 0, None, None, ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_load_edges(None, None, 0, 3, 3, None, None, ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    # NULL edge arrays with edges
    assert lib.tc_load_edges(None, None, 5, 3, tc.TC_PTR_HOST, None, None, ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    # edges on an empty vertex set are out of range
    a = (ctypes.c_int32 * 1)(0)
    assert lib.tc_load_edges(a, a, 1, 0, tc.TC_PTR_HOST, None, None, ctypes.byref(out)) == tc.TC_ERR_OUT_OF_RANGE
    assert out.value is None
    # NULL handles
    assert lib.tc_build(None, None) == tc.TC_ERR_INVALID_ARG
    v = ctypes.c_uint64()
    assert lib.tc_count(None, ctypes.byref(v), None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_device(None, None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_per_vertex(None, None, None, tc.TC_PTR_HOST, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_graph_get_info(None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_copy_csr(None, None, None, None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_batch(None, -1, None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_batch(None, 0, None, None) == tc.TC_OK
    lib.tc_free(None)  # no-op
    # serving loop: argument checks that return before any device call
    rid = ctypes.c_uint64()
    assert lib.tc_server_create(None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_server_submit(None, None, None, 0, 0, ctypes.byref(rid)) == tc.TC_ERR_INVALID_ARG
    k = ctypes.c_int32()
    assert lib.tc_server_poll(None, None, 0, 0, ctypes.byref(k)) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_server_get_stats(None, None) == tc.TC_ERR_INVALID_ARG
    lib.tc_server_destroy(None)  # no-op
    plan = ctypes.c_void_p()
    assert lib.tc_batch_plan_create(None, 0, None, ctypes.byref(plan)) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_batch_plan_run(None, None, None) == tc.TC_ERR_INVALID_ARG
    lib.tc_batch_plan_free(None)  # no-op
    # many graphs: argument checks before any device call
    cnt = (ctypes.c_uint64 * 1)()
    assert lib.tc_count_many(None, None, None, None, -1, tc.TC_PTR_HOST, None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_many(None, None, None, None, 1, tc.TC_PTR_HOST, cnt, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_many(None, None, None, None, 0, 3, None, None) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count_many(None, None, None, None, 0, tc.TC_PTR_HOST, None, None) == tc.TC_OK
    ptrs = (ctypes.c_void_p * 1)(None)
    ne = (ctypes.c_int64 * 1)(3)
    nv = (ctypes.c_int64 * 1)(5)
    assert lib.tc_count_many(ptrs, ptrs, ne, nv, 1, tc.TC_PTR_HOST, cnt, None) == tc.TC_ERR_INVALID_ARG  # NULL arrays
    nv0 = (ctypes.c_int64 * 1)(0)
    arr = (ctypes.c_int32 * 3)(0, 1, 2)
    aptr = (ctypes.c_void_p * 1)(ctypes.addressof(arr))
    assert lib.tc_count_many(aptr, aptr, ne, nv0, 1, tc.TC_PTR_HOST, cnt, None) == tc.TC_ERR_OUT_OF_RANGE


def test_missing_library_fails_loudly(tmp_path):
    import paper_1909_02127_gb300 as tc
    saved = tc._lib
    try:
        tc._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            tc.load_library(str(tmp_path / "nope.so"))
    finally:
        tc._lib = saved


def test_tuning_table_round_trip_without_gpu(lib):
    import paper_1909_02127_gb300 as tc
    saved = tc.tc_get_tuning()
    try:
        tc.tc_set_tuning([(1000, 5), (1 << 40, 1 << 15)])
        assert tc.tc_get_tuning() == [(1000, 5), (1 << 40, 1 << 15)]
        with pytest.raises(tc.TCError):
            tc.tc_set_tuning([(1000, 5), (10, 7)])  # bounds not ascending
        with pytest.raises(tc.TCError):
            tc.tc_set_tuning([(1000, -1)])
        assert tc.tc_get_tuning() == [(1000, 5), (1 << 40, 1 << 15)]
        ratio = tc.tc_get_isect_max_wedges_milli()
        tc.tc_set_tuning([(1 << 40, 1 << 15)], isect_max_wedges_milli=2500)
        assert tc.tc_get_isect_max_wedges_milli() == 2500
        with pytest.raises(tc.TCError):
            tc.tc_set_tuning([(1 << 40, 1 << 15)], isect_max_wedges_milli=-1)
        tc.tc_set_tuning([(1 << 40, 1 << 15)], isect_max_wedges_milli=ratio)
        # per-vertex counters without read-back: only below 2^31 edges, where no counter can reach 2^32
        assert tc.tc_get_vertex_plain_max_edges() == tc.VERTEX_PLAIN_MAX_EDGES == (1 << 31) - 1
        tc.tc_set_tuning(tc.tc_get_tuning(), vertex_plain_max_edges=0)
        assert tc.tc_get_vertex_plain_max_edges() == 0
        for bad in (-1, 1 << 31):
            with pytest.raises(tc.TCError):
                tc.tc_set_tuning(tc.tc_get_tuning(), vertex_plain_max_edges=bad)
        assert tc.tc_get_vertex_plain_max_edges() == 0
        tc.tc_set_tuning(tc.tc_get_tuning(), vertex_plain_max_edges=tc.VERTEX_PLAIN_MAX_EDGES)
    finally:
        tc.tc_set_tuning(saved, vertex_plain_max_edges=tc.VERTEX_PLAIN_MAX_EDGES)


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor in the binding's argument checks (no GPU here)."""

    def __init__(self, numel, element_size=8, contiguous=True, is_cuda=True):
        self._numel, self._es, self._contig, self.is_cuda = numel, element_size, contiguous, is_cuda

    def numel(self):
        return self._numel

    def element_size(self):
        return self._es

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return 0x1000


def test_noalloc_binding_rejects_bad_outputs_before_any_launch(monkeypatch):
    """tc_count_per_vertex_noalloc checks its output tensors in Python (CUDA, 8-byte, contiguous, at least n and
    1 entries) and raises ValueError without calling into the library; raw ints pass through."""
    import torch

    import paper_1909_02127_gb300 as tc
    calls = []

    class FakeLib:
        def tc_count_per_vertex_noalloc(self, *args):
            calls.append(args)
            return tc.TC_OK

    monkeypatch.setattr(tc, "load_library", lambda *a, **k: FakeLib())
    monkeypatch.setattr(tc, "tc_graph_get_info", lambda g: {"num_vertices": 10})
    monkeypatch.setattr(tc, "_stream_ptr", lambda s: 0)
    ok_pv, ok_tot = _FakeDeviceTensor(10), _FakeDeviceTensor(1)
    bad = [
        (torch.zeros(10, dtype=torch.int64), ok_tot),          # host tensor
        (_FakeDeviceTensor(9), ok_tot),                        # shorter than n
        (_FakeDeviceTensor(10, element_size=4), ok_tot),       # 32-bit entries
        (_FakeDeviceTensor(10, contiguous=False), ok_tot),     # strided
        (ok_pv, _FakeDeviceTensor(0)),                         # no room for T
        (ok_pv, torch.zeros(1, dtype=torch.int64)),            # host total
    ]
    for pv, tot in bad:
        with pytest.raises(ValueError):
            tc.tc_count_per_vertex_noalloc(1, pv, tot)
    assert calls == []
    tc.tc_count_per_vertex_noalloc(1, ok_pv, ok_tot)
    tc.tc_count_per_vertex_noalloc(1, 0x2000, 0x3000)  # raw device addresses: the caller vouches for them
    assert len(calls) == 2


def test_tuning_file_applies_only_on_its_device(lib, tmp_path, monkeypatch):
    """tuning.json is installed only when its device name and SM count match the current GPU (faked here: no GPU),
    keeps the fields it does not name, and leaves the table alone otherwise."""
    import json
    import types

    import torch

    import paper_1909_02127_gb300 as tc
    saved = tc.tc_get_tuning()
    saved_tiny = tc.tc_get_tiny_max_pairs()
    whole = tc.tc_tuning()
    assert lib.tc_get_tuning(ctypes.byref(whole)) == tc.TC_OK
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps({"device": "Fake GPU", "sms": 7, "classes": [[1000, 11], [1 << 40, 22]],
                                "compact_max_pairs": 12345}))
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    try:
        monkeypatch.setattr(torch.cuda, "get_device_properties",
                            lambda i: types.SimpleNamespace(name="Other GPU", multi_processor_count=7))
        assert not tc._apply_tuning_file(lib, str(path))
        assert tc.tc_get_tuning() == saved
        monkeypatch.setattr(torch.cuda, "get_device_properties",
                            lambda i: types.SimpleNamespace(name="Fake GPU", multi_processor_count=7))
        assert tc._apply_tuning_file(lib, str(path))
        assert tc.tc_get_tuning() == [(1000, 11), (1 << 40, 22)]
        assert tc.tc_get_compact_max_pairs() == 12345
        assert tc.tc_get_tiny_max_pairs() == saved_tiny                     # not in the file: kept
        assert tc.tc_get_isect_max_wedges_milli() == whole.isect_max_wedges_milli
        assert tc.tc_get_vertex_plain_max_edges() == tc.VERTEX_PLAIN_MAX_EDGES
    finally:
        assert lib.tc_set_tuning(ctypes.byref(whole)) == tc.TC_OK
