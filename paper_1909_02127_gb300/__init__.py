"""Python binding of libtc, the GB300 exact triangle counter (Wang & Owens, "Fast BFS-Based Triangle Counting on
GPUs", HPEC 2019).

Argument marshalling only: every step of the computation runs in the CUDA kernels of ``csrc/`` behind the C ABI of
``include/tc.h``.  The functions carry the C names.  PyTorch supplies streams and, on request (allocator="torch"),
device memory through the allocator hook; by default the library's own stream-ordered pool is used.  There is no
CPU fallback: if ``libtc.so`` is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TC_OK, TC_ERR_INVALID_ARG, TC_ERR_OUT_OF_RANGE, TC_ERR_NO_MEMORY, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_INTERNAL, \
    TC_ERR_STATE = range(8)
TC_PTR_HOST, TC_PTR_DEVICE = 1, 2
STATUS_NAMES = ["TC_OK", "TC_ERR_INVALID_ARG", "TC_ERR_OUT_OF_RANGE", "TC_ERR_NO_MEMORY", "TC_ERR_CUDA",
                "TC_ERR_TIMEOUT", "TC_ERR_INTERNAL", "TC_ERR_STATE"]


class TCError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {message}")


class tc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)),
                ("ctx", ctypes.c_void_p)]


class tc_graph_info(ctypes.Structure):
    _fields_ = [("num_vertices", ctypes.c_int64), ("num_input_pairs", ctypes.c_int64), ("num_edges", ctypes.c_int64),
                ("csr_entries", ctypes.c_int64), ("max_out_degree", ctypes.c_int64), ("num_wedges", ctypes.c_int64),
                ("active_sources", ctypes.c_int64), ("bin_warp", ctypes.c_int64), ("bin_block", ctypes.c_int64),
                ("built", ctypes.c_int32), ("count_ctas", ctypes.c_int32), ("dense_rows", ctypes.c_int64),
                ("dense_wedges", ctypes.c_int64), ("dense_quads", ctypes.c_int64), ("bin_thread", ctypes.c_int64)]


TC_TUNING_MAX_CLASSES = 16
TINY_MAX_VERTICES = 1 << 14          # the one-launch build: at most this many vertices
TINY_MAX_PAIRS = (1 << 18) - 1       # and fewer than 2^18 input pairs
VERTEX_PLAIN_MAX_EDGES = (1 << 31) - 1  # per-vertex counters without read-back up to this many edges


class tc_tuning(ctypes.Structure):
    _fields_ = [("num_classes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("batch_warp_max_edges", ctypes.c_int64),
                ("class_max_edges", ctypes.c_int64 * TC_TUNING_MAX_CLASSES),
                ("block_min_work", ctypes.c_int64 * TC_TUNING_MAX_CLASSES),
                ("isect_max_wedges_milli", ctypes.c_int64), ("bucket_max_pairs", ctypes.c_int64),
                ("compact_max_pairs", ctypes.c_int64), ("stage_min_csr_bytes", ctypes.c_int64),
                ("tiny_max_pairs", ctypes.c_int64), ("vertex_plain_max_edges", ctypes.c_int64)]


class tc_server_config(ctypes.Structure):
    _fields_ = [("build_workers", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("batching", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("hbm_reserve_bytes", ctypes.c_int64),
                ("hbm_budget_bytes", ctypes.c_int64)]


class tc_request_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("triangles", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_built_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


class tc_prune_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("rounds", "edges_removed", "vertices_removed", "reserved")]


class tc_unfused_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("candidates", "frontier1", "partials", "frontier2", "matches",
                                                    "chunks", "peak_bytes", "reserved")]


class tc_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("submitted", "admitted", "completed", "failed", "launches",
                                                    "max_batch_seen", "budget_bytes", "held_bytes",
                                                    "peak_held_bytes", "pending")]


EXPORTED = ["tc_load_edges", "tc_build", "tc_build_pruned", "tc_count", "tc_count_device", "tc_count_per_vertex",
            "tc_count_per_vertex_noalloc", "tc_list_triangles", "tc_count_unfused", "tc_count_intersect", "tc_count_batch", "tc_server_create", "tc_server_submit",
            "tc_server_poll", "tc_server_get_stats", "tc_server_destroy", "tc_batch_plan_create",
            "tc_batch_plan_run", "tc_batch_plan_free",
            "tc_graph_get_info", "tc_copy_csr", "tc_free", "tc_last_error", "tc_kernel_launches", "tc_set_tuning",
            "tc_get_tuning", "tc_count_many"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtc.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c 'import __graft_entry__ as g;"
                           " g.build()')")
    lib = ctypes.CDLL(path)
    vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    st = ctypes.c_int
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.tc_load_edges.argtypes = [vp, vp, i64, i64, u32, ctypes.POINTER(tc_allocator), vp, ctypes.POINTER(vp)]
    lib.tc_load_edges.restype = st
    lib.tc_build.argtypes = [vp, vp]
    lib.tc_build.restype = st
    lib.tc_build_pruned.argtypes = [vp, i32, ctypes.POINTER(tc_prune_stats), vp]
    lib.tc_build_pruned.restype = st
    lib.tc_count.argtypes = [vp, u64p, vp]
    lib.tc_count.restype = st
    lib.tc_count_device.argtypes = [vp, vp, vp]
    lib.tc_count_device.restype = st
    lib.tc_count_per_vertex.argtypes = [vp, vp, u64p, u32, vp]
    lib.tc_count_per_vertex.restype = st
    lib.tc_list_triangles.argtypes = [vp, i64, i64, vp, i64, u64p, u32, vp]
    lib.tc_list_triangles.restype = st
    lib.tc_count_unfused.argtypes = [vp, u64p, i64, ctypes.POINTER(tc_unfused_stats), vp]
    lib.tc_count_unfused.restype = st
    lib.tc_count_intersect.argtypes = [vp, u64p, vp]
    lib.tc_count_intersect.restype = st
    lib.tc_count_per_vertex_noalloc.argtypes = [vp, vp, vp, vp]
    lib.tc_count_per_vertex_noalloc.restype = st
    lib.tc_count_batch.argtypes = [ctypes.POINTER(vp), i32, u64p, vp]
    lib.tc_count_batch.restype = st
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.tc_count_many.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i64p, i64p, i32, u32, u64p, vp]
    lib.tc_count_many.restype = st
    lib.tc_graph_get_info.argtypes = [vp, ctypes.POINTER(tc_graph_info)]
    lib.tc_graph_get_info.restype = st
    lib.tc_copy_csr.argtypes = [vp, vp, vp, vp, vp]
    lib.tc_copy_csr.restype = st
    lib.tc_free.argtypes = [vp]
    lib.tc_free.restype = None
    lib.tc_server_create.argtypes = [ctypes.POINTER(tc_server_config), ctypes.POINTER(vp)]
    lib.tc_server_create.restype = st
    lib.tc_server_submit.argtypes = [vp, vp, vp, i64, i64, ctypes.POINTER(ctypes.c_uint64)]
    lib.tc_server_submit.restype = st
    lib.tc_server_poll.argtypes = [vp, ctypes.POINTER(tc_request_result), i32, i32, ctypes.POINTER(i32)]
    lib.tc_server_poll.restype = st
    lib.tc_server_get_stats.argtypes = [vp, ctypes.POINTER(tc_server_stats)]
    lib.tc_server_get_stats.restype = st
    lib.tc_server_destroy.argtypes = [vp]
    lib.tc_server_destroy.restype = None
    lib.tc_batch_plan_create.argtypes = [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)]
    lib.tc_batch_plan_create.restype = st
    lib.tc_batch_plan_run.argtypes = [vp, u64p, vp]
    lib.tc_batch_plan_run.restype = st
    lib.tc_batch_plan_free.argtypes = [vp]
    lib.tc_batch_plan_free.restype = None
    lib.tc_set_tuning.argtypes = [ctypes.POINTER(tc_tuning)]
    lib.tc_set_tuning.restype = st
    lib.tc_get_tuning.argtypes = [ctypes.POINTER(tc_tuning)]
    lib.tc_get_tuning.restype = st
    lib.tc_kernel_launches.argtypes = []
    lib.tc_kernel_launches.restype = ctypes.c_uint64
    lib.tc_last_error.argtypes = []
    lib.tc_last_error.restype = ctypes.c_char_p
    _lib = lib
    _apply_tuning_file(lib)
    return lib


TUNING_FILE = os.path.join(_HERE, "tuning.json")


def _apply_tuning_file(lib, path: str = TUNING_FILE) -> bool:
    """Install the autotuner's table when it was measured on this kind of device (name and SM count match); a field
    the file does not name keeps its current value."""
    if not os.path.exists(path):
        return False
    try:
        import json
        import torch
        if not torch.cuda.is_available():
            return False
        with open(path) as f:
            data = json.load(f)
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        if data.get("device") != props.name or int(data.get("sms", -1)) != props.multi_processor_count:
            return False
        cur = tc_tuning()
        lib.tc_get_tuning(ctypes.byref(cur))
        t = _tuning_struct(data["classes"], data.get("batch_warp_max_edges", cur.batch_warp_max_edges),
                           data.get("isect_max_wedges_milli", cur.isect_max_wedges_milli),
                           data.get("bucket_max_pairs", cur.bucket_max_pairs),
                           data.get("compact_max_pairs", cur.compact_max_pairs),
                           data.get("stage_min_csr_bytes", cur.stage_min_csr_bytes),
                           data.get("tiny_max_pairs", cur.tiny_max_pairs), cur.vertex_plain_max_edges)
        return lib.tc_set_tuning(ctypes.byref(t)) == TC_OK
    except Exception:
        return False


def _tuning_struct(classes, batch_warp_max_edges: int = 1 << 25, isect_max_wedges_milli: int = 0,
                   bucket_max_pairs: int = 1 << 29, compact_max_pairs: int = 1 << 25,
                   stage_min_csr_bytes: int = 4 << 30, tiny_max_pairs: int = TINY_MAX_PAIRS,
                   vertex_plain_max_edges: int = VERTEX_PLAIN_MAX_EDGES) -> "tc_tuning":
    t = tc_tuning()
    t.num_classes = len(classes)
    t.batch_warp_max_edges = int(batch_warp_max_edges)
    t.isect_max_wedges_milli = int(isect_max_wedges_milli)
    t.bucket_max_pairs = int(bucket_max_pairs)
    t.compact_max_pairs = int(compact_max_pairs)
    t.stage_min_csr_bytes = int(stage_min_csr_bytes)
    t.tiny_max_pairs = int(tiny_max_pairs)
    t.vertex_plain_max_edges = int(vertex_plain_max_edges)
    for i, (max_edges, work) in enumerate(classes):
        t.class_max_edges[i] = int(max_edges)
        t.block_min_work[i] = int(work)
    return t


def tc_set_tuning(classes, batch_warp_max_edges: Optional[int] = None,
                  isect_max_wedges_milli: Optional[int] = None, bucket_max_pairs: Optional[int] = None,
                  compact_max_pairs: Optional[int] = None, stage_min_csr_bytes: Optional[int] = None,
                  tiny_max_pairs: Optional[int] = None, vertex_plain_max_edges: Optional[int] = None) -> None:
    """classes: [(max_edges, block_min_work), ...] with ascending max_edges; batch_warp_max_edges,
    isect_max_wedges_milli, bucket_max_pairs, compact_max_pairs, stage_min_csr_bytes, tiny_max_pairs and
    vertex_plain_max_edges: keep the current values if None."""
    if not 1 <= len(classes) <= TC_TUNING_MAX_CLASSES:
        raise ValueError("1..16 classes")
    cur = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(cur)))
    if batch_warp_max_edges is None:
        batch_warp_max_edges = cur.batch_warp_max_edges
    if isect_max_wedges_milli is None:
        isect_max_wedges_milli = cur.isect_max_wedges_milli
    if bucket_max_pairs is None:
        bucket_max_pairs = cur.bucket_max_pairs
    if compact_max_pairs is None:
        compact_max_pairs = cur.compact_max_pairs
    if stage_min_csr_bytes is None:
        stage_min_csr_bytes = cur.stage_min_csr_bytes
    if tiny_max_pairs is None:
        tiny_max_pairs = cur.tiny_max_pairs
    if vertex_plain_max_edges is None:
        vertex_plain_max_edges = cur.vertex_plain_max_edges
    t = _tuning_struct(classes, batch_warp_max_edges, isect_max_wedges_milli, bucket_max_pairs, compact_max_pairs,
                       stage_min_csr_bytes, tiny_max_pairs, vertex_plain_max_edges)
    _check(load_library().tc_set_tuning(ctypes.byref(t)))


def tc_get_tuning():
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return [(int(t.class_max_edges[i]), int(t.block_min_work[i])) for i in range(t.num_classes)]


def tc_get_stage_min_csr_bytes() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.stage_min_csr_bytes)


def tc_get_tiny_max_pairs() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.tiny_max_pairs)


def tc_get_vertex_plain_max_edges() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.vertex_plain_max_edges)


def tc_get_compact_max_pairs() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.compact_max_pairs)


def tc_get_bucket_max_pairs() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.bucket_max_pairs)


def tc_get_isect_max_wedges_milli() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.isect_max_wedges_milli)


def tc_get_batch_warp_max_edges() -> int:
    t = tc_tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return int(t.batch_warp_max_edges)


def _check(status: int):
    if status != TC_OK:
        raise TCError(status, load_library().tc_last_error().decode(errors="replace"))


def tc_kernel_launches() -> int:
    return int(load_library().tc_kernel_launches())


def tc_last_error() -> str:
    return load_library().tc_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------------------------------------------
# Streams and the torch allocator hook
# ---------------------------------------------------------------------------------------------------------------
def _stream_ptr(stream) -> Optional[int]:
    """A torch.cuda.Stream, a raw cudaStream_t (int) or None (torch's current stream)."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _TorchAllocator:
    """Device memory from torch's caching allocator, handed to libtc through tc_allocator."""

    def __init__(self):
        self.live = {}
        self.allocations = 0  # number of alloc callbacks served (diagnostic)
        self._alloc = tc_allocator._fields_[0][1](self._do_alloc)
        self._free = tc_allocator._fields_[1][1](self._do_free)
        self.struct = tc_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, stream, ctx):
        try:
            import torch
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            p = t.data_ptr()
            self.live[p] = (t, stream)
            self.allocations += 1
            return p
        except Exception:
            return None

    def _do_free(self, ptr, stream, ctx):
        entry = self.live.pop(ptr, None)
        if entry is None:
            return
        t, s0 = entry
        if stream and stream != s0:
            import torch
            t.record_stream(torch.cuda.ExternalStream(stream))
        del t


_torch_alloc = None


def torch_allocator() -> _TorchAllocator:
    global _torch_alloc
    if _torch_alloc is None:
        _torch_alloc = _TorchAllocator()
    return _torch_alloc


# ---------------------------------------------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------------------------------------------
def _edge_ptrs(src, dst):
    """Returns (src_ptr, dst_ptr, num_edges, flags, keepalive)."""
    try:
        import torch
        is_t = isinstance(src, torch.Tensor)
    except ImportError:
        is_t = False
    if is_t:
        if src.dtype != torch.int32 or dst.dtype != torch.int32:
            raise TypeError("edge tensors must be int32")
        if src.shape != dst.shape or src.dim() != 1:
            raise ValueError("src and dst must be 1-D and the same length")
        src, dst = src.contiguous(), dst.contiguous()
        flags = TC_PTR_DEVICE if src.is_cuda else TC_PTR_HOST
        if src.is_cuda != dst.is_cuda:
            raise ValueError("src and dst must both be on the host or both on the device")
        return src.data_ptr(), dst.data_ptr(), src.numel(), flags, (src, dst)
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    if s.shape != d.shape or s.ndim != 1:
        raise ValueError("src and dst must be 1-D and the same length")
    return s.ctypes.data, d.ctypes.data, s.size, TC_PTR_HOST, (s, d)


def tc_load_edges(src, dst, num_vertices: int, stream=None, allocator=None) -> int:
    """Load the undirected pairs (src[i], dst[i]) of a graph on [0, num_vertices); returns a tc_graph handle.
    allocator: None (the library's per-device stream-ordered pool) or "torch" (torch's caching allocator, through
    a callback per allocation)."""
    lib = load_library()
    sp, dp, m, flags, keep = _edge_ptrs(src, dst)
    alloc = ctypes.byref(torch_allocator().struct) if allocator == "torch" else None
    out = ctypes.c_void_p()
    _check(lib.tc_load_edges(sp, dp, m, num_vertices, flags, alloc, _stream_ptr(stream), ctypes.byref(out)))
    del keep
    return out.value


def tc_build(g: int, stream=None) -> None:
    _check(load_library().tc_build(g, _stream_ptr(stream)))


def tc_build_pruned(g: int, max_rounds: int = 0, stream=None) -> dict:
    """tc_build on the 2-core (max_rounds = 0) or after max_rounds rounds of the NE filter; returns what was
    removed."""
    st = tc_prune_stats()
    _check(load_library().tc_build_pruned(g, int(max_rounds), ctypes.byref(st), _stream_ptr(stream)))
    return {name: int(getattr(st, name)) for name, _ in tc_prune_stats._fields_ if name != "reserved"}


def tc_count(g: int, stream=None) -> int:
    out = ctypes.c_uint64(0)
    _check(load_library().tc_count(g, ctypes.byref(out), _stream_ptr(stream)))
    return int(out.value)


def tc_count_device(g: int, d_total, stream=None) -> None:
    """Asynchronous count into the device word d_total (a torch tensor with at least 8 bytes, or a pointer)."""
    ptr = d_total if isinstance(d_total, int) else d_total.data_ptr()
    _check(load_library().tc_count_device(g, ptr, _stream_ptr(stream)))


def tc_count_per_vertex(g: int, out=None, stream=None):
    """Returns (T, t): t is `out` if given (uint64/int64 numpy array or CUDA tensor of n entries) else a new numpy
    uint64 array."""
    lib = load_library()
    n = tc_graph_get_info(g)["num_vertices"]
    if out is None:
        out = np.zeros(n, dtype=np.uint64)
    total = ctypes.c_uint64(0)
    if isinstance(out, np.ndarray):
        if out.dtype not in (np.uint64, np.int64) or out.size < n or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous 64-bit array of n entries")
        _check(lib.tc_count_per_vertex(g, out.ctypes.data, ctypes.byref(total), TC_PTR_HOST, _stream_ptr(stream)))
    else:
        if out.element_size() != 8 or out.numel() < n or not out.is_contiguous():
            raise ValueError("out must be a contiguous 64-bit tensor of n entries")
        flags = TC_PTR_DEVICE if out.is_cuda else TC_PTR_HOST
        _check(lib.tc_count_per_vertex(g, out.data_ptr(), ctypes.byref(total), flags, _stream_ptr(stream)))
    return int(total.value), out


def _device_words(t, need: int, what: str) -> int:
    """Address of a CUDA tensor that holds at least `need` contiguous 64-bit entries (ValueError otherwise)."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor (or a raw device address as an int)")
    if t.element_size() != 8 or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous tensor of 64-bit entries")
    if t.numel() < need:
        raise ValueError(f"{what} holds {t.numel()} entries; {need} are needed")
    return t.data_ptr()


def tc_count_per_vertex_noalloc(g: int, d_per_vertex, d_total, stream=None) -> None:
    """Per-vertex counts into caller-provided DEVICE memory, allocating nothing (scratch is a static device array
    of 2^20 entries; larger graphs are rejected).  d_per_vertex: a CUDA tensor of at least n 64-bit entries;
    d_total: a CUDA tensor of at least one 64-bit entry.  Both are checked here (ValueError before any launch);
    raw device addresses given as ints are passed through unchecked, and then the caller vouches for their size.
    Asynchronous on `stream`."""
    if isinstance(d_per_vertex, int) and isinstance(d_total, int):
        pv, tot = d_per_vertex, d_total
    else:
        n = tc_graph_get_info(g)["num_vertices"]
        pv = d_per_vertex if isinstance(d_per_vertex, int) else _device_words(d_per_vertex, n, "d_per_vertex")
        tot = d_total if isinstance(d_total, int) else _device_words(d_total, 1, "d_total")
    _check(load_library().tc_count_per_vertex_noalloc(g, pv, tot, _stream_ptr(stream)))


def tc_list_triangles(g: int, first_source: int = 0, num_sources: Optional[int] = None, capacity: Optional[int] = None,
                      stream=None):
    """Triangles whose first vertex (in the visiting order) has rank in [first_source, first_source+num_sources),
    as an int32 array of shape (k, 3) of ascending original ids, and the number found (which exceeds k when the
    capacity was too small).  capacity defaults to the graph's triangle count."""
    lib = load_library()
    n = tc_graph_get_info(g)["num_vertices"]
    if num_sources is None:
        num_sources = n - first_source
    if capacity is None:
        capacity = tc_count(g, stream)
    out = np.zeros((max(int(capacity), 1), 3), dtype=np.int32)
    found = ctypes.c_uint64(0)
    _check(lib.tc_list_triangles(g, first_source, num_sources, out.ctypes.data, int(capacity), ctypes.byref(found),
                                 TC_PTR_HOST, _stream_ptr(stream)))
    k = min(int(found.value), int(capacity))
    return out[:k], int(found.value)


def tc_count_intersect(g: int, stream=None) -> int:
    """T by segmented intersection (one lane per oriented edge)."""
    out = ctypes.c_uint64(0)
    _check(load_library().tc_count_intersect(g, ctypes.byref(out), _stream_ptr(stream)))
    return int(out.value)


def tc_count_unfused(g: int, max_chunk_bytes: int = 0, stream=None):
    """T by the unfused verification loop (materialised frontiers), and its frontier sizes as a dict."""
    lib = load_library()
    T = ctypes.c_uint64(0)
    st = tc_unfused_stats()
    _check(lib.tc_count_unfused(g, ctypes.byref(T), int(max_chunk_bytes), ctypes.byref(st), _stream_ptr(stream)))
    return int(T.value), {name: int(getattr(st, name)) for name, _ in tc_unfused_stats._fields_ if name != "reserved"}


def tc_count_batch(gs: Sequence[int], stream=None) -> np.ndarray:
    lib = load_library()
    arr = (ctypes.c_void_p * len(gs))(*gs)
    out = np.zeros(len(gs), dtype=np.uint64)
    _check(lib.tc_count_batch(arr, len(gs), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              _stream_ptr(stream)))
    return out


def tc_count_many(graphs, stream=None) -> np.ndarray:
    """Triangle counts of several graphs counted as one pipeline (their disjoint union built once).  graphs: a
    sequence of (src, dst, num_vertices) with src/dst int32 numpy arrays (host) or CUDA tensors (device), all of one
    kind.  Returns a uint64 array of the counts."""
    lib = load_library()
    k = len(graphs)
    keep, sp, dp = [], [], []
    flags = None
    for src, dst, _ in graphs:
        s_, d_, m, f, kp = _edge_ptrs(src, dst)
        if flags is not None and f != flags:
            raise ValueError("all graphs' arrays must be on the host, or all on the device")
        flags = f
        keep.append(kp)
        sp.append(s_)
        dp.append(d_)
    ne = np.array([len(g[0]) for g in graphs], dtype=np.int64)
    nv = np.array([int(g[2]) for g in graphs], dtype=np.int64)
    out = np.zeros(k, dtype=np.uint64)
    if k == 0:
        return out
    arr_s = (ctypes.c_void_p * k)(*sp)
    arr_d = (ctypes.c_void_p * k)(*dp)
    i64p = ctypes.POINTER(ctypes.c_int64)
    _check(lib.tc_count_many(arr_s, arr_d, ne.ctypes.data_as(i64p), nv.ctypes.data_as(i64p), k, flags,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _stream_ptr(stream)))
    del keep
    return out


def tc_batch_plan_create(gs: Sequence[int], stream=None) -> int:
    arr = (ctypes.c_void_p * len(gs))(*gs)
    out = ctypes.c_void_p()
    _check(load_library().tc_batch_plan_create(arr, len(gs), _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def tc_batch_plan_run(plan: int, num_graphs: int, stream=None, out: Optional[np.ndarray] = None) -> np.ndarray:
    if out is None:
        out = np.zeros(num_graphs, dtype=np.uint64)
    _check(load_library().tc_batch_plan_run(plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                            _stream_ptr(stream)))
    return out


def tc_batch_plan_free(plan: int) -> None:
    if plan:
        load_library().tc_batch_plan_free(plan)


def tc_graph_get_info(g: int) -> dict:
    info = tc_graph_info()
    _check(load_library().tc_graph_get_info(g, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in tc_graph_info._fields_}


def tc_copy_csr(g: int, stream=None):
    """Returns (offsets, cols, perm): the oriented CSR in rank space (rows padded to multiples of 4 with n) and
    perm[r] = original id of rank r."""
    info = tc_graph_get_info(g)
    n = info["num_vertices"]
    off = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(info["csr_entries"], 1), dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    _check(load_library().tc_copy_csr(g, off.ctypes.data, col.ctypes.data, perm.ctypes.data, _stream_ptr(stream)))
    return off, col[: info["csr_entries"]], perm[:n]


def tc_free(g: int) -> None:
    if g:
        load_library().tc_free(g)


def tc_server_create(build_workers: int = 4, max_batch: int = 4096, batching=True, max_inflight: int = 8192,
                     hbm_reserve_bytes: int = -1, hbm_budget_bytes: int = 0) -> int:
    """batching: True / 1 batches the count, 2 (or "pipeline") the whole path, False / 0 neither."""
    mode = 2 if batching == "pipeline" else int(batching)
    cfg = tc_server_config(build_workers, max_batch, mode, max_inflight, hbm_reserve_bytes, hbm_budget_bytes)
    out = ctypes.c_void_p()
    _check(load_library().tc_server_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def tc_server_submit(s: int, src_ptr: int, dst_ptr: int, num_edges: int, num_vertices: int) -> int:
    """Raw submit: src_ptr/dst_ptr are host addresses that must stay valid until the result is polled (the Server
    class keeps them alive)."""
    rid = ctypes.c_uint64(0)
    _check(load_library().tc_server_submit(s, src_ptr, dst_ptr, num_edges, num_vertices, ctypes.byref(rid)))
    return int(rid.value)


def tc_server_poll(s: int, max_results: int = 4096, timeout_ms: int = 0):
    buf = (tc_request_result * max(1, max_results))()
    k = ctypes.c_int32(0)
    _check(load_library().tc_server_poll(s, buf, max_results, timeout_ms, ctypes.byref(k)))
    return [{name: getattr(buf[i], name) for name, _ in tc_request_result._fields_} for i in range(k.value)]


def tc_server_get_stats(s: int) -> dict:
    st = tc_server_stats()
    _check(load_library().tc_server_get_stats(s, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in tc_server_stats._fields_}


def tc_server_destroy(s: int) -> None:
    if s:
        load_library().tc_server_destroy(s)


class Server:
    """Owning wrapper over a tc_server: submit(src, dst, n) with host arrays (kept alive until their result is
    polled), poll(), stats(), close()."""

    def __init__(self, **cfg):
        self.handle = tc_server_create(**cfg)
        self._keep = {}

    def submit(self, src, dst, num_vertices: int) -> int:
        sp, dp, m, flags, keep = _edge_ptrs(src, dst)
        if flags != TC_PTR_HOST:
            raise ValueError("server requests take host arrays")
        rid = tc_server_submit(self.handle, sp, dp, m, num_vertices)
        self._keep[rid] = keep
        return rid

    def poll(self, max_results: int = 4096, timeout_ms: int = 0):
        out = tc_server_poll(self.handle, max_results, timeout_ms)
        for r in out:
            self._keep.pop(r["id"], None)
        return out

    def stats(self) -> dict:
        return tc_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            tc_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    """Owning wrapper: Graph(src, dst, n) loads and builds; count() / count_per_vertex(); freed on close()."""

    def __init__(self, src, dst, num_vertices: int, stream=None, allocator=None, build: bool = True):
        self.handle = tc_load_edges(src, dst, num_vertices, stream=stream, allocator=allocator)
        self.stream = stream
        if build:
            tc_build(self.handle, stream)

    def build(self):
        tc_build(self.handle, self.stream)

    def count(self) -> int:
        return tc_count(self.handle, self.stream)

    def count_per_vertex(self, out=None):
        return tc_count_per_vertex(self.handle, out, self.stream)

    def info(self) -> dict:
        return tc_graph_get_info(self.handle)

    def csr(self):
        return tc_copy_csr(self.handle, self.stream)

    def close(self):
        if self.handle:
            tc_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
