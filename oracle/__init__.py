"""CPU oracle for exact triangle counting — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this package.  It
shares no code with the CUDA library and is never used by it.

The arithmetic lives in ``tc_oracle.cpp`` (plain C++, see its header for the definitions it follows: Def. 1 and
Def. 2 of Sec. II-A, the |M|/|Q| result of Algorithm 1 and the increasing-id visiting order of Sec. III-A/III-C).
This module compiles it with g++ on first use and marshals numpy arrays to it.

Parity status: oracle_count is pinned by closed forms, dense trace(A^3)/6 brute force and invariances
(tests/test_oracle.py); oracle_vertex_triangles is pinned by the same closed forms, by the brute-force diagonal
diag(A^3)/2 and by agreement with oracle_count's per-vertex output; oracle_list_triangles is pinned by the clique
closed form (every 3-subset listed) and by dense brute force (the right number of distinct triples, each a
triangle) in tests/test_listing.py.  frontiers.py (numpy) gives the frontier sizes of the unfused loop of
Algorithm 1, pinned by closed forms and loop enumeration in tests/test_unfused.py; prune.py (numpy) is the NE
filter applied until it settles (the 2-core), pinned by networkx's k_core and closed forms in tests/test_prune.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "tc_oracle.cpp")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2, portable flags: the same source builds on x86-64 and aarch64)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SRC) > os.path.getmtime(_SO):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_count.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, u64p, i64p, u64p]
        lib.oracle_count.restype = ctypes.c_int
        lib.oracle_vertex_triangles.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, i32p, ctypes.c_int64,
                                                ctypes.c_int, u64p, i64p]
        lib.oracle_vertex_triangles.restype = ctypes.c_int
        lib.oracle_list_triangles.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, i32p, ctypes.c_int64, u64p]
        lib.oracle_list_triangles.restype = ctypes.c_int
        _lib = lib
    return _lib


def _threads(threads):
    return max(1, os.cpu_count() or 1) if threads is None else int(threads)


def _as_i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


class OracleError(ValueError):
    pass


def count(src, dst, n: int, per_vertex: bool = False, threads=None):
    """Exact triangle count of the simple undirected graph given by the pairs (src[i], dst[i]) on [0, n).

    Returns (T, m) or (T, m, t) with t the uint64 per-vertex counts; m is the number of distinct undirected edges.
    """
    src, dst = _as_i32(src), _as_i32(dst)
    if src.shape != dst.shape:
        raise OracleError("src and dst differ in length")
    lib = _load()
    T = ctypes.c_uint64(0)
    m = ctypes.c_int64(0)
    t = np.zeros(max(n, 0), dtype=np.uint64) if per_vertex else None
    rc = lib.oracle_count(src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          dst.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), src.size, n, _threads(threads),
                          ctypes.byref(T), ctypes.byref(m),
                          t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if per_vertex else None)
    if rc != 0:
        raise OracleError(f"oracle_count failed with code {rc}")
    return (int(T.value), int(m.value), t) if per_vertex else (int(T.value), int(m.value))


def list_triangles(src, dst, n: int, capacity=None):
    """Every triangle as an ascending id triple (shape (T, 3), in the order the enumeration finds them)."""
    src, dst = _as_i32(src), _as_i32(dst)
    lib = _load()
    if capacity is None:
        capacity = count(src, dst, n)[0]
    out = np.zeros((max(int(capacity), 1), 3), dtype=np.int32)
    T = ctypes.c_uint64(0)
    rc = lib.oracle_list_triangles(src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   dst.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), src.size, n,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(capacity), ctypes.byref(T))
    if rc != 0:
        raise OracleError(f"oracle_list_triangles failed with code {rc}")
    return out[: min(int(T.value), int(capacity))], int(T.value)


def vertex_triangles(src, dst, n: int, xs, threads=None):
    """t(x) for each x in xs, from the definition t(x) = #edges {a,b} with a, b in N(x).  Returns (t, deg)."""
    src, dst, xs = _as_i32(src), _as_i32(dst), _as_i32(xs)
    lib = _load()
    out = np.zeros(xs.size, dtype=np.uint64)
    deg = np.zeros(xs.size, dtype=np.int64)
    rc = lib.oracle_vertex_triangles(src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     dst.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), src.size, n,
                                     xs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), xs.size, _threads(threads),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                     deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise OracleError(f"oracle_vertex_triangles failed with code {rc}")
    return out, deg
