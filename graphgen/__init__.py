"""Seeded synthetic graph inputs for the triangle counter's tests and benchmark.

This module is the one thing the CPU oracle and the CUDA library have in common: it produces edge lists and holds
none of the counting arithmetic.  The per-edge generators live in ``gg.h`` and are evaluated either by the threaded
host library (``gg_host.cpp``) or by the device library (``gg_dev.cu``); the two give identical edges for the same
seed (checked by the tests).  Workload parameters that need floating point (R-MAT level thresholds with noise, the
log-uniform graph sizes of the batch and serving mixes) are computed here in Python, in IEEE double, and handed to
both sides as integers.

Workloads (the paper measures on HPEC Graph Challenge files, which are not available here; these seeded synthetic
graphs stand in for them, with the graph500 R-MAT parameters a/b/c/d = 0.57/0.19/0.19/0.05 for the Kronecker rows):

* ``er4096``   Erdos-Renyi G(n = 4096, p = 16/4095): every pair present independently (mean degree 16).
* ``rmat20``   R-MAT scale 20, edge factor 16 (16.8M sampled edges), per-level noise.
* ``rmat26``   R-MAT scale 26, edge factor 16 (2^30 sampled edges), per-level noise, ids relabelled by a seeded
               bijection.
* ``batch``    4096 graphs, n log-uniform in [64, 65536]; even index: G(n, p) with mean degree d uniform in
               [4, 64] (p = d / (n - 1)); odd index: R-MAT with edge factor in {8..32} (endpoints >= n redrawn).
* ``serve``    a pool of request graphs with edge counts log-uniform in [1e3, 4e6] (G(n, p) with mean degree 16 /
               R-MAT by parity).

Besides G(n, p) there is a uniform pair sampler (kind ``er``: a fixed number of pairs drawn with replacement,
self-loops and repeats left in), which tests use for repeat-heavy inputs.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libgg_host.so")
_DEV_SO = os.path.join(_HERE, "libgg_dev.so")

BASE_SEED = 0x190902127
BATCH_SEED_OFFSET = 0x10000
SERVE_SEED_OFFSET = 0x20000
RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)
RMAT_NOISE = 0.1

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


# ----------------------------------------------------------------------------------------------------------------
# Counter-based draws in pure Python (same definition as gg.h), used for workload parameters.
# ----------------------------------------------------------------------------------------------------------------
def mix64(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64((seed + GAMMA * (2 * stream + 1)) & M64) ^ mix64((stream + 0x632BE59BD9B4E019) & M64)


def draw(key: int, ctr: int) -> int:
    return mix64((key + ((ctr + 1) * GAMMA)) & M64)


def uniform01(key: int, ctr: int) -> float:
    """53-bit double in [0, 1)."""
    return (draw(key, ctr) >> 11) * (1.0 / (1 << 53))


STREAM_RMAT_NOISE = 4
STREAM_PARAMS = 5


LOG_FRAC_BITS = 40


def log2_q40(x: int) -> int:
    """log2(x) for an integer x >= 1 in Q.40 fixed point, truncated: the same integer steps as gg_log2_q40 in
    gg.h (integer part from the top bit; each fraction bit from squaring the mantissa in [1, 2), a square of 2 or
    more giving a 1 bit and being halved)."""
    if x < 1:
        raise ValueError("log2_q40 needs x >= 1")
    e = x.bit_length() - 1
    m = x << (63 - e)
    r = e << LOG_FRAC_BITS
    for b in range(LOG_FRAC_BITS - 1, -1, -1):
        sq = m * m
        if sq >> 127:
            r |= 1 << b
            m = sq >> 64
        else:
            m = sq >> 63
    return r


def gnp_lq(p: float) -> int:
    """-log2(1 - p) in Q.40, the input of the G(n, p) generator: 1 - p as a 63-bit fraction x / 2^63, then
    63 - log2(x) by log2_q40.  0 when p is too small to move 1 - p (an empty graph)."""
    if not 0.0 <= p < 1.0:
        raise ValueError("G(n, p) needs 0 <= p < 1")
    x = int(math.floor((1.0 - p) * 9223372036854775808.0))
    return (63 << LOG_FRAC_BITS) - log2_q40(max(1, min(x, 1 << 63)))


def rmat_thresholds(seed: int, scale: int, abcd=RMAT_ABCD, noise: float = RMAT_NOISE) -> np.ndarray:
    """Per-level cumulative R-MAT thresholds (uint32[3*scale]).  Level l scales each of a, b, c, d by
    (1 - noise/2 + noise*U) with its own uniform U, then renormalises to 1."""
    key = stream_key(seed, STREAM_RMAT_NOISE)
    out = np.zeros(3 * scale, dtype=np.uint32)
    for level in range(scale):
        p = [abcd[q] * (1.0 - noise / 2 + noise * uniform01(key, 4 * level + q)) for q in range(4)]
        tot = p[0] + p[1] + p[2] + p[3]
        cum = [p[0] / tot, (p[0] + p[1]) / tot, (p[0] + p[1] + p[2]) / tot]
        for i in range(3):
            out[3 * level + i] = min((1 << 32) - 1, int(math.floor(cum[i] * 4294967296.0)))
    return out


# ----------------------------------------------------------------------------------------------------------------
# Native libraries (built in-tree on first use, or by __graft_entry__.build()).
# ----------------------------------------------------------------------------------------------------------------
def _stale(target: str, sources) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build_host(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, "gg_host.cpp"), os.path.join(_HERE, "gg.h")]
    if force or _stale(_HOST_SO, srcs):
        tmp = _HOST_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", srcs[0], "-o", tmp])
        os.replace(tmp, _HOST_SO)
    return _HOST_SO


def build_dev(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, "gg_dev.cu"), os.path.join(_HERE, "gg.h")]
    if force or _stale(_DEV_SO, srcs):
        tmp = _DEV_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-Xcompiler", "-fPIC", "-shared", srcs[0], "-o", tmp])
        os.replace(tmp, _DEV_SO)
    return _DEV_SO


_host_lib = None
_dev_lib = None


def _host():
    global _host_lib
    if _host_lib is None:
        lib = ctypes.CDLL(build_host())
        i64, u64, u32, i32p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)
        lib.gg_er_host.argtypes = [u64, u32, i64, i64, i32p, i32p, ctypes.c_int]
        lib.gg_rmat_host.argtypes = [u64, ctypes.c_int, u32, ctypes.POINTER(ctypes.c_uint32), i64, i64, i32p, i32p,
                                     ctypes.c_int]
        lib.gg_permute_host.argtypes = [u64, u32, i32p, i64, ctypes.c_int]
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.gg_gnp_count_host.argtypes = [u64, u32, u64, i64p, ctypes.c_int]
        lib.gg_gnp_count_host.restype = ctypes.c_int64
        lib.gg_gnp_write_host.argtypes = [u64, u32, u64, i64p, i32p, i32p, ctypes.c_int]
        lib.gg_log2_q40_host.argtypes = [u64]
        lib.gg_log2_q40_host.restype = u64
        lib.gg_geometric_host.argtypes = [u64, u64]
        lib.gg_geometric_host.restype = u64
        _host_lib = lib
    return _host_lib


def _dev():
    global _dev_lib
    if _dev_lib is None:
        lib = ctypes.CDLL(build_dev())
        i64, u64, u32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.gg_er_dev.argtypes = [u64, u32, i64, i64, vp, vp, vp]
        lib.gg_rmat_dev.argtypes = [u64, ctypes.c_int, u32, vp, i64, i64, vp, vp, vp]
        lib.gg_permute_dev.argtypes = [u64, u32, vp, i64, vp]
        lib.gg_gnp_count_dev.argtypes = [u64, u32, u64, vp, vp]
        lib.gg_gnp_write_dev.argtypes = [u64, u32, u64, vp, vp, vp, vp]
        _dev_lib = lib
    return _dev_lib


def _threads() -> int:
    return max(1, os.cpu_count() or 1)


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


# ----------------------------------------------------------------------------------------------------------------
# Graph specifications
# ----------------------------------------------------------------------------------------------------------------
_gnp_counts = {}


def _gnp_offsets(seed: int, n: int, lq: int) -> np.ndarray:
    """Row offsets (int64[n + 1]) of a G(n, p) graph from the host generator."""
    off = np.empty(n + 1, dtype=np.int64)
    tot = _host().gg_gnp_count_host(seed, n, lq, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _threads())
    if tot < 0:
        raise RuntimeError("host G(n, p) generator failed")
    _gnp_counts[(seed, n, lq)] = int(tot)
    return off


@dataclass(frozen=True)
class GraphSpec:
    kind: str            # "gnp" (Erdos-Renyi G(n, p)), "er" (uniform pair sampling) or "rmat"
    n: int               # number of vertices
    pairs: int           # er / rmat: number of sampled (uncleaned) pairs; gnp: 0 (the number is drawn)
    seed: int
    scale: int = 0       # R-MAT only: 2^scale >= n
    permute: bool = False
    name: str = ""
    lq: int = 0          # gnp only: -log2(1 - p) in Q.40 (gnp_lq)
    p: float = 0.0       # gnp only: the pair probability

    @property
    def num_edges(self) -> int:
        """Number of pairs the generator produces: the sampled pairs, or for G(n, p) the pairs drawn (counted by
        the host generator on first use)."""
        if self.kind != "gnp":
            return self.pairs
        key = (self.seed, self.n, self.lq)
        if key not in _gnp_counts:
            _gnp_offsets(self.seed, self.n, self.lq)
        return _gnp_counts[key]

    @property
    def expected_edges(self) -> float:
        """Mean number of pairs (p * n(n-1)/2 for G(n, p)), known without generating anything."""
        return self.p * self.n * (self.n - 1) / 2.0 if self.kind == "gnp" else float(self.pairs)

    def thresholds(self) -> np.ndarray:
        return rmat_thresholds(self.seed, self.scale)

    def _gnp_edges(self, device):
        if device is None:
            off = _gnp_offsets(self.seed, self.n, self.lq)
            m = int(off[-1])
            src = np.empty(m, dtype=np.int32)
            dst = np.empty(m, dtype=np.int32)
            if _host().gg_gnp_write_host(self.seed, self.n, self.lq, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         _i32p(src), _i32p(dst), _threads()) != 0:
                raise RuntimeError("host G(n, p) generator failed")
            return src, dst
        import torch
        dev = torch.device(device)
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        lib = _dev()
        off = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        if lib.gg_gnp_count_dev(self.seed, self.n, self.lq, off.data_ptr(), stream) != 0:
            raise RuntimeError("device G(n, p) generator failed")
        torch.cumsum(off, 0, out=off)
        m = int(off[-1].item())
        _gnp_counts[(self.seed, self.n, self.lq)] = m
        src = torch.empty(m, dtype=torch.int32, device=dev)
        dst = torch.empty(m, dtype=torch.int32, device=dev)
        if m and lib.gg_gnp_write_dev(self.seed, self.n, self.lq, off.data_ptr(), src.data_ptr(), dst.data_ptr(),
                                      stream) != 0:
            raise RuntimeError("device G(n, p) generator failed")
        return src, dst

    def edges(self, device=None, e0: int = 0, length: Optional[int] = None):
        """Generated pairs [e0, e0+length) as (src, dst) int32 arrays: numpy on the host (device=None), else torch
        tensors on `device`, written on torch's current stream."""
        if self.kind == "gnp":
            src, dst = self._gnp_edges(device)
            end = src.shape[0] if length is None else e0 + length
            if e0 == 0 and end == src.shape[0]:
                return src, dst
            return src[e0:end], dst[e0:end]
        length = self.num_edges - e0 if length is None else length
        if device is None:
            src = np.empty(length, dtype=np.int32)
            dst = np.empty(length, dtype=np.int32)
            lib = _host()
            if self.kind == "er":
                rc = lib.gg_er_host(self.seed, self.n, e0, length, _i32p(src), _i32p(dst), _threads())
            else:
                thr = self.thresholds()
                rc = lib.gg_rmat_host(self.seed, self.scale, self.n,
                                      thr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), e0, length, _i32p(src),
                                      _i32p(dst), _threads())
            if rc != 0:
                raise RuntimeError(f"host generator failed ({rc}) for {self}")
            if self.permute:
                for a in (src, dst):
                    if lib.gg_permute_host(self.seed, self.n, _i32p(a), length, _threads()) != 0:
                        raise RuntimeError("host permutation failed")
            return src, dst
        import torch
        dev = torch.device(device)
        src = torch.empty(length, dtype=torch.int32, device=dev)
        dst = torch.empty(length, dtype=torch.int32, device=dev)
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        lib = _dev()
        if self.kind == "er":
            rc = lib.gg_er_dev(self.seed, self.n, e0, length, src.data_ptr(), dst.data_ptr(), stream)
        else:
            thr = torch.from_numpy(self.thresholds().view(np.int32)).to(dev)
            rc = lib.gg_rmat_dev(self.seed, self.scale, self.n, thr.data_ptr(), e0, length, src.data_ptr(),
                                 dst.data_ptr(), stream)
        if rc != 0:
            raise RuntimeError(f"device generator failed ({rc}) for {self}")
        if self.permute:
            for a in (src, dst):
                if lib.gg_permute_dev(self.seed, self.n, a.data_ptr(), length, stream) != 0:
                    raise RuntimeError("device permutation failed")
        return src, dst


def gnp(n: int, p: float, seed: int, name: str = "") -> GraphSpec:
    """Erdos-Renyi G(n, p): each of the n(n-1)/2 pairs present independently with probability p."""
    return GraphSpec("gnp", n, 0, seed, name=name, lq=gnp_lq(p), p=float(p))


def er(n: int, num_edges: int, seed: int, name: str = "") -> GraphSpec:
    return GraphSpec("er", n, num_edges, seed, name=name)


def rmat(scale: int, edge_factor: int, seed: int, n: Optional[int] = None, permute: bool = False,
         num_edges: Optional[int] = None, name: str = "") -> GraphSpec:
    n = (1 << scale) if n is None else n
    m = edge_factor * n if num_edges is None else num_edges
    return GraphSpec("rmat", n, m, seed, scale=scale, permute=permute, name=name)


def config(name: str) -> GraphSpec:
    """The three single-graph workloads."""
    if name == "er4096":
        return gnp(4096, 16.0 / 4095.0, BASE_SEED + 0, name="ER G(4096, 16/4095)")
    if name == "rmat20":
        return rmat(20, 16, BASE_SEED + 1, name="R-MAT scale 20 ef 16")
    if name == "rmat26":
        return rmat(26, 16, BASE_SEED + 2, permute=True, name="R-MAT scale 26 ef 16 (permuted ids)")
    if name.startswith("rmat") and name[4:].isdigit():  # other scales, for profiling and sweeps
        scale = int(name[4:])
        return rmat(scale, 16, BASE_SEED + 100 + scale, name=f"R-MAT scale {scale} ef 16")
    raise KeyError(name)


def batch_mix(num_graphs: int = 4096, base_seed: int = BASE_SEED + BATCH_SEED_OFFSET):
    """The batched workload: n log-uniform in [64, 65536]; even i G(n, p) with mean degree d ~ U[4, 64],
    p = d / (n - 1); odd i R-MAT with edge factor uniform in {8..32}."""
    specs = []
    lo, hi = math.log(64.0), math.log(65536.0)
    for i in range(num_graphs):
        seed = base_seed + i
        key = stream_key(seed, STREAM_PARAMS)
        n = int(math.floor(math.exp(lo + (hi - lo) * uniform01(key, 0))))
        n = max(64, min(65536, n))
        if i % 2 == 0:
            deg = 4.0 + 60.0 * uniform01(key, 1)
            specs.append(gnp(n, min(deg / (n - 1), 0.999), seed, name=f"batch{i}"))
        else:
            ef = 8 + int(draw(key, 2) % 25)
            scale = max(1, (n - 1).bit_length())
            specs.append(rmat(scale, ef, seed, n=n, name=f"batch{i}"))
    return specs


def serve_pool(pool_size: int = 1024, base_seed: int = BASE_SEED + SERVE_SEED_OFFSET, lo_edges: float = 1e3,
               hi_edges: float = 4e6):
    """Request graphs of the serving workload: edge count log-uniform in [lo_edges, hi_edges] (for G(n, p) its
    mean); even j G(n, p) with mean degree 16 on n = m / 8 vertices, odd j R-MAT with edge factor 16."""
    specs = []
    lo, hi = math.log(lo_edges), math.log(hi_edges)
    for j in range(pool_size):
        seed = base_seed + j
        key = stream_key(seed, STREAM_PARAMS)
        m = int(math.floor(math.exp(lo + (hi - lo) * uniform01(key, 0))))
        if j % 2 == 0:
            n = max(33, int(round(m / 8.0)))
            specs.append(gnp(n, 16.0 / (n - 1), seed, name=f"serve{j}"))
        else:
            n = max(32, (m + 15) // 16)
            scale = max(1, (n - 1).bit_length())
            specs.append(rmat(scale, 16, seed, n=n, num_edges=m, name=f"serve{j}"))
    return specs


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int = BASE_SEED + SERVE_SEED_OFFSET - 1):
    """Arrival times (seconds) of a Poisson stream: exponential gaps from counter-based uniforms."""
    key = stream_key(seed, STREAM_PARAMS)
    t, out, i = 0.0, [], 0
    while True:
        u = uniform01(key, i)
        i += 1
        t += -math.log(1.0 - u) / rate_per_s
        if t >= duration_s:
            return np.array(out, dtype=np.float64)
        out.append(t)
