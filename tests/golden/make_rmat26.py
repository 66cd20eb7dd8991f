"""Writes tests/golden/rmat26_oracle.json: the CPU oracle's exact result on the R-MAT scale 26 workload.

Calls only graphgen/ (the seeded input) and oracle/ (the plain merge-intersection counter of Def. 2, Sec. II-A,
whose result is the |M|/|Q| of Algorithm 1).  Nothing here touches the CUDA library.  The stored values are:

* T, the exact triangle count, and m, the number of distinct undirected edges;
* sha256 of the per-vertex counts t(x) for x = 0..n-1, as little-endian uint64 (537 MB hashed, not stored);
* t(x) at 256 chosen vertices (the 64 largest input-pair counts, 64 at spread ranks, 128 seeded random ids);
* a fingerprint of the input itself (sha256 of the pairs at 2^16 spread indices), so that a test can tell a changed
  generator from a wrong count.

Run on a host with about 45 GB of free memory (2^30 pairs: 8.6 GB of input, the oracle's edge keys and adjacency
about 17 GB, per-thread t arrays 0.5 GB each):

    python tests/golden/make_rmat26.py --threads 8

It takes tens of minutes on 8 cores (the merge work grows with the sum of squared degrees).
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat26_oracle.json")


def fingerprint_indices(num_edges: int, k: int = 1 << 16) -> np.ndarray:
    """Spread indices of the sampled pairs hashed into the input fingerprint (first, last, and evenly between)."""
    return np.unique(np.linspace(0, num_edges - 1, k).astype(np.int64))


def input_fingerprint(src: np.ndarray, dst: np.ndarray, idx: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(src[idx]).astype("<i4").tobytes())
    h.update(np.ascontiguousarray(dst[idx]).astype("<i4").tobytes())
    return h.hexdigest()


def sample_vertices(src: np.ndarray, dst: np.ndarray, n: int) -> np.ndarray:
    cnt = np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    order = np.argsort(-cnt, kind="stable")
    spread = np.unique(np.geomspace(64, n - 1, 64).astype(np.int64))
    rng = np.random.default_rng(0x26)
    xs = np.concatenate([order[:64], order[spread], rng.integers(0, n, size=128)])
    return xs.astype(np.int32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--workload", default="rmat26")
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()

    spec = graphgen.config(args.workload)
    t0 = time.time()
    src, dst = spec.edges()
    t_gen = time.time() - t0
    fp_idx = fingerprint_indices(spec.num_edges)
    fp = input_fingerprint(src, dst, fp_idx)
    xs = sample_vertices(src, dst, spec.n)

    t0 = time.time()
    T, m, t = oracle.count(src, dst, spec.n, per_vertex=True, threads=args.threads)
    t_oracle = time.time() - t0
    assert int(t.sum()) == 3 * T  # each triangle has three vertices
    rec = {
        "workload": args.workload,
        "spec": {"kind": spec.kind, "n": spec.n, "num_edges": spec.num_edges, "seed": spec.seed,
                 "scale": spec.scale, "permute": spec.permute, "name": spec.name},
        "T": int(T),
        "m": int(m),
        "t_sha256": hashlib.sha256(np.ascontiguousarray(t).astype("<u8").tobytes()).hexdigest(),
        "t_max": int(t.max()),
        "sample_x": xs.tolist(),
        "sample_t": [int(v) for v in t[xs]],
        "input_fingerprint": {"indices": "numpy.unique(numpy.linspace(0, num_edges - 1, 65536).astype(int64))",
                              "sha256": fp},
        "command": f"python tests/golden/make_rmat26.py --threads {args.threads} --workload {args.workload}",
        "oracle_threads": args.threads,
        "seconds": {"generate": round(t_gen, 1), "oracle": round(t_oracle, 1)},
    }
    with open(args.out + ".tmp", "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    os.replace(args.out + ".tmp", args.out)
    print(json.dumps({k: rec[k] for k in ("T", "m", "t_sha256", "seconds")}))


if __name__ == "__main__":
    main()
