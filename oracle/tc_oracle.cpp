// tc_oracle.cpp — CPU ORACLE for exact triangle counting.  TEST INFRASTRUCTURE ONLY.
//
// Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this library.  It shares no code,
// header, table or helper with the CUDA library; it is deliberately plain and slow, written so that a reader can
// check it against the definitions by eye.
//
// What it computes (Wang & Owens, "Fast BFS-Based Triangle Counting on GPUs", Sec. II-A):
//   * The data graph G = (V, E) is undirected (Def. 1); (u,v) and (v,u) name the same edge.  The input lists
//     ordered pairs; a pair (u,v) puts the undirected edge {u,v} in E.  Self-loops and repeated pairs are dropped:
//     E is a set of 2-element vertex sets (a simple graph).
//   * A triangle is an embedding of the 3-vertex query graph Q = K3 (Def. 2): a vertex set {a,b,c} with ab, bc and
//     ca all in E.  Each such set is one match; the count is the number of distinct sets (the |M|/|Q| result of
//     Algorithm 1, one match per triangle under the unique mapping order u1 < u2 < u3 of Sec. III-A).
//   * The per-vertex count t(x) is the number of triangles that contain x.
//
// oracle_count enumerates each triangle exactly once as its id-ordered triple a < b < c: for every edge {a,b} with
// a < b, every c > b adjacent to both a and b closes one (this is the increasing-node-id visiting order that
// Sec. III-A and Sec. III-C use to avoid duplicate matches).  The intersection is a merge of two sorted lists.
//
// oracle_list_triangles writes the triangles themselves (the matched node id lists of Sec. II-A) as the same
// id-ordered triples a < b < c, in the order oracle_count finds them.
//
// oracle_vertex_triangles computes t(x) for chosen vertices straight from the definition
//   t(x) = |{ {a,b} : a,b in N(x), a != b, {a,b} in E }|
// without building any adjacency structure: one scan of the input collects N(x), a second collects the distinct
// edges with both ends in N(x).  It is used for spot checks on graphs too large for oracle_count.
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

int clamp_threads(int t) { return t < 1 ? 1 : (t > 256 ? 256 : t); }

// Steps 1-2: drop self-loops, canonicalise {u,v} as (min, max), sort and drop repeats.
// Returns 0, or 2 if an id is outside [0, n).
int simple_edges(const int32_t* src, const int32_t* dst, int64_t M, int32_t n, std::vector<uint64_t>& E) {
  E.clear();
  E.reserve((size_t)M);
  for (int64_t i = 0; i < M; ++i) {
    const int32_t a = src[i], b = dst[i];
    if (a < 0 || a >= n || b < 0 || b >= n) return 2;
    if (a == b) continue;
    const uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
    E.push_back(((uint64_t)lo << 32) | hi);
  }
  std::sort(E.begin(), E.end());
  E.erase(std::unique(E.begin(), E.end()), E.end());
  return 0;
}

}  // namespace

extern "C" {

// Exact triangle count T of the simple undirected graph given by the pairs (src[i], dst[i]), i < M, on vertices
// [0, n).  Writes T, the number m of distinct undirected edges, and (if per_vertex != NULL) t(x) for every x.
// Returns 0 on success, 1 on a bad argument, 2 if an id is outside [0, n).
int oracle_count(const int32_t* src, const int32_t* dst, int64_t M, int32_t n, int threads, uint64_t* out_T,
                 int64_t* out_m, uint64_t* per_vertex) {
  if (M < 0 || n < 0 || !out_T || (M > 0 && (!src || !dst))) return 1;
  threads = clamp_threads(threads);
  std::vector<uint64_t> E;
  if (int rc = simple_edges(src, dst, M, n, E)) return rc;
  if (out_m) *out_m = (int64_t)E.size();

  // Step 3: full adjacency, each list sorted ascending.
  std::vector<int64_t> off((size_t)n + 1, 0);
  for (uint64_t e : E) {
    off[(e >> 32) + 1]++;
    off[(uint32_t)e + 1]++;
  }
  for (int32_t x = 0; x < n; ++x) off[x + 1] += off[x];
  std::vector<int32_t> adj((size_t)off[n]);
  {
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (uint64_t e : E) {
      const int32_t a = (int32_t)(e >> 32), b = (int32_t)(uint32_t)e;
      adj[fill[a]++] = b;
      adj[fill[b]++] = a;
    }
  }
  for (int32_t x = 0; x < n; ++x) std::sort(adj.begin() + off[x], adj.begin() + off[x + 1]);

  // Step 4: for each edge a < b, merge-intersect the parts of adj[a] and adj[b] above b.
  std::atomic<int64_t> cursor{0};
  const int64_t chunk = 1024;
  std::vector<uint64_t> T_part(threads, 0);
  std::vector<std::vector<uint64_t>> t_part(per_vertex ? threads : 0);
  auto work = [&](int tid) {
    uint64_t T = 0;
    uint64_t* t = nullptr;
    if (per_vertex) {
      t_part[tid].assign((size_t)n, 0);
      t = t_part[tid].data();
    }
    for (;;) {
      const int64_t lo = cursor.fetch_add(chunk);
      if (lo >= (int64_t)E.size()) break;
      const int64_t hi = std::min<int64_t>((int64_t)E.size(), lo + chunk);
      for (int64_t i = lo; i < hi; ++i) {
        const int32_t a = (int32_t)(E[i] >> 32), b = (int32_t)(uint32_t)E[i];
        const int32_t* pa = std::lower_bound(adj.data() + off[a], adj.data() + off[a + 1], b + 1);
        const int32_t* ea = adj.data() + off[a + 1];
        const int32_t* pb = std::lower_bound(adj.data() + off[b], adj.data() + off[b + 1], b + 1);
        const int32_t* eb = adj.data() + off[b + 1];
        while (pa < ea && pb < eb) {
          if (*pa < *pb) {
            ++pa;
          } else if (*pb < *pa) {
            ++pb;
          } else {  // c = *pa closes the triangle a < b < c
            ++T;
            if (t) {
              t[a]++;
              t[b]++;
              t[*pa]++;
            }
            ++pa;
            ++pb;
          }
        }
      }
    }
    T_part[tid] = T;
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < threads; ++i) pool.emplace_back(work, i);
  work(0);
  for (auto& th : pool) th.join();

  // Step 5: integer sums, independent of the order the threads finished in.
  uint64_t T = 0;
  for (uint64_t x : T_part) T += x;
  *out_T = T;
  if (per_vertex) {
    for (int32_t x = 0; x < n; ++x) {
      uint64_t s = 0;
      for (int i = 0; i < threads; ++i) s += t_part[i][x];
      per_vertex[x] = s;
    }
  }
  return 0;
}

// The triangles themselves (the matched node id lists of Sec. II-A), as id triples a < b < c, enumerated exactly as
// oracle_count counts them.  Writes min(T, capacity) triples to out (3 int32 each) and T to *out_T.
// Returns 0, 1 (bad argument) or 2 (id out of range).  Single-threaded.
int oracle_list_triangles(const int32_t* src, const int32_t* dst, int64_t M, int32_t n, int32_t* out,
                          int64_t capacity, uint64_t* out_T) {
  if (M < 0 || n < 0 || capacity < 0 || !out_T || (capacity > 0 && !out) || (M > 0 && (!src || !dst))) return 1;
  std::vector<uint64_t> E;
  if (int rc = simple_edges(src, dst, M, n, E)) return rc;
  std::vector<int64_t> off((size_t)n + 1, 0);
  for (uint64_t e : E) {
    off[(e >> 32) + 1]++;
    off[(uint32_t)e + 1]++;
  }
  for (int32_t x = 0; x < n; ++x) off[x + 1] += off[x];
  std::vector<int32_t> adj((size_t)off[n]);
  {
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (uint64_t e : E) {
      const int32_t a = (int32_t)(e >> 32), b = (int32_t)(uint32_t)e;
      adj[fill[a]++] = b;
      adj[fill[b]++] = a;
    }
  }
  for (int32_t x = 0; x < n; ++x) std::sort(adj.begin() + off[x], adj.begin() + off[x + 1]);
  uint64_t T = 0;
  for (uint64_t e : E) {
    const int32_t a = (int32_t)(e >> 32), b = (int32_t)(uint32_t)e;
    const int32_t* pa = std::lower_bound(adj.data() + off[a], adj.data() + off[a + 1], b + 1);
    const int32_t* ea = adj.data() + off[a + 1];
    const int32_t* pb = std::lower_bound(adj.data() + off[b], adj.data() + off[b + 1], b + 1);
    const int32_t* eb = adj.data() + off[b + 1];
    while (pa < ea && pb < eb) {
      if (*pa < *pb) {
        ++pa;
      } else if (*pb < *pa) {
        ++pb;
      } else {
        if ((int64_t)T < capacity) {
          out[3 * T] = a;
          out[3 * T + 1] = b;
          out[3 * T + 2] = *pa;
        }
        ++T;
        ++pa;
        ++pb;
      }
    }
  }
  *out_T = T;
  return 0;
}

// t(x) for the k vertices xs[0..k) of the graph given by the pairs, from the definition (see file comment).
// out[j] = t(xs[j]); out_deg[j] (if not NULL) = |N(xs[j])|.  Returns 0, 1 (bad argument) or 2 (id out of range).
int oracle_vertex_triangles(const int32_t* src, const int32_t* dst, int64_t M, int32_t n, const int32_t* xs,
                            int64_t k, int threads, uint64_t* out, int64_t* out_deg) {
  if (M < 0 || n < 0 || k < 0 || (k > 0 && (!xs || !out)) || (M > 0 && (!src || !dst))) return 1;
  threads = clamp_threads(threads);
  for (int64_t j = 0; j < k; ++j)
    if (xs[j] < 0 || xs[j] >= n) return 2;
  for (int64_t i = 0; i < M; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return 2;

  // Which sample indices each vertex is (a vertex may be listed more than once).
  std::unordered_map<int32_t, std::vector<int32_t>> sample_of;
  for (int64_t j = 0; j < k; ++j) sample_of[xs[j]].push_back((int32_t)j);

  auto split = [&](auto&& body) {
    std::vector<std::thread> pool;
    const int64_t per = (M + threads - 1) / threads;
    for (int i = 0; i < threads; ++i) {
      const int64_t lo = i * per, hi = std::min<int64_t>(M, lo + per);
      if (lo >= hi) break;
      pool.emplace_back(body, i, lo, hi);
    }
    for (auto& th : pool) th.join();
  };

  // Scan 1: N(x) = distinct neighbours y != x.
  std::vector<std::vector<std::vector<int32_t>>> nb_part(threads, std::vector<std::vector<int32_t>>((size_t)k));
  split([&](int tid, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      const int32_t a = src[i], b = dst[i];
      if (a == b) continue;
      auto ia = sample_of.find(a);
      if (ia != sample_of.end())
        for (int32_t j : ia->second) nb_part[tid][j].push_back(b);
      auto ib = sample_of.find(b);
      if (ib != sample_of.end())
        for (int32_t j : ib->second) nb_part[tid][j].push_back(a);
    }
  });
  std::vector<std::vector<int32_t>> N((size_t)k);
  for (int64_t j = 0; j < k; ++j) {
    for (int t = 0; t < threads; ++t) N[j].insert(N[j].end(), nb_part[t][j].begin(), nb_part[t][j].end());
    std::sort(N[j].begin(), N[j].end());
    N[j].erase(std::unique(N[j].begin(), N[j].end()), N[j].end());
    if (out_deg) out_deg[j] = (int64_t)N[j].size();
  }
  nb_part.clear();

  // Inverse index: vertex y -> samples j with y in N(xs[j]).
  std::unordered_map<int32_t, std::vector<int32_t>> in_nbhd;
  for (int64_t j = 0; j < k; ++j)
    for (int32_t y : N[j]) in_nbhd[y].push_back((int32_t)j);

  // Scan 2: the distinct edges {a,b} with a, b both in N(xs[j]).
  std::vector<std::vector<std::vector<uint64_t>>> e_part(threads, std::vector<std::vector<uint64_t>>((size_t)k));
  split([&](int tid, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      const int32_t a = src[i], b = dst[i];
      if (a == b) continue;
      auto ia = in_nbhd.find(a);
      if (ia == in_nbhd.end()) continue;
      auto ib = in_nbhd.find(b);
      if (ib == in_nbhd.end()) continue;
      const uint64_t key = ((uint64_t)(uint32_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b);
      // samples in both lists (both lists ascending)
      auto p = ia->second.begin(), q = ib->second.begin();
      while (p != ia->second.end() && q != ib->second.end()) {
        if (*p < *q) {
          ++p;
        } else if (*q < *p) {
          ++q;
        } else {
          e_part[tid][*p].push_back(key);
          ++p;
          ++q;
        }
      }
    }
  });
  for (int64_t j = 0; j < k; ++j) {
    std::vector<uint64_t> Ej;
    for (int t = 0; t < threads; ++t) {
      Ej.insert(Ej.end(), e_part[t][j].begin(), e_part[t][j].end());
      std::vector<uint64_t>().swap(e_part[t][j]);
    }
    std::sort(Ej.begin(), Ej.end());
    out[j] = (uint64_t)(std::unique(Ej.begin(), Ej.end()) - Ej.begin());
  }
  return 0;
}

}  // extern "C"
