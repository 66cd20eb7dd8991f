// tc_serve.cu — a serving loop for triangle-count requests with continuous batching.
//
// Requests (edge lists in host memory) are submitted from any thread.  Admission is decided by device memory:
// a request is admitted when its estimated peak footprint fits in the HBM budget (free memory at start-up minus a
// reserve, less what admitted requests hold) and the in-flight limit allows it.  Build workers, each with its own
// CUDA stream, copy and build admitted requests concurrently (tc_load_edges + tc_build); the CSR then stays
// resident until counted.  One counting thread runs continuously: each time a launch finishes it takes every
// graph that became ready meanwhile and counts them all in one persistent launch (tc_count_batch), so requests
// that arrive while others are on the GPU join the next launch instead of waiting for a queue to drain.  With
// batching off, it counts one graph per launch instead (the baseline).
//
// Pipeline batching (batching = 2) batches the whole path, not only the count: each build worker takes every
// pending request that the memory budget admits (up to the compact build's pair limit) and ingests, builds and
// counts them together as their disjoint union (tc_count_many), so the launch sequence of a build, which costs more
// than the count for most requests, is paid once per batch.  Every wait is on a host condition variable; nothing
// spins on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tc_build.cuh"
#include "tc_internal.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  tc_request_result res{};
  const int32_t* src = nullptr;
  const int32_t* dst = nullptr;
  const int32_t* dsrc = nullptr;  // pipeline batching: device-readable arrays (mapped host memory), or the host ones
  const int32_t* ddst = nullptr;
  uint8_t stage = 0;              // pipeline batching: 1 if the arrays must be copied to the device
  int64_t m = 0;
  int64_t n = 0;
  int64_t bytes = 0;
  tc_graph* g = nullptr;
};

// Peak device bytes of building one request: two 8-byte key buffers per pair, the 8-byte staging of the host copy,
// the CSR (4-byte columns plus padding) and about ten 4- or 8-byte arrays per vertex.
int64_t estimate_bytes(int64_t m, int64_t n) { return 32 * m + 48 * n + (1 << 20); }

void* pool_alloc(size_t bytes, void* stream, void* ctx) {
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, (cudaMemPool_t)ctx, (cudaStream_t)stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}
void pool_free(void* p, void* stream, void*) { (void)cudaFreeAsync(p, (cudaStream_t)stream); }

}  // namespace

struct tc_server {
  tc_server_config cfg{};
  int device = 0;
  cudaMemPool_t pool = nullptr;
  tc_allocator alloc{};
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::vector<Request*> ready;
  std::deque<Request*> done;
  int64_t held = 0;
  int64_t inflight = 0;
  uint64_t next_id = 1;
  bool stop = false;
  tc_server_stats stats{};
  std::vector<std::thread> builders;
  std::thread counter;
  cudaStream_t count_stream = nullptr;
};

namespace {

void finish(tc_server* s, Request* r, tc_status st, uint64_t count) {
  if (r->g) {
    tc_free(r->g);
    r->g = nullptr;
  }
  r->res.status = st;
  r->res.triangles = count;
  r->res.t_done_ns = now_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  s->held -= r->bytes;
  s->inflight -= 1;
  s->done.push_back(r);
  if (st == TC_OK)
    s->stats.completed += 1;
  else
    s->stats.failed += 1;
  s->cv.notify_all();
}

void builder_loop(tc_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->stop) return true;
        if (s->pending.empty()) return false;
        Request* h = s->pending.front();
        const bool fits = s->held + h->bytes <= s->budget || s->inflight == 0;  // a lone request always runs
        return fits && s->inflight < s->cfg.max_inflight;
      });
      if (s->stop) break;
      r = s->pending.front();
      s->pending.pop_front();
      s->held += r->bytes;
      s->inflight += 1;
      s->stats.admitted += 1;
      s->stats.peak_held_bytes = std::max<int64_t>(s->stats.peak_held_bytes, s->held);
    }
    r->res.t_admit_ns = now_ns();
    tc_graph* g = nullptr;
    tc_status rc = tc_load_edges(r->src, r->dst, r->m, r->n, TC_PTR_HOST, &s->alloc, st, &g);
    if (rc == TC_OK) rc = tc_build(g, st);
    r->g = g;
    r->res.t_built_ns = now_ns();
    if (rc != TC_OK) {
      finish(s, r, rc, 0);
      continue;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->ready.push_back(r);
    s->cv.notify_all();
  }
  cudaStreamDestroy(st);
}

// Pipeline batching: a build worker that counts batches of pending requests as one disjoint union.
void batch_builder_loop(tc_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  const int64_t pair_cap = std::max<int64_t>(1, tc::compact_max_pairs());
  std::vector<Request*> batch;
  std::vector<const int32_t*> srcs, dsts;
  std::vector<int64_t> ne, nv;
  std::vector<uint8_t> stage;
  std::vector<uint64_t> counts;
  while (true) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->stop) return true;
        if (s->pending.empty()) return false;
        Request* h = s->pending.front();
        const bool fits = s->held + h->bytes <= s->budget || s->inflight == 0;  // a lone request always runs
        return fits && s->inflight < s->cfg.max_inflight;
      });
      if (s->stop) break;
      int64_t pairs = 0;
      while (!s->pending.empty() && (int64_t)batch.size() < s->cfg.max_batch) {
        Request* h = s->pending.front();
        const bool fits = s->held + h->bytes <= s->budget || s->inflight == 0;
        if (!fits || s->inflight >= s->cfg.max_inflight) break;
        if (!batch.empty() && pairs + h->m > pair_cap) break;
        s->pending.pop_front();
        s->held += h->bytes;
        s->inflight += 1;
        s->stats.admitted += 1;
        s->stats.peak_held_bytes = std::max<int64_t>(s->stats.peak_held_bytes, s->held);
        pairs += h->m;
        batch.push_back(h);
      }
      s->stats.launches += 1;
      s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, (int64_t)batch.size());
    }
    const int64_t t_admit = now_ns();
    const int32_t k = (int32_t)batch.size();
    srcs.resize(k);
    dsts.resize(k);
    ne.resize(k);
    nv.resize(k);
    stage.resize(k);
    counts.assign(k, 0);
    for (int32_t i = 0; i < k; ++i) {
      Request* r = batch[i];
      r->res.t_admit_ns = t_admit;
      srcs[i] = r->dsrc;
      dsts[i] = r->ddst;
      ne[i] = r->m;
      nv[i] = r->n;
      stage[i] = r->stage;
    }
    tc_status rc = tc::count_many(srcs.data(), dsts.data(), ne.data(), nv.data(), stage.data(), k, counts.data(),
                              &s->alloc, st);
    if (rc == TC_ERR_OUT_OF_RANGE && k > 1) {  // one bad request: every request of the batch on its own
      for (int32_t i = 0; i < k; ++i) {
        uint64_t c = 0;
        const tc_status ri = tc::count_many(&srcs[i], &dsts[i], &ne[i], &nv[i], &stage[i], 1, &c, &s->alloc, st);
        batch[i]->res.t_built_ns = now_ns();
        finish(s, batch[i], ri, ri == TC_OK ? c : 0);
      }
      continue;
    }
    const int64_t t_built = now_ns();
    for (int32_t i = 0; i < k; ++i) {
      batch[i]->res.t_built_ns = t_built;
      finish(s, batch[i], rc, rc == TC_OK ? counts[i] : 0);
    }
  }
  cudaStreamDestroy(st);
}

void counter_loop(tc_server* s) {
  cudaSetDevice(s->device);
  std::vector<Request*> batch;
  std::vector<tc_graph*> graphs;
  std::vector<uint64_t> counts;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->ready.empty(); });
      if (s->stop && s->ready.empty()) break;
      const size_t take = std::min<size_t>(s->ready.size(), (size_t)s->cfg.max_batch);
      batch.assign(s->ready.begin(), s->ready.begin() + take);
      s->ready.erase(s->ready.begin(), s->ready.begin() + take);
    }
    if (s->cfg.batching) {
      graphs.resize(batch.size());
      counts.assign(batch.size(), 0);
      for (size_t i = 0; i < batch.size(); ++i) graphs[i] = batch[i]->g;
      const tc_status rc = tc_count_batch(graphs.data(), (int32_t)graphs.size(), counts.data(), s->count_stream);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.launches += 1;
        s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, (int64_t)batch.size());
      }
      for (size_t i = 0; i < batch.size(); ++i) finish(s, batch[i], rc, rc == TC_OK ? counts[i] : 0);
    } else {
      for (Request* r : batch) {
        uint64_t c = 0;
        const tc_status rc = tc_count(r->g, &c, s->count_stream);
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->stats.launches += 1;
          s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, 1);
        }
        finish(s, r, rc, c);
      }
    }
  }
}

}  // namespace

using namespace tc;

extern "C" {

TC_API tc_status tc_server_create(const tc_server_config* cfg, tc_server** out) {
  if (!out) {
    set_error("tc_server_create: out is NULL");
    return TC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  tc_server_config c{};
  c.build_workers = 4;
  c.max_batch = 4096;
  c.batching = 1;
  c.max_inflight = 8192;
  c.hbm_reserve_bytes = (int64_t)8 << 30;
  if (cfg) {
    if (cfg->build_workers > 0) c.build_workers = cfg->build_workers;
    if (cfg->max_batch > 0) c.max_batch = cfg->max_batch;
    c.batching = cfg->batching;
    if (cfg->max_inflight > 0) c.max_inflight = cfg->max_inflight;
    if (cfg->hbm_reserve_bytes >= 0) c.hbm_reserve_bytes = cfg->hbm_reserve_bytes;
    c.hbm_budget_bytes = cfg->hbm_budget_bytes;
  }
  if (c.build_workers > 64 || c.max_batch > (1 << 20) || c.batching < 0 || c.batching > 2) {
    set_error("tc_server_create: build_workers must be <= 64, max_batch <= 2^20 and batching 0, 1 or 2");
    return TC_ERR_INVALID_ARG;
  }
  tc_server* s = new (std::nothrow) tc_server();
  if (!s) {
    set_error("tc_server_create: host allocation failed");
    return TC_ERR_NO_MEMORY;
  }
  s->cfg = c;
  tc_status st = TC_OK;
  do {
    if ((st = cuda_status(cudaGetDevice(&s->device), "cudaGetDevice"))) break;
    size_t free_b = 0, total_b = 0;
    if ((st = cuda_status(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo"))) break;
    s->budget = (int64_t)free_b - c.hbm_reserve_bytes;
    if (c.hbm_budget_bytes > 0) s->budget = std::min<int64_t>(s->budget, c.hbm_budget_bytes);
    if (s->budget <= 0) {
      set_error("tc_server_create: no device memory left beyond the reserve");
      st = TC_ERR_NO_MEMORY;
      break;
    }
    s->stats.budget_bytes = s->budget;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if ((st = cuda_status(cudaMemPoolCreate(&s->pool, &props), "cudaMemPoolCreate"))) break;
    uint64_t keep = UINT64_MAX;  // keep freed memory in the pool between requests
    if ((st = cuda_status(cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep), "pool attr"))) break;
    s->alloc.alloc = pool_alloc;
    s->alloc.free = pool_free;
    s->alloc.ctx = (void*)s->pool;
    if ((st = cuda_status(cudaStreamCreateWithFlags(&s->count_stream, cudaStreamNonBlocking), "stream"))) break;
  } while (0);
  if (st != TC_OK) {
    if (s->count_stream) cudaStreamDestroy(s->count_stream);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return st;
  }
  for (int i = 0; i < c.build_workers; ++i) s->builders.emplace_back(c.batching == 2 ? batch_builder_loop : builder_loop, s);
  s->counter = std::thread(counter_loop, s);
  *out = s;
  return TC_OK;
}

TC_API tc_status tc_server_submit(tc_server* s, const int32_t* src, const int32_t* dst, int64_t num_edges,
                                  int64_t num_vertices, uint64_t* id_out) {
  if (!s || num_edges < 0 || num_vertices < 0 || (num_edges > 0 && (!src || !dst))) {
    set_error("tc_server_submit: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) {
    set_error("tc_server_submit: host allocation failed");
    return TC_ERR_NO_MEMORY;
  }
  r->src = src;
  r->dst = dst;
  r->m = num_edges;
  r->n = num_vertices;
  r->bytes = estimate_bytes(num_edges, num_vertices);
  r->res.t_submit_ns = now_ns();
  r->dsrc = src;
  r->ddst = dst;
  if (s->cfg.batching == 2 && num_edges > 0) {  // where the union's ingest reads this request's arrays from
    const int32_t* ms = tc::mapped_for_device(src, num_edges);
    const int32_t* md = ms ? tc::mapped_for_device(dst, num_edges) : nullptr;
    if (ms && md) {
      r->dsrc = ms;
      r->ddst = md;
    } else {
      r->stage = 1;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    set_error("tc_server_submit: server is shutting down");
    return TC_ERR_STATE;
  }
  if (r->bytes > s->budget) {
    delete r;
    set_error("tc_server_submit: the request alone exceeds the device memory budget");
    return TC_ERR_NO_MEMORY;
  }
  r->res.id = s->next_id++;
  if (id_out) *id_out = r->res.id;
  s->pending.push_back(r);
  s->stats.submitted += 1;
  s->cv.notify_all();
  return TC_OK;
}

TC_API tc_status tc_server_poll(tc_server* s, tc_request_result* out, int32_t max_results, int32_t timeout_ms,
                                int32_t* n_out) {
  if (!s || !n_out || max_results < 0 || (max_results > 0 && !out)) {
    set_error("tc_server_poll: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  *n_out = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (timeout_ms > 0)
    s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < max_results && !s->done.empty()) {
    Request* r = s->done.front();
    s->done.pop_front();
    out[k++] = r->res;
    delete r;
  }
  *n_out = k;
  return TC_OK;
}

TC_API tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out) {
  if (!s || !out) {
    set_error("tc_server_get_stats: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->held_bytes = s->held;
  out->pending = (int64_t)s->pending.size();
  return TC_OK;
}

TC_API void tc_server_destroy(tc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto& t : s->builders) t.join();
  s->counter.join();
  for (Request* r : s->ready) {
    if (r->g) tc_free(r->g);
    delete r;
  }
  for (Request* r : s->pending) delete r;
  for (Request* r : s->done) delete r;
  cudaStreamSynchronize(s->count_stream);
  cudaStreamDestroy(s->count_stream);
  cudaDeviceSynchronize();
  cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
