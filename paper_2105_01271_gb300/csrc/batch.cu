// Batching form: many independent decompositions through the single-matrix
// C ABI, overlapped on several CUDA streams (declared in include/lrs.h), and
// the same batch captured as one CUDA graph (lrs_batch_graph_*, below).
//
// Each worker thread owns one lrs_ctx on its own non-blocking stream and its
// own sketch / C-PWR / basis buffers, kept in a per-device pool across runs
// (so a warm executor allocates nothing), and takes items from a shared queue
// ordered largest-first (longest-processing-time-first keeps the tail short).  Every step of an item is the same call
// sequence as the single-matrix path, so results are bit-identical to running
// the items one by one; what changes is that the latency-bound kernels of
// different matrices (pivoted QR steps, small factorizations, host syncs of
// one context) overlap on the GPU.  Cooperative launches from different
// streams are safe: each waits until its whole grid is resident.
#include "common.cuh"
#include "internal.h"

#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace lrs {
namespace {

int64_t grid_points(const lrs_grid& g, bool coarse) {
  int64_t n = 1;
  for (int d = 0; d < g.ndim && d < 3; ++d) n *= coarse ? g.N[d] / (g.s[d] > 0 ? g.s[d] : 1) : g.N[d];
  return n;
}

// cost proxy for the largest-first order: the A-pass bytes plus the sketch QR
double item_cost(const lrs_batch_item& it) {
  const double n = (double)grid_points(it.sketch, false), l = (double)grid_points(it.sketch, true);
  return (double)it.m * n + 64.0 * (double)it.m * l;
}

struct Scratch {
  double *Y = nullptr, *G = nullptr, *Q = nullptr;
  size_t cap = 0;   // doubles per buffer
  ~Scratch() {
    if (Y) cudaFree(Y);
    if (G) cudaFree(G);
    if (Q) cudaFree(Q);
  }
  bool reserve(size_t n) {
    if (n <= cap) return true;
    if (Y) cudaFree(Y);
    if (G) cudaFree(G);
    if (Q) cudaFree(Q);
    Y = G = Q = nullptr;
    cap = 0;
    if (cudaMalloc(&Y, n * 8) != cudaSuccess || cudaMalloc(&G, n * 8) != cudaSuccess ||
        cudaMalloc(&Q, n * 8) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cap = n;
    return true;
  }
};

// one item, SVD then ID, on ctx; returns the item's status
lrs_status run_item(lrs_ctx* ctx, Scratch& sc, lrs_batch_item& it) {
  const int64_t n = grid_points(it.sketch, false), l = grid_points(it.sketch, true);
  const int64_t m = it.m;
  if (!sc.reserve((size_t)(m * (l > m ? l : m)))) return LRS_ENOMEM;
  const lrs_grid* gram = it.q > 0 ? &it.gram : nullptr;
  lrs_status worst = LRS_OK;
  it.r = 0;
  it.err_svd = it.err_id = 0.0;
  if (it.do_svd) {
    int64_t gc = 0;
    lrs_status st = lrs_power_pass(ctx, it.A, it.dtype, m, it.lda, &it.sketch, gram, it.q, 1, it.rtol, it.prec,
                                   sc.Y, l, sc.G, l, &gc);
    if (st) return st;
    const double* Qb = sc.G;
    int64_t ldq = l, r = gc;
    if (it.q == 0) {
      ldq = l < m ? l : m;
      st = lrs_range_find(ctx, sc.G, m, gc, l, it.rtol, sc.Q, ldq, &r);
      if (st) return st;
      Qb = sc.Q;
    }
    it.r = r;
    st = lrs_svd_k(ctx, it.A, it.dtype, m, n, it.lda, Qb, ldq, r, it.k, it.prec, it.U, it.ldu, it.S, it.V, it.ldv,
                   &it.err_svd);
    if (st != LRS_OK && st != LRS_ERANK) return st;
    worst = st;
  }
  if (it.do_id) {
    int64_t gc = 0;
    lrs_status st = lrs_power_pass(ctx, it.A, it.dtype, m, it.lda, &it.sketch, gram, it.q, 0, it.rtol, it.prec,
                                   sc.Y, l, sc.G, l, &gc);
    if (st) return st;
    // gc: the columns of the iterate's form (l, or r for the row-Gram form)
    st = lrs_id_k(ctx, sc.G, m, gc, l, it.k, it.J, it.P, it.ldp, &it.err_id);
    if (st != LRS_OK && st != LRS_ERANK) return st;
    if (st == LRS_ERANK) worst = st;
  }
  return worst;
}

// Worker state kept across runs: a context on its own non-blocking stream and
// the sketch / basis buffers.  Keeping them means a warm executor allocates
// nothing (cudaMalloc / cudaFree of a workspace would synchronise the whole
// device and serialise the workers).  One batch run per device at a time.
struct Worker {
  cudaStream_t stream = nullptr;
  lrs_ctx* ctx = nullptr;
  Scratch sc;
};

struct DevicePool {
  std::mutex run;                       // one lrs_batch_run per device at a time
  std::vector<Worker*> workers;
};

std::mutex g_pools_mu;
std::map<int, DevicePool*> g_pools;

DevicePool* pool_of(int device) {
  std::lock_guard<std::mutex> lk(g_pools_mu);
  DevicePool*& p = g_pools[device];
  if (!p) p = new DevicePool();
  return p;
}

lrs_status grow_pool(DevicePool* p, int device, int n) {
  while ((int)p->workers.size() < n) {
    Worker* w = new Worker();
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete w;
      return LRS_ECUDA;
    }
    if (lrs_create(&w->ctx, device, w->stream) != LRS_OK) {
      cudaStreamDestroy(w->stream);
      delete w;
      return LRS_ECUDA;
    }
    p->workers.push_back(w);
  }
  return LRS_OK;
}

lrs_status run_list(int device, lrs_batch_item* items, const std::vector<int64_t>& order, int32_t n_streams) {
  if (n_streams < 1) n_streams = 1;
  if ((int64_t)n_streams > (int64_t)order.size()) n_streams = (int32_t)std::max<size_t>(1, order.size());
  if (cudaSetDevice(device) != cudaSuccess) return LRS_ECUDA;
  DevicePool* pool = pool_of(device);
  std::lock_guard<std::mutex> run_lock(pool->run);
  const lrs_status gs = grow_pool(pool, device, n_streams);
  if (gs) return gs;
  std::atomic<int64_t> next{0};
  std::vector<lrs_status> wstat((size_t)n_streams, LRS_OK);
  auto work = [&](int wi) {
    if (cudaSetDevice(device) != cudaSuccess) { wstat[wi] = LRS_ECUDA; return; }
    Worker* w = pool->workers[(size_t)wi];
    for (int64_t i = next++; i < (int64_t)order.size(); i = next++) {
      lrs_batch_item& it = items[order[(size_t)i]];
      const int64_t l0 = lrs_launch_count(w->ctx);
      const lrs_status st = run_item(w->ctx, w->sc, it);
      it.status = (int32_t)st;
      it.launches = lrs_launch_count(w->ctx) - l0;
      it.error[0] = 0;
      if (st != LRS_OK && st != LRS_ERANK) {
        snprintf(it.error, sizeof(it.error), "%s", lrs_last_error(w->ctx));
        if (!it.error[0]) snprintf(it.error, sizeof(it.error), "status %d", (int)st);
        if (wstat[wi] == LRS_OK) wstat[wi] = st;
      }
    }
    cudaStreamSynchronize(w->stream);
  };
  std::vector<std::thread> threads;
  for (int wi = 1; wi < n_streams; ++wi) threads.emplace_back(work, wi);
  work(0);
  for (auto& t : threads) t.join();
  for (lrs_status s : wstat)
    if (s != LRS_OK) return s;
  for (size_t i = 0; i < order.size(); ++i) {
    const int32_t s = items[order[i]].status;
    if (s != LRS_OK && s != LRS_ERANK) return (lrs_status)s;
  }
  return LRS_OK;
}

std::vector<int64_t> largest_first(const lrs_batch_item* items, int64_t n, int64_t stride) {
  std::vector<int64_t> order;
  for (int64_t i = 0; i < n; i += stride) order.push_back(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return item_cost(items[a]) > item_cost(items[b]); });
  return order;
}

}  // namespace
}  // namespace lrs

using namespace lrs;

extern "C" {

lrs_status lrs_batch_run(int device, lrs_batch_item* items, int64_t n_items, int32_t n_streams) {
  if (n_items < 0 || (n_items > 0 && !items) || n_streams < 1 || n_streams > 64) return LRS_EINVAL;
  for (int64_t i = 0; i < n_items; ++i) items[i].status = (int32_t)LRS_OK;
  if (n_items == 0) return LRS_OK;
  return run_list(device, items, largest_first(items, n_items, 1), n_streams);
}

lrs_status lrs_batch_autotune(int device, lrs_batch_item* items, int64_t n_items, const int32_t* candidates,
                              int32_t n_candidates, int32_t* best, double* ms_per_item) {
  if (n_items < 1 || !items || !candidates || n_candidates < 1 || !best) return LRS_EINVAL;
  const int64_t stride = n_items >= 32 ? 4 : std::max<int64_t>(1, n_items / 8);
  const std::vector<int64_t> sample = largest_first(items, n_items, stride);
  double best_ms = -1.0;
  *best = candidates[0];
  for (int32_t c = 0; c < n_candidates; ++c) {
    if (candidates[c] < 1 || candidates[c] > 64) return LRS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return LRS_ECUDA;
    cudaDeviceSynchronize();
    const auto t0 = std::chrono::steady_clock::now();
    const lrs_status st = run_list(device, items, sample, candidates[c]);
    cudaDeviceSynchronize();
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st != LRS_OK) return st;
    if (best_ms < 0.0 || ms < best_ms) {
      best_ms = ms;
      *best = candidates[c];
    }
  }
  if (ms_per_item) *ms_per_item = best_ms / (double)sample.size();
  return LRS_OK;
}

lrs_status lrs_batch_release(int device) {
  DevicePool* p = pool_of(device);
  std::lock_guard<std::mutex> run_lock(p->run);
  if (cudaSetDevice(device) != cudaSuccess) return LRS_ECUDA;
  for (Worker* w : p->workers) {
    cudaStreamSynchronize(w->stream);
    lrs_destroy(w->ctx);
    cudaStreamDestroy(w->stream);
    delete w;
  }
  p->workers.clear();
  return LRS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The batch as one CUDA graph (lrs_batch_graph_*).
//
// The single-matrix calls read a few values back to the host as they go
// (ranks that size the next launches, breakdown checks, the bounded waits'
// error flags), which a stream capture cannot contain.  So the batch is run
// once eagerly with every context recording the values it reads back, in
// call order (lrs_ctx::replay = record); then the same call sequence is
// captured with each read-back replaced by the recorded value and a one-
// thread guard kernel that compares the device's value with it when the
// graph runs (replay = capture), and the error estimates computed on the
// device.  Items go to `branches` parallel branches of the graph (one
// context and stream each, largest-first onto the least loaded branch).
// A launch replays the whole batch; an item whose guard finds another value
// (its data now takes another rank or route) is run again eagerly, so the
// results are those of lrs_batch_run in every case.
// ---------------------------------------------------------------------------
struct lrs_batch_graph {
  struct Branch {
    cudaStream_t stream = nullptr;
    lrs_ctx* ctx = nullptr;
    lrs::Scratch sc;
    std::vector<int64_t> items;
    cudaEvent_t done = nullptr;
  };
  int device = 0;
  int64_t n = 0;
  std::vector<Branch*> br;
  std::vector<int> branch_of;
  cudaStream_t origin = nullptr;
  cudaEvent_t start = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<lrs_batch_item> snap;
  std::vector<char> in_graph;
  std::vector<int32_t> rec_status;
  std::vector<int64_t> rec_r, rec_launches;
  int* d_guard = nullptr;
  double* d_err = nullptr;
  int* h_guard = nullptr;
  double* h_err = nullptr;
};

namespace lrs {
namespace {

void graph_free(lrs_batch_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->origin) cudaStreamSynchronize(g->origin);
  for (auto* b : g->br) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->ctx) lrs_destroy(b->ctx);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->start) cudaEventDestroy(g->start);
  if (g->origin) cudaStreamDestroy(g->origin);
  if (g->d_guard) cudaFree(g->d_guard);
  if (g->d_err) cudaFree(g->d_err);
  if (g->h_guard) cudaFreeHost(g->h_guard);
  if (g->h_err) cudaFreeHost(g->h_err);
  cudaGetLastError();
  delete g;
}

// the fields a captured launch bakes in
bool same_item(const lrs_batch_item& a, const lrs_batch_item& b) {
  bool grid = a.sketch.ndim == b.sketch.ndim && a.sketch.kind == b.sketch.kind;
  for (int d = 0; d < 3; ++d) grid = grid && a.sketch.N[d] == b.sketch.N[d] && a.sketch.s[d] == b.sketch.s[d];
  return grid && a.A == b.A && a.dtype == b.dtype && a.m == b.m && a.lda == b.lda && a.q == b.q && a.k == b.k &&
         a.prec == b.prec &&
         a.rtol == b.rtol && a.do_svd == b.do_svd && a.do_id == b.do_id && a.U == b.U && a.ldu == b.ldu &&
         a.S == b.S && a.V == b.V && a.ldv == b.ldv && a.J == b.J && a.P == b.P && a.ldp == b.ldp;
}

void set_error(lrs_batch_item& it, lrs_ctx* ctx, lrs_status st) {
  it.error[0] = 0;
  if (st != LRS_OK && st != LRS_ERANK) {
    snprintf(it.error, sizeof(it.error), "%s", lrs_last_error(ctx));
    if (!it.error[0]) snprintf(it.error, sizeof(it.error), "status %d", (int)st);
  }
}

}  // namespace
}  // namespace lrs

extern "C" {

lrs_status lrs_batch_graph_create(int device, lrs_batch_item* items, int64_t n_items, int32_t branches,
                                  lrs_batch_graph** out) {
  if (!out) return LRS_EINVAL;
  *out = nullptr;
  if (n_items < 1 || !items || branches < 1 || branches > 64) return LRS_EINVAL;
  for (int64_t i = 0; i < n_items; ++i) {
    if (items[i].q != 0) return LRS_EINVAL;           // the graph form takes q = 0 items
    items[i].status = (int32_t)LRS_OK;
  }
  if (cudaSetDevice(device) != cudaSuccess) return LRS_ECUDA;
  lrs_batch_graph* g = new lrs_batch_graph();
  g->device = device;
  g->n = n_items;
  if ((int64_t)branches > n_items) branches = (int32_t)n_items;
  bool ok = cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->start, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc((void**)&g->d_guard, sizeof(int) * (size_t)n_items) == cudaSuccess &&
            cudaMalloc((void**)&g->d_err, 2 * sizeof(double) * (size_t)n_items) == cudaSuccess &&
            cudaMallocHost((void**)&g->h_guard, sizeof(int) * (size_t)n_items) == cudaSuccess &&
            cudaMallocHost((void**)&g->h_err, 2 * sizeof(double) * (size_t)n_items) == cudaSuccess;
  for (int b = 0; ok && b < branches; ++b) {
    auto* br = new lrs_batch_graph::Branch();
    g->br.push_back(br);
    ok = cudaStreamCreateWithFlags(&br->stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&br->done, cudaEventDisableTiming) == cudaSuccess &&
         lrs_create(&br->ctx, device, br->stream) == LRS_OK;
  }
  if (!ok) {
    cudaGetLastError();
    lrs::graph_free(g);
    return LRS_ENOMEM;
  }
  // largest first onto the least loaded branch
  const std::vector<int64_t> order = lrs::largest_first(items, n_items, 1);
  std::vector<double> load((size_t)branches, 0.0);
  g->branch_of.assign((size_t)n_items, 0);
  for (int64_t i : order) {
    int b = 0;
    for (int c = 1; c < branches; ++c)
      if (load[(size_t)c] < load[(size_t)b]) b = c;
    load[(size_t)b] += lrs::item_cost(items[i]);
    g->br[(size_t)b]->items.push_back(i);
    g->branch_of[(size_t)i] = b;
  }
  // ---- the recorded eager run (its results are the batch's results) ----
  g->in_graph.assign((size_t)n_items, 1);
  g->rec_status.assign((size_t)n_items, 0);
  g->rec_r.assign((size_t)n_items, 0);
  g->rec_launches.assign((size_t)n_items, 0);
  auto record = [&](int b) {
    if (cudaSetDevice(device) != cudaSuccess) return;
    auto* br = g->br[(size_t)b];
    br->ctx->replay = lrs::kReplayRecord;
    br->ctx->log.clear();
    for (int64_t i : br->items) {
      lrs_batch_item& it = items[i];
      const size_t mark = br->ctx->log.size();
      const int64_t l0 = lrs_launch_count(br->ctx);
      const lrs_status st = lrs::run_item(br->ctx, br->sc, it);
      it.status = (int32_t)st;
      it.launches = lrs_launch_count(br->ctx) - l0;
      lrs::set_error(it, br->ctx, st);
      g->rec_status[(size_t)i] = (int32_t)st;
      g->rec_r[(size_t)i] = it.r;
      g->rec_launches[(size_t)i] = it.launches;
      if (st != LRS_OK && st != LRS_ERANK) {
        g->in_graph[(size_t)i] = 0;                   // runs eagerly at every launch
        br->ctx->log.resize(mark);
      }
    }
    cudaStreamSynchronize(br->stream);
    br->ctx->replay = 0;
  };
  {
    std::vector<std::thread> th;
    for (int b = 1; b < branches; ++b) th.emplace_back(record, b);
    record(0);
    for (auto& t : th) t.join();
  }
  g->snap.assign(items, items + n_items);
  // ---- capture the same call sequence into one graph ----
  lrs_status res = LRS_OK;
  cudaError_t e = cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_guard, 0, sizeof(int) * (size_t)n_items, g->origin);
  if (e == cudaSuccess) e = cudaEventRecord(g->start, g->origin);
  for (int b = 0; b < branches && e == cudaSuccess && res == LRS_OK; ++b) {
    auto* br = g->br[(size_t)b];
    e = cudaStreamWaitEvent(br->stream, g->start, 0);
    if (e != cudaSuccess) break;
    br->ctx->replay = lrs::kReplayCapture;
    br->ctx->log_pos = 0;
    for (int64_t i : br->items) {
      if (!g->in_graph[(size_t)i]) continue;
      lrs_batch_item copy = g->snap[(size_t)i];
      br->ctx->cap_guard = g->d_guard + i;
      br->ctx->cap_err = g->d_err + 2 * i;
      const lrs_status st = lrs::run_item(br->ctx, br->sc, copy);
      if ((int32_t)st != g->rec_status[(size_t)i]) {
        snprintf(items[i].error, sizeof(items[i].error), "capture: %s", lrs_last_error(br->ctx));
        res = st != LRS_OK && st != LRS_ERANK ? st : LRS_ECUDA;
        break;
      }
    }
    br->ctx->replay = 0;
    if (res == LRS_OK && br->ctx->log_pos != br->ctx->log.size()) res = LRS_ECUDA;
    if (res == LRS_OK) {
      e = cudaEventRecord(br->done, br->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(g->origin, br->done, 0);
    }
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(g->origin, &graph);
  g->graph = graph;
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && res == LRS_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess || res != LRS_OK) {
    cudaGetLastError();
    lrs::graph_free(g);
    return res != LRS_OK ? res : LRS_ECUDA;
  }
  *out = g;
  for (int64_t i = 0; i < n_items; ++i) {
    const int32_t s = items[i].status;
    if (s != LRS_OK && s != LRS_ERANK) return (lrs_status)s;
  }
  return LRS_OK;
}

lrs_status lrs_batch_graph_launch(lrs_batch_graph* g, lrs_batch_item* items, int64_t n_items, int64_t* reruns) {
  if (!g || !items || n_items != g->n) return LRS_EINVAL;
  for (int64_t i = 0; i < n_items; ++i)
    if (!lrs::same_item(items[i], g->snap[(size_t)i])) {
      snprintf(items[i].error, sizeof(items[i].error), "the item differs from the captured one");
      return LRS_EINVAL;
    }
  if (cudaSetDevice(g->device) != cudaSuccess) return LRS_ECUDA;
  cudaError_t e = cudaGraphLaunch(g->exec, g->origin);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->h_guard, g->d_guard, sizeof(int) * (size_t)n_items, cudaMemcpyDeviceToHost, g->origin);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->h_err, g->d_err, 2 * sizeof(double) * (size_t)n_items, cudaMemcpyDeviceToHost,
                        g->origin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->origin);
  if (e != cudaSuccess) return LRS_ECUDA;
  int64_t again = 0;
  lrs_status worst = LRS_OK;
  for (int64_t i = 0; i < n_items; ++i) {
    lrs_batch_item& it = items[i];
    if (g->in_graph[(size_t)i] && g->h_guard[i] == 0) {
      it.status = g->rec_status[(size_t)i];
      it.r = g->rec_r[(size_t)i];
      it.launches = g->rec_launches[(size_t)i];
      it.err_svd = it.do_svd ? g->h_err[2 * i] : 0.0;
      it.err_id = it.do_id ? g->h_err[2 * i + 1] : 0.0;
      it.error[0] = 0;
    } else {
      // a guard found another value (or the item never entered the graph):
      // the single-matrix path, eagerly, on its branch's context
      auto* br = g->br[(size_t)g->branch_of[(size_t)i]];
      const int64_t l0 = lrs_launch_count(br->ctx);
      const lrs_status st = lrs::run_item(br->ctx, br->sc, it);
      it.status = (int32_t)st;
      it.launches = lrs_launch_count(br->ctx) - l0;
      lrs::set_error(it, br->ctx, st);
      cudaStreamSynchronize(br->stream);
      ++again;
    }
    if (it.status != LRS_OK && it.status != LRS_ERANK && worst == LRS_OK) worst = (lrs_status)it.status;
  }
  if (reruns) *reruns = again;
  return worst;
}

void lrs_batch_graph_destroy(lrs_batch_graph* g) { lrs::graph_free(g); }

}  // extern "C"
