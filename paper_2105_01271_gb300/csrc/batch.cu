// Batching form: many independent decompositions through the single-matrix
// C ABI, overlapped on several CUDA streams (declared in include/lrs.h).
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
