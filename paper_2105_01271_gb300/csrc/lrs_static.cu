// lrs_id_k_static: the row ID of lrs_id_k with all of its scratch in one
// file-scope device array instead of the context's cudaMalloc'ed workspace.
//
// For callers that must not allocate device memory while they run: a
// real-time loop whose time budget has no room for cudaMalloc (it can
// synchronise the whole device), or a host framework that owns every device
// allocation and does not let a library make its own.
//
// The array (LRS_ID_STATIC_SCRATCH_BYTES) is part of the library's device
// image: every GPU that loads the library holds it until the process exits.
// Host code cannot pass the array's name to a kernel (on the host it is only a
// stand-in for the symbol), so the first call on a device looks up its device
// address with cudaGetSymbolAddress and keeps it.  Every call shares the
// array; calls whose work overlaps on the GPU (two streams, two contexts) race.
#include "common.cuh"
#include "internal.h"

#include <mutex>

namespace {

static __device__ __align__(256) unsigned char g_id_scratch[LRS_ID_STATIC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void* g_scratch_ptr[256] = {};

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of g_id_scratch on ctx's device (looked up once per device,
// with that device current).
lrs_status static_scratch(lrs_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= 256) return lrs_fail(ctx, LRS_EINVAL, "id_k_static: device %d", ctx->device);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[ctx->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_id_scratch);
    if (e != cudaSuccess || !p)
      return lrs_fail(ctx, LRS_ECUDA, "id_k_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_ptr[ctx->device] = p;
  }
  *out = g_scratch_ptr[ctx->device];
  return LRS_OK;
}

}  // namespace

using namespace lrs;

extern "C" lrs_status lrs_id_k_static(lrs_ctx* ctx, const double* Ysk, int64_t m, int64_t l, int64_t ldy,
                                      int32_t k, int32_t* J, double* P, int64_t ldp, double* err_est) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!Ysk || !J || !P) return lrs_fail(ctx, LRS_EINVAL, "id_k_static: NULL pointer");
  if (m < 1 || l < 1 || k < 1) return lrs_fail(ctx, LRS_EINVAL, "id_k_static: m=%lld l=%lld k=%d", (long long)m, (long long)l, k);
  if (k > m) return lrs_fail(ctx, LRS_EINVAL, "id_k_static: k=%d exceeds m=%lld", k, (long long)m);
  if (k > l) return lrs_fail(ctx, LRS_ERANK, "id_k_static: sketch rank <= l=%lld < k=%d", (long long)l, k);
  if (ldy < l || ldp < k) return lrs_fail(ctx, LRS_EINVAL, "id_k_static: strides too small");
  // exact scratch of this call: copy of the sketch, CPQR outputs and scratch, ||.||^2 partials
  const int64_t nfro = m < (int64_t)ctx->num_sms * 8 ? m : (int64_t)ctx->num_sms * 8;
  const size_t need = a256(8 * (size_t)(m * l)) + a256(4 * (size_t)m) + a256(8 * (size_t)k * m) +
                      a256(8 * (size_t)l * k) + 3 * 256 + a256(8 * (size_t)(nfro > 0 ? nfro : 1)) +
                      cpqr_scratch_bytes(l, m, k, ctx->num_sms);
  if (need > (size_t)LRS_ID_STATIC_SCRATCH_BYTES)
    return lrs_fail(ctx, LRS_EINVAL,
                    "id_k_static: m=%lld, l=%lld, k=%d needs %zu bytes of scratch; the static scratch holds %zu",
                    (long long)m, (long long)l, k, need, (size_t)LRS_ID_STATIC_SCRATCH_BYTES);
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  void* base = nullptr;
  lrs_status st = static_scratch(ctx, &base);
  if (st) return st;

  // Point the context's arena at the static array for this call only; every
  // launcher below takes its scratch with ws_alloc, none grows the arena.
  char* const save_ws = ctx->ws;
  const size_t save_cap = ctx->ws_cap, save_top = ctx->ws_top;
  ctx->ws = (char*)base;
  ctx->ws_cap = (size_t)LRS_ID_STATIC_SCRATCH_BYTES;
  ctx->ws_top = 0;
  auto run = [&]() -> lrs_status {
    double* Mc = (double*)ws_alloc(ctx, 8 * (size_t)(m * l));
    CpqrOut o{};
    o.perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)m);
    o.R = (double*)ws_alloc(ctx, 8 * (size_t)k * m);
    o.V = (double*)ws_alloc(ctx, 8 * (size_t)l * k);
    o.tail2 = (double*)ws_alloc(ctx, 8);
    o.rank = (int32_t*)ws_alloc(ctx, 8);
    double* nrm2 = (double*)ws_alloc(ctx, 8);
    if (!Mc || !o.perm || !o.R || !o.V || !o.tail2 || !o.rank || !nrm2)
      return lrs_fail(ctx, LRS_EINVAL, "id_k_static: static scratch exhausted");
    // Y^T (l x m) column-major is Y's row-major storage; the copy is overwritten
    // in full, and the QR's barrier words are zeroed by its launcher.
    LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(Mc, l * 8, Ysk, ldy * 8, l * 8, m, cudaMemcpyDeviceToDevice, ctx->stream));
    lrs_status s2 = launch_fro2(ctx, Mc, LRS_F64, m, l, l, nrm2);
    if (s2) return s2;
    s2 = launch_cpqr(ctx, Mc, l, m, l, k, 0.0, o);
    if (s2) return s2;
    // scalars come back through the context's pinned host buffer (made at lrs_create)
    double* h = (double*)ctx->host_scratch;
    int32_t* hr = (int32_t*)(h + 2);
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(hr, o.rank, 4, cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h, o.tail2, 8, cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 1, nrm2, 8, cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const int32_t rank = *hr;
    if (rank < k) return lrs_fail(ctx, LRS_ERANK, "id_k_static: sketch rank %d < k=%d", rank, k);
    s2 = launch_id_coeffs(ctx, o.R, k, m, o.perm, J, P, ldp);
    if (s2) return s2;
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (err_est) *err_est = h[1] > 0.0 ? sqrt(fmax(h[0], 0.0) / h[1]) : 0.0;
    return LRS_OK;
  };
  st = run();
  // A call that failed after queueing work (e.g. an occupancy check after the
  // norm kernels) waits for that work, so nothing of it still writes the
  // shared array when the next call, maybe on another stream, begins.
  if (st != LRS_OK) cudaStreamSynchronize(ctx->stream);
  ctx->ws = save_ws;
  ctx->ws_cap = save_cap;
  ctx->ws_top = save_top;
  return st;
}
