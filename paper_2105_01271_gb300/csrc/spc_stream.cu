// Single-read SPC over streamed snapshots (Sec. 3.2, Alg. 3; Sec. 4, Algs. 5
// and 6), declared in include/lrs.h.
//
// The rows of A_f arrive in blocks -- from host memory (a file, a network, a
// simulation on the CPU) or from device memory a simulation fills as it runs --
// and each block is read exactly once:
//     A_c(rows, :) = a_f D                 (the sketch rows, FP64)
//     H^T         += A_c(rows, :)^T a_f    (l x n, FP32; FP64 for FP64 products)
//     ||A_f||_F^2 += ||a_f||_F^2,   rows c-1, 2c-1, ... kept for SPC-ID-ERR.
// Host blocks go through two pinned-or-not staging buffers on a copy stream;
// each staging slot has two events, "copied" (the compute stream waits on it
// before reading the slot) and "free" (the copy stream waits on it before
// overwriting the slot), so the copy of block i+1 overlaps the work on block i.
// The finishers then work on A_c and H^T alone:
//   SVD (Alg. 3): U_r, S_r, V_r of A_c (lrs_sketch_svd); B = S_r^-1 V_r^T H^T
//                 (= U_r^T A_f); U = U_r U_B, S, V = B^T U_B S^-1.
//   ID  (Alg. 5): (J, P) = row ID of A_c; S_f = A_c(J,:) T_r with
//                 T_r = V_r S_r^-2 V_r^T H^T (the operator as printed, through H).
//   ERR (Alg. 6): eps_hat(tau) from the kept rows and the matching rows of A_c.
#include "common.cuh"
#include "internal.h"

#include <math.h>

struct lrs_spc_stream {
  lrs_ctx* ctx = nullptr;
  int32_t dtype = LRS_F32, prec = LRS_PREC_SPLIT_BF16, err_c = 0;
  int64_t m = 0, n = 0, l = 0, block_rows = 0, pushed = 0, blocks = 0;
  lrs::GridDev grid{};
  size_t esz = 4;
  double* Ac = nullptr;         // m x l FP64
  void* Ht = nullptr;           // l x n, FP32 (FP64 when prec is FP64)
  void* stage[2] = {nullptr, nullptr};
  void* kept = nullptr;         // (m / err_c) x n, storage dtype
  double* fro2_parts = nullptr; // one per block
  double* fro2 = nullptr;
  cudaStream_t copy = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  int slot = 0;
  // leading triplets of A_c, computed once per r by the finishers
  int32_t svd_r = 0;
  double *Q = nullptr, *Ur = nullptr, *Sr = nullptr, *Vr = nullptr;
  // single-read C-PWR (lrs_spc_stream_cpwr): the subsample rows W (m x |I|)
  // and Z^T = W^T A_f (|I| x n), FP64; G0 / Gs (m x l) hold the ID's iterate
  int cpwr = 0, skip_ht = 0;
  lrs::GridDev ggrid{};
  int64_t nI = 0;
  double *W = nullptr, *Zt = nullptr, *G0 = nullptr, *Gs = nullptr;
};

namespace lrs {
namespace {

constexpr int32_t kStreamMaxR = 112;
constexpr int64_t kHtSlab = 256;        // rows of H^T per tensor-core product (the TMA A-pass holds <= 256)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void k_div_cols(const double* __restrict__ V, int64_t rows, int64_t r, int64_t ldv,
                           const double* __restrict__ s, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * r) return;
  const int64_t i = e / r, j = e - i * r;
  out[e] = V[i * ldv + j] / s[j];
}

__global__ void k_square(const double* __restrict__ s, int64_t r, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < r) out[e] = s[e] * s[e];
}

void destroy(lrs_spc_stream* s) {
  if (!s) return;
  if (s->ctx) cudaStreamSynchronize(s->ctx->stream);
  if (s->copy) cudaStreamSynchronize(s->copy);
  void* bufs[] = {s->Ac, s->Ht, s->stage[0], s->stage[1], s->kept, s->fro2_parts, s->fro2, s->Q, s->Ur, s->Sr, s->Vr,
                  s->W, s->Zt, s->G0, s->Gs};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int i = 0; i < 2; ++i) {
    if (s->copied[i]) cudaEventDestroy(s->copied[i]);
    if (s->freed[i]) cudaEventDestroy(s->freed[i]);
  }
  if (s->copy) cudaStreamDestroy(s->copy);
  delete s;
}

// the leading r triplets of A_c (cached per r)
lrs_status stream_triplets(lrs_spc_stream* s, int32_t r, double rtol) {
  if (s->svd_r == r) return LRS_OK;
  int64_t rank = 0;
  const int64_t mn = s->m < s->l ? s->m : s->l;
  const lrs_status st = lrs_sketch_svd(s->ctx, s->Ac, s->m, s->l, s->l, rtol, s->Q, mn, r, s->Ur, r, s->Sr, s->Vr, r,
                                       &rank);
  if (st) return st;
  s->svd_r = r;
  return LRS_OK;
}

lrs_status check_complete(lrs_spc_stream* s) {
  if (s->pushed != s->m)
    return lrs_fail(s->ctx, LRS_EINVAL, "spc_stream: %lld of %lld rows pushed", (long long)s->pushed, (long long)s->m);
  return LRS_OK;
}

}  // namespace
}  // namespace lrs

using namespace lrs;

extern "C" {

lrs_status lrs_spc_stream_create(lrs_ctx* ctx, int32_t dtype, int64_t m, const lrs_grid* sketch, int64_t block_rows,
                                 int32_t err_c, int32_t prec, lrs_spc_stream** out) {
  if (!ctx || !out) return LRS_EINVAL;
  ctx->err[0] = 0;
  *out = nullptr;
  GridDev g;
  char why[256];
  if (!grid_from_abi(sketch, &g, why, sizeof why)) return lrs_fail(ctx, LRS_EINVAL, "spc_stream: sketch grid: %s", why);
  if (dtype != LRS_F64 && dtype != LRS_F32 && dtype != LRS_BF16) return lrs_fail(ctx, LRS_EINVAL, "spc_stream: bad dtype");
  if (prec < LRS_PREC_FP64 || prec > LRS_PREC_BF16X3) return lrs_fail(ctx, LRS_EINVAL, "spc_stream: bad prec");
  if (m < 1 || block_rows < 1 || err_c < 0) return lrs_fail(ctx, LRS_EINVAL, "spc_stream: bad sizes");
  if (err_c > 0 && (m / err_c < 1 || m / err_c > 128))
    return lrs_fail(ctx, LRS_EINVAL, "spc_stream: m / err_c = %lld kept rows outside [1, 128]", (long long)(m / err_c));
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_spc_stream* s = new lrs_spc_stream();
  s->ctx = ctx;
  s->dtype = dtype;
  s->prec = prec;
  s->err_c = err_c;
  s->m = m;
  s->n = g.n;
  s->l = g.l;
  s->grid = g;
  s->block_rows = block_rows < m ? block_rows : m;
  s->esz = dtype == LRS_F64 ? 8 : (dtype == LRS_F32 ? 4 : 2);
  const size_t hsz = prec == LRS_PREC_FP64 ? 8 : 4;
  const int64_t mn = m < g.l ? m : g.l;
  const int64_t rmax = mn < kStreamMaxR ? mn : kStreamMaxR;
  bool ok = cudaMalloc((void**)&s->Ac, 8 * (size_t)(m * g.l)) == cudaSuccess &&
            cudaMalloc(&s->Ht, hsz * (size_t)(g.l * g.n)) == cudaSuccess &&
            cudaMalloc((void**)&s->fro2_parts, 8 * (size_t)m) == cudaSuccess &&
            cudaMalloc((void**)&s->fro2, 8) == cudaSuccess &&
            cudaMalloc((void**)&s->Q, 8 * (size_t)(m * mn)) == cudaSuccess &&
            cudaMalloc((void**)&s->Ur, 8 * (size_t)(m * rmax)) == cudaSuccess &&
            cudaMalloc((void**)&s->Sr, 8 * (size_t)rmax) == cudaSuccess &&
            cudaMalloc((void**)&s->Vr, 8 * (size_t)(g.l * rmax)) == cudaSuccess;
  for (int i = 0; ok && i < 2; ++i)
    ok = cudaMalloc(&s->stage[i], s->esz * (size_t)(s->block_rows * g.n)) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->freed[i], cudaEventDisableTiming) == cudaSuccess;
  if (ok && err_c > 0) ok = cudaMalloc(&s->kept, s->esz * (size_t)((m / err_c) * g.n)) == cudaSuccess;
  if (ok) ok = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    destroy(s);
    return lrs_fail(ctx, LRS_ENOMEM, "spc_stream: cannot allocate the stream's buffers (H^T is %zu bytes)",
                    hsz * (size_t)(g.l * g.n));
  }
  *out = s;
  return LRS_OK;
}

void lrs_spc_stream_destroy(lrs_spc_stream* s) { destroy(s); }

lrs_status lrs_spc_stream_reset(lrs_spc_stream* s) {
  if (!s) return LRS_EINVAL;
  // queued work on the old rows may still read the staging buffers: wait for it
  LRS_CUDA_TRY(s->ctx, cudaStreamSynchronize(s->ctx->stream));
  LRS_CUDA_TRY(s->ctx, cudaStreamSynchronize(s->copy));
  s->pushed = 0;
  s->blocks = 0;
  s->svd_r = 0;
  s->slot = 0;
  return LRS_OK;
}

const double* lrs_spc_stream_sketch(const lrs_spc_stream* s) { return s ? s->Ac : nullptr; }

lrs_status lrs_spc_stream_push(lrs_spc_stream* s, const void* rows, int64_t nrows, int64_t ld, int32_t on_device) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  if (!rows || nrows < 1 || ld < s->n) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_push: bad rows");
  if (s->pushed + nrows > s->m)
    return lrs_fail(ctx, LRS_EINVAL, "spc_stream_push: %lld rows beyond m = %lld", (long long)(s->pushed + nrows),
                    (long long)s->m);
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const bool tc = s->prec >= LRS_PREC_SPLIT_BF16;
  const int hf64 = s->prec == LRS_PREC_FP64;
  const int64_t ml = s->l < kHtSlab ? s->l : kHtSlab;
  const size_t need = (tc ? gemm_tc_workspace(ml, s->block_rows, s->prec) +
                                gemm_tc_splitk_workspace(ml, s->n, s->block_rows, ctx->num_sms)
                          : 0) + 65536;
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  const size_t base = ctx->ws_top;
  for (int64_t done = 0; done < nrows;) {
    ctx->ws_top = base;                               // per-block scratch, stream-ordered reuse
    const int64_t b = (nrows - done) < s->block_rows ? (nrows - done) : s->block_rows;
    const int64_t r0 = s->pushed;
    const char* src = (const char*)rows + (size_t)done * (size_t)ld * s->esz;
    const void* blk;
    int64_t ldb;
    const int sl = s->slot;
    if (on_device) {
      blk = src;
      ldb = ld;
    } else {
      // the slot is free once the compute stream has finished with its previous block
      LRS_CUDA_TRY(ctx, cudaStreamWaitEvent(s->copy, s->freed[sl], 0));
      LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(s->stage[sl], (size_t)s->n * s->esz, src, (size_t)ld * s->esz,
                                          (size_t)s->n * s->esz, (size_t)b, cudaMemcpyHostToDevice, s->copy));
      LRS_CUDA_TRY(ctx, cudaEventRecord(s->copied[sl], s->copy));
      LRS_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, s->copied[sl], 0));
      blk = s->stage[sl];
      ldb = s->n;
    }
    // the sketch rows, then H^T += A_c(rows,:)^T a_f, then ||a_f||^2
    st = launch_sketch(ctx, blk, s->dtype, b, ldb, s->grid, s->Ac + (size_t)r0 * (size_t)s->l, s->l);
    if (st) return st;
    const size_t mark = ctx->ws_top;
    if (s->skip_ht) {
      // C-PWR alone (lrs_spc_stream_cpwr with spc_too = 0): no H^T
    } else if (!tc) {
      GemmArgs ga{s->l, s->n, b, s->Ac + (size_t)r0 * (size_t)s->l, LRS_F64, s->l, blk, s->dtype, ldb,
                  s->Ht, hf64, 0, s->n, 1.0, r0 > 0 ? 1 : 0};
      st = launch_gemm_simt(ctx, ga, hf64);
      if (st) return st;
    } else {
      // row slabs of H^T of at most kHtSlab rows: each is one TMA A-pass over the block
      // (the block is re-read per slab, 4 b n bytes, against 8 l n bytes of H^T traffic)
      for (int64_t j0 = 0; j0 < s->l; j0 += kHtSlab) {
        const int64_t mj = (s->l - j0) < kHtSlab ? (s->l - j0) : kHtSlab;
        GemmArgs ga{mj, s->n, b, s->Ac + (size_t)r0 * (size_t)s->l + j0, LRS_F64, s->l, blk, s->dtype, ldb,
                    (float*)s->Ht + (size_t)j0 * (size_t)s->n, 0, 0, s->n, 1.0, r0 > 0 ? 1 : 0};
        st = launch_gemm_tc(ctx, ga, s->prec);
        ctx->ws_top = mark;
        if (st) return st;
      }
    }
    ctx->ws_top = mark;
    if (s->cpwr) {
      // the block's subsample rows, then Z^T += W(rows,:)^T a_f in FP64
      double* Wb = s->W + (size_t)r0 * (size_t)s->nI;
      st = launch_gather(ctx, blk, s->dtype, b, ldb, s->ggrid, Wb, s->nI);
      if (st) return st;
      GemmArgs gz{s->nI, s->n, b, Wb, LRS_F64, s->nI, blk, s->dtype, ldb, s->Zt, 1, 0, s->n, 1.0, r0 > 0 ? 1 : 0};
      st = launch_gemm_simt(ctx, gz, 1);
      if (st) return st;
    }
    st = launch_fro2(ctx, blk, s->dtype, b, s->n, ldb, s->fro2_parts + s->blocks);
    if (st) return st;
    // rows i (global) with (i + 1) % c == 0 are kept for SPC-ID-ERR
    if (s->err_c > 0) {
      const int64_t c = s->err_c;
      const int64_t first = ((r0 + 1 + c - 1) / c) * c - 1;          // smallest kept index >= r0
      if (first < r0 + b && (first + 1) / c <= s->m / c) {
        int64_t cnt = (r0 + b - 1 - first) / c + 1;
        const int64_t kmax = s->m / c - (first + 1) / c + 1;
        if (cnt > kmax) cnt = kmax;
        if (cnt > 0)
          LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync((char*)s->kept + (size_t)((first + 1) / c - 1) * (size_t)s->n * s->esz,
                                              (size_t)s->n * s->esz,
                                              (const char*)blk + (size_t)(first - r0) * (size_t)ldb * s->esz,
                                              (size_t)c * (size_t)ldb * s->esz, (size_t)s->n * s->esz, (size_t)cnt,
                                              cudaMemcpyDeviceToDevice, ctx->stream));
      }
    }
    if (!on_device) {
      LRS_CUDA_TRY(ctx, cudaEventRecord(s->freed[sl], ctx->stream));
      s->slot = 1 - sl;
    }
    s->pushed += b;
    s->blocks += 1;
    s->svd_r = 0;
    done += b;
  }
  return LRS_OK;
}

lrs_status lrs_spc_stream_svd(lrs_spc_stream* s, double rtol, int32_t r, int32_t k, double* U, int64_t ldu, double* S,
                              void* V, int64_t ldv, double* err_est) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  lrs_status st = check_complete(s);
  if (st) return st;
  if (s->skip_ht) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_svd: the stream keeps no H^T (C-PWR only)");
  if (!U || !S || !V || k < 1 || r < k || r > kStreamMaxR) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_svd: bad r / k");
  if (ldu < k || ldv < k) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_svd: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  st = stream_triplets(s, r, rtol);
  if (st) return st;
  const bool tc = s->prec >= LRS_PREC_SPLIT_BF16;
  const int f64 = s->prec == LRS_PREC_FP64;
  const size_t bsz = f64 ? 8 : 4;
  const size_t need = align256(bsz * (size_t)(r * s->n)) + align256(8 * (size_t)(s->l * r)) + 1024 +
                      (tc ? gemm_tc_workspace(r, s->l, s->prec) + gemm_tc_splitk_workspace(r, s->n, s->l, ctx->num_sms)
                          : 0) +
                      svd_from_b_ws(r, s->n, s->m, k, s->prec, ctx->num_sms);
  st = ws_reserve(ctx, need);
  if (st) return st;
  void* B = ws_alloc(ctx, bsz * (size_t)(r * s->n));
  double* Xl = (double*)ws_alloc(ctx, 8 * (size_t)(s->l * r));
  double* f2 = (double*)ws_alloc(ctx, 8);
  if (!B || !Xl || !f2) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (spc_stream_svd)");
  // B = (V_r S_r^-1)^T H^T = S_r^-1 V_r^T A_c^T A_f = U_r^T A_f   (r x n)
  k_div_cols<<<(unsigned)((s->l * r + 255) / 256), 256, 0, ctx->stream>>>(s->Vr, s->l, r, r, s->Sr, Xl);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  const size_t mark = ctx->ws_top;
  st = gemm_prec(ctx, s->prec, r, s->n, s->l, Xl, LRS_F64, r, s->Ht, f64 ? LRS_F64 : LRS_F32, s->n, B, f64, 0, s->n);
  if (st) return st;
  ctx->ws_top = mark;
  st = launch_sum(ctx, s->fro2_parts, (int)s->blocks, f2);
  if (st) return st;
  return svd_from_b(ctx, B, r, s->n, s->Ur, r, s->m, k, s->prec, U, ldu, S, V, ldv, f2, err_est);
}

lrs_status lrs_spc_stream_id(lrs_spc_stream* s, double rtol, int32_t r, int32_t k, int32_t* J, double* P, int64_t ldp,
                             void* Sf, int64_t ldsf, double* err_est) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  lrs_status st = check_complete(s);
  if (st) return st;
  if (s->skip_ht) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_id: the stream keeps no H^T (C-PWR only)");
  if (!J || !P || !Sf || k < 1 || r < k || r > kStreamMaxR) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_id: bad r / k");
  if (ldp < k || ldsf < s->n) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_id: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  st = stream_triplets(s, r, rtol);
  if (st) return st;
  st = lrs_id_k(ctx, s->Ac, s->m, s->l, s->l, k, J, P, ldp, err_est);
  if (st) return st;
  const bool tc = s->prec >= LRS_PREC_SPLIT_BF16;
  const size_t need = 8 * (size_t)(r * k + s->l * k + r) + 4096 +
                      (tc ? gemm_tc_workspace(k, s->l, s->prec) + gemm_tc_splitk_workspace(k, s->n, s->l, ctx->num_sms)
                          : 0);
  st = ws_reserve(ctx, need);
  if (st) return st;
  double* M1 = (double*)ws_alloc(ctx, 8 * (size_t)(r * k));        // S_r^-2 V_r^T A_c(J,:)^T
  double* Wt = (double*)ws_alloc(ctx, 8 * (size_t)(s->l * k));     // V_r M1 = (A_c(J,:) V_r S_r^-2 V_r^T)^T
  double* S2 = (double*)ws_alloc(ctx, 8 * (size_t)r);
  if (!M1 || !Wt || !S2) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (spc_stream_id)");
  k_square<<<(unsigned)((r + 255) / 256), 256, 0, ctx->stream>>>(s->Sr, r, S2);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  st = spc_small_gemm(ctx, r, k, s->l, s->Vr, 1, r, s->Ac, 1, s->l, J, S2, M1, k);
  if (st) return st;
  st = spc_small_gemm(ctx, s->l, k, r, s->Vr, r, 1, M1, k, 1, nullptr, nullptr, Wt, k);
  if (st) return st;
  // S_f = Wt^T H^T = A_c(J,:) T_r   (k x n)
  return gemm_prec(ctx, s->prec, k, s->n, s->l, Wt, LRS_F64, k, s->Ht, s->prec == LRS_PREC_FP64 ? LRS_F64 : LRS_F32,
                   s->n, Sf, s->prec == LRS_PREC_FP64 ? 1 : 0, 0, ldsf);
}

lrs_status lrs_spc_stream_err(lrs_spc_stream* s, const double* taus, int32_t ntau, double* eps_hat) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  lrs_status st = check_complete(s);
  if (st) return st;
  if (s->err_c < 1 || !s->kept) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_err: the stream keeps no rows (err_c = 0)");
  if (!taus || !eps_hat) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_err: NULL pointer");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int64_t c = s->err_c;
  return spc_err_from_rows(ctx, s->kept, s->dtype, s->m / c, s->n, s->n, s->Ac + (size_t)(c - 1) * (size_t)s->l, s->l,
                           c * s->l, (double)c, taus, ntau, eps_hat);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// single-read C-PWR
// ---------------------------------------------------------------------------
extern "C" {

lrs_status lrs_spc_stream_cpwr(lrs_spc_stream* s, const lrs_grid* gram, int32_t spc_too) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  if (s->pushed != 0) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr: rows were already pushed");
  if (s->cpwr) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr: already enabled");
  GridDev g;
  char why[256];
  if (!grid_from_abi(gram, &g, why, sizeof why)) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr: gram grid: %s", why);
  if (g.n != s->n) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr: gram grid has n=%lld, sketch n=%lld",
                                   (long long)g.n, (long long)s->n);
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const size_t bw = 8 * (size_t)(s->m * g.l), bz = 8 * (size_t)(g.l * s->n), bg = 8 * (size_t)(s->m * s->l);
  bool ok = cudaMalloc((void**)&s->W, bw) == cudaSuccess && cudaMalloc((void**)&s->Zt, bz) == cudaSuccess &&
            cudaMalloc((void**)&s->G0, bg) == cudaSuccess && cudaMalloc((void**)&s->Gs, bg) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    double* bufs[] = {s->W, s->Zt, s->G0, s->Gs};
    for (double* b : bufs)
      if (b) cudaFree(b);
    s->W = s->Zt = s->G0 = s->Gs = nullptr;
    return lrs_fail(ctx, LRS_ENOMEM, "spc_stream_cpwr: cannot allocate W and Z^T (%zu + %zu bytes)", bw, bz);
  }
  g.kind = LRS_INJECT;
  s->ggrid = g;
  s->nI = g.l;
  s->cpwr = 1;
  s->skip_ht = spc_too ? 0 : 1;
  return LRS_OK;
}

lrs_status lrs_spc_stream_cpwr_svd(lrs_spc_stream* s, int32_t q, double rtol, int32_t k, double* U, int64_t ldu,
                                   double* S, double* V, int64_t ldv, double* err_est, int64_t* r_out) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  lrs_status st = check_complete(s);
  if (st) return st;
  if (!s->cpwr) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_svd: lrs_spc_stream_cpwr was not called");
  if (!U || !S || !V || k < 1 || q < 1 || q > 16) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_svd: bad q / k");
  if (!(rtol >= 0.0) || rtol >= 1.0) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_svd: rtol=%g", rtol);
  if (ldu < k || ldv < k) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_svd: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int64_t m = s->m, l = s->l, nI = s->nI, n = s->n;
  const int64_t cmax = m < l ? m : l;              // columns of any iterate
  const int64_t tmax = cmax < 128 ? cmax : 128;    // the final basis: Cholesky-QR refinement holds <= 128
  const size_t a = 256;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t o1 = orth_ws_of(m, cmax, ctx->num_sms), o2 = orth_ws_of(nI, cmax, ctx->num_sms);
  size_t need = al(8 * (size_t)(nI * m)) +                       // W^T
                al(8 * (size_t)(m * cmax)) * 4 +                 // Q_np, G, G2, Q_b
                al(8 * (size_t)(nI * cmax)) * 3 +                // T0, T, M
                al(8 * (size_t)(cmax * m)) * 2 +                 // G column-major, Householder vectors
                al(8 * (size_t)(cmax * cmax)) * 3 + al(4 * (size_t)cmax) * 2 + 4 * a +
                al(8 * (size_t)(m * cmax)) + al(8 * (size_t)(nI * cmax)) +   // Q1, M1
                al(8 * (size_t)(tmax * n)) +                                   // B
                cpqr_scratch_bytes(m, cmax, cmax, ctx->num_sms) +
                al(8 * (size_t)ctx->num_sms * (size_t)(tmax * (tmax + 1) / 2)) +
                (o1 > o2 ? o1 : o2) + svd_from_b_ws(tmax, n, m, k < tmax ? k : tmax, LRS_PREC_FP64, ctx->num_sms) +
                65536;
  st = ws_reserve(ctx, need);
  if (st) return st;
  double* WT = (double*)ws_alloc(ctx, 8 * (size_t)(nI * m));
  double* Qnp = (double*)ws_alloc(ctx, 8 * (size_t)(m * cmax));
  double* G = (double*)ws_alloc(ctx, 8 * (size_t)(m * cmax));
  double* G2 = (double*)ws_alloc(ctx, 8 * (size_t)(m * cmax));
  double* T0 = (double*)ws_alloc(ctx, 8 * (size_t)(nI * cmax));
  double* T = (double*)ws_alloc(ctx, 8 * (size_t)(nI * cmax));
  if (!WT || !Qnp || !G || !G2 || !T0 || !T) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpwr_svd)");
  st = launch_transpose(ctx, s->W, m, nI, nI, WT, m);
  if (st) return st;
  const size_t mark = ctx->ws_top;
  int64_t gc = 0, t = 0;
  st = orth_basis(ctx, s->Ac, m, l, l, rtol, Qnp, cmax, &gc);
  if (st) return st;
  ctx->ws_top = mark;
  const double* Gcur = Qnp;
  for (int it = 0; it < q; ++it) {
    // T = QR(W^T G)  (|I| x t), then G = W T  (m x t)
    st = gemm_prec(ctx, LRS_PREC_FP64, nI, gc, m, s->W, LRS_F64, nI, Gcur, LRS_F64, cmax, T0, 1, 0, cmax);
    if (st) return st;
    ctx->ws_top = mark;
    st = orth_basis(ctx, T0, nI, gc, cmax, rtol, T, cmax, &t);
    if (st) return st;
    ctx->ws_top = mark;
    st = gemm_prec(ctx, LRS_PREC_FP64, m, t, nI, WT, LRS_F64, m, T, LRS_F64, cmax, G, 1, 0, cmax);
    if (st) return st;
    ctx->ws_top = mark;
    if (it + 1 < q) {
      st = orth_basis(ctx, G, m, t, cmax, rtol, G2, cmax, &gc);
      if (st) return st;
      ctx->ws_top = mark;
      Gcur = G2;
    }
  }
  if (t > 128) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_svd: %lld directions (the final basis holds <= 128)",
                               (long long)t);
  // Q_b = QR(G): pivoted Householder QR of G (column-major copy), then
  // Q_1 = G(:, piv) R_11^-1 and the same solve on T (M_1 = T(:, piv) R_11^-1)
  double* GT = (double*)ws_alloc(ctx, 8 * (size_t)(t * m));
  CpqrOut o{};
  o.perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)t);
  o.R = (double*)ws_alloc(ctx, 8 * (size_t)(t * t));
  o.V = (double*)ws_alloc(ctx, 8 * (size_t)(m * t));
  o.tail2 = (double*)ws_alloc(ctx, 8);
  o.rank = (int32_t*)ws_alloc(ctx, 8);
  double* Q1 = (double*)ws_alloc(ctx, 8 * (size_t)(m * t));
  double* M1 = (double*)ws_alloc(ctx, 8 * (size_t)(nI * t));
  double* Gr = (double*)ws_alloc(ctx, 8 * (size_t)(t * t));
  double* R2 = (double*)ws_alloc(ctx, 8 * (size_t)(t * t));
  int32_t* p2 = (int32_t*)ws_alloc(ctx, 4 * (size_t)t);
  int32_t* rk2 = (int32_t*)ws_alloc(ctx, 8);
  double* Qb = (double*)ws_alloc(ctx, 8 * (size_t)(m * t));
  double* Mb = (double*)ws_alloc(ctx, 8 * (size_t)(nI * t));
  double* f2 = (double*)ws_alloc(ctx, 8);
  if (!GT || !o.perm || !o.R || !o.V || !o.tail2 || !o.rank || !Q1 || !M1 || !Gr || !R2 || !p2 || !rk2 || !Qb ||
      !Mb || !f2)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpwr_svd)");
  st = launch_transpose(ctx, G, m, t, cmax, GT, m);
  if (st) return st;
  st = launch_cpqr(ctx, GT, m, t, m, t, rtol, o);
  if (st) return st;
  int32_t* h = (int32_t*)ctx->host_scratch;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 48, o.rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const int r = h[48];
  if (r < 1) return lrs_fail(ctx, LRS_ERANK, "spc_stream_cpwr_svd: the C-PWR basis is empty");
  st = launch_trsm_rows(ctx, G, m, cmax, o.perm, o.R, t, r, Q1, t);
  if (st) return st;
  st = launch_trsm_rows(ctx, T, nI, cmax, o.perm, o.R, t, r, M1, t);
  if (st) return st;
  // one Cholesky-QR pass: Q_1^T Q_1 = R_2^T R_2, Q_b = Q_1 R_2^-1, M = M_1 R_2^-1
  st = launch_gram(ctx, Q1, m, r, t, Gr);
  if (st) return st;
  st = launch_pchol(ctx, Gr, r, r, 0.0, 0, p2, R2, r, rk2);
  if (st) return st;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 49, rk2, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (h[49] != r) return lrs_fail(ctx, LRS_ERANK, "spc_stream_cpwr_svd: Cholesky-QR refinement broke down (%d < %d)",
                                  h[49], r);
  st = launch_trsm_rows(ctx, Q1, m, t, nullptr, R2, r, r, Qb, r);
  if (st) return st;
  st = launch_trsm_rows(ctx, M1, nI, t, nullptr, R2, r, r, Mb, r);
  if (st) return st;
  // B = M^T Z^T = Q_b^T A_f  (r x n, FP64)
  double* B = (double*)ws_alloc(ctx, 8 * (size_t)(r * n));
  if (!B) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpwr_svd)");
  const size_t mark2 = ctx->ws_top;
  st = gemm_prec(ctx, LRS_PREC_FP64, r, n, nI, Mb, LRS_F64, r, s->Zt, LRS_F64, n, B, 1, 0, n);
  if (st) return st;
  ctx->ws_top = mark2;
  st = launch_sum(ctx, s->fro2_parts, (int)s->blocks, f2);
  if (st) return st;
  st = svd_from_b(ctx, B, r, n, Qb, r, m, k, LRS_PREC_FP64, U, ldu, S, V, ldv, f2, err_est);
  if (st) return st;
  if (r_out) *r_out = r;
  return r < k ? lrs_fail(ctx, LRS_ERANK, "spc_stream_cpwr_svd: rank r=%d < k=%d", r, k) : LRS_OK;
}

lrs_status lrs_spc_stream_cpwr_id(lrs_spc_stream* s, int32_t q, double rtol, int32_t k, int32_t* J, double* P,
                                  int64_t ldp, double* err_est) {
  if (!s) return LRS_EINVAL;
  lrs_ctx* ctx = s->ctx;
  ctx->err[0] = 0;
  lrs_status st = check_complete(s);
  if (st) return st;
  if (!s->cpwr) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_id: lrs_spc_stream_cpwr was not called");
  if (q < 1 || q > 16) return lrs_fail(ctx, LRS_EINVAL, "spc_stream_cpwr_id: q=%d", q);
  int64_t g0 = 0, gc = 0;
  st = lrs_power_pass_from(ctx, s->Ac, s->l, s->W, s->nI, s->m, s->l, s->nI, q, rtol, LRS_PREC_FP64, s->G0, s->l, &g0,
                           s->Gs, s->l, &gc);
  if (st) return st;
  return lrs_id_k(ctx, s->G0, s->m, g0, s->l, k, J, P, ldp, err_est);
}

}  // extern "C"
