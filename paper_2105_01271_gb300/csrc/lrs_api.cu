// C ABI of the library (include/lrs.h): argument validation, workspace, and
// the order of kernel launches for each call of the paper's path.
#include "common.cuh"
#include "internal.h"

#include <map>
#include <mutex>
#include <utility>

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

lrs_status lrs_fail(lrs_ctx* ctx, lrs_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

namespace lrs {

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

lrs_status ws_reserve(lrs_ctx* ctx, size_t bytes) {
  ctx->ws_top = 0;
  if (ctx->ws_limit && bytes > ctx->ws_limit)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace limit: %zu bytes needed, %zu allowed", bytes, ctx->ws_limit);
  if (bytes <= ctx->ws_cap) return LRS_OK;
  if (ctx->replay == kReplayCapture)
    return lrs_fail(ctx, LRS_EINVAL, "replay: the workspace would grow during a capture (%zu bytes)", bytes);
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
  }
  size_t cap = bytes + (bytes >> 3) + (1 << 20);
  if (cudaMalloc((void**)&ctx->ws, cap) != cudaSuccess) {
    cudaGetLastError();
    return lrs_fail(ctx, LRS_ENOMEM, "cannot allocate a %zu-byte workspace", cap);
  }
  ctx->ws_cap = cap;
  return LRS_OK;
}

lrs_status aux_reserve(lrs_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->aux_cap) return LRS_OK;
  if (ctx->replay == kReplayCapture)
    return lrs_fail(ctx, LRS_EINVAL, "replay: the split-K buffer would grow during a capture (%zu bytes)", bytes);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->aux);
    ctx->aux = nullptr;
    ctx->aux_cap = 0;
  }
  const size_t cap = bytes + (bytes >> 2);
  if (cudaMalloc(&ctx->aux, cap) != cudaSuccess) {
    cudaGetLastError();
    return lrs_fail(ctx, LRS_ENOMEM, "cannot allocate a %zu-byte split-K buffer", cap);
  }
  ctx->aux_cap = cap;
  return LRS_OK;
}

void* ws_alloc(lrs_ctx* ctx, size_t bytes) {
  const size_t b = align256(bytes);
  if (ctx->ws_top + b > ctx->ws_cap) return nullptr;
  void* p = ctx->ws + ctx->ws_top;
  ctx->ws_top += b;
  return p;
}

// bytes of workspace the TSQR reduction levels of an r x n matrix need
static size_t tsqr_ws(int64_t r, int64_t n, size_t tsz) {
  int64_t C = (int64_t)((200 * 1024) / (tsz * (size_t)r));
  if (C > 1024) C = 1024;
  if (C < 1) C = 1;
  size_t b = 0;
  int64_t cur = n;
  for (int guard = 0; guard < 64; ++guard) {
    const int64_t chunks = (cur + C - 1) / C;
    if (chunks <= 1) break;
    cur = chunks * r;
    b += align256(tsz * (size_t)(r * cur));
  }
  return b;
}

// bytes of scratch launch_cpqr takes for a p x c matrix and kmax steps
static size_t cpqr_ws(int64_t p, int64_t c, int64_t kmax) {
  const size_t nbmax = 1024;                      // > any SM count
  size_t b = 0;
  b += 2 * align256(8 * nbmax * (size_t)c);       // per-block partial sums (norms, dots)
  b += 2 * align256(8 * (size_t)c);               // column sums, row buffer
  b += 2 * align256(4 * (size_t)c) + align256((size_t)c);   // positions, done
  b += align256(8 * (size_t)((kmax > 0 ? kmax : 1) * c));  // R by physical column
  b += 4 * align256(8 * nbmax) + 256;             // per-block best, barrier
  // slab storage when a block's rows do not fit in shared memory
  b += align256(8 * (size_t)(p * c + 3 * nbmax * c + 2 * nbmax + p));
  // column-owner form: two candidate columns per block (at most min(c, 1024) blocks)
  b += align256(8 * (size_t)(2 * (c < (int64_t)nbmax ? c : (int64_t)nbmax) * p));
  return b + 4096;
}

// bytes of workspace one orthonormalisation of a p x c matrix needs (either
// route: the Gram route's buffers are released before a CPQR fallback)
static size_t orth_ws(int64_t p, int64_t c, int num_sms) {
  const int64_t kmax = p < c ? p : c;
  // the Gram route only runs for c <= 128 (c here may be an upper bound)
  const size_t g = orth_gram_ws(p, c < 128 ? c : 128, num_sms);
  size_t b = 0;
  b += align256(8 * (size_t)(p * c));            // column-major copy
  b += align256(4 * (size_t)c);                  // perm
  b += align256(8 * (size_t)(kmax * c));         // R
  b += align256(8 * (size_t)(p * kmax));         // V
  b += 2 * 256;                                  // scalars
  b += cpqr_ws(p, c, kmax);
  b += form_q_ws(p, kmax);                       // Q's columns when too long for shared memory
  if (b < g) b = g;
  if (c > 128) {
    const size_t w = orth_wide_ws(p, c, num_sms);
    if (b < w) b = w;
  }
  return b;
}

// Orthonormal basis of the numerical range of Min (p x c, row-major ldi):
// Q (p x r, row-major ldq), r returned through *r_out.  Synchronises.
// intermediate = true: the basis only feeds a product that is orthonormalised
// again (the W^T G step of C-PWR), so a well-conditioned basis of the same
// range suffices (the Gram route then skips its refinement pass).
__global__ void k_abs_diag(const double* __restrict__ R, int64_t ld, int64_t r, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) out[i] = fabs(R[i * ld + i]);
}

lrs_status launch_abs_diag(lrs_ctx* ctx, const double* R, int64_t ld, int64_t r, double* out) {
  if (r < 1) return LRS_OK;
  k_abs_diag<<<(unsigned)((r + 255) / 256), 256, 0, ctx->stream>>>(R, ld, r, out);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// Rt (optional, device, r x c row-major, room for 128 rows): the factor with
// Min ~= Q Rt, columns in their original order (every route: the triangular
// factor of its pivoted QR scattered back, the refinement folded in); not
// written when r > 128.
static lrs_status orth(lrs_ctx* ctx, const double* Min, int64_t p, int64_t c, int64_t ldi,
                       double rtol, double* Q, int64_t ldq, int64_t* r_out, bool intermediate = false,
                       double* rdiag = nullptr, int64_t kcap = 0, double* Rt = nullptr) {
  int64_t kmax = p < c ? p : c;
  if (kcap > 0 && kcap < kmax) kmax = kcap;           // at most kcap pivoted steps (Householder route)
  if (kcap <= 0 && orth_wide_eligible(p, c, rtol, ctx->num_sms)) {
    // wide: left-looking pivoted Cholesky (same pivots and stop rule)
    const size_t mark = ctx->ws_top;
    lrs_status ws = launch_orth_wide(ctx, Min, p, c, ldi, rtol, Q, ldq, r_out, !intermediate, rdiag, Rt);
    ctx->ws_top = mark;
    if (ws != LRS_ERANK) return ws;
  }
  if (kcap <= 0 && orth_gram_eligible(p, c, rtol)) {
    // tall-skinny: pivoted Cholesky of the Gram (same pivots and stop rule)
    const size_t mark = ctx->ws_top;
    lrs_status gs = launch_orth_gram(ctx, Min, p, c, ldi, rtol, Q, ldq, r_out, !intermediate, rdiag, Rt);
    ctx->ws_top = mark;
    if (gs != LRS_ERANK) return gs;
  }
  double* Mc = (double*)ws_alloc(ctx, 8 * (size_t)(p * c));
  CpqrOut o{};
  o.perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)c);
  o.R = (double*)ws_alloc(ctx, 8 * (size_t)(kmax * c));
  o.V = (double*)ws_alloc(ctx, 8 * (size_t)(p * kmax));
  o.tail2 = (double*)ws_alloc(ctx, 8);
  o.rank = (int32_t*)ws_alloc(ctx, 8);
  if (!Mc || !o.perm || !o.R || !o.V || !o.tail2 || !o.rank)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (orth)");
  lrs_status st = launch_transpose(ctx, Min, p, c, ldi, Mc, p);   // column-major copy
  if (st) return st;
  st = launch_cpqr(ctx, Mc, p, c, p, kmax, rtol, o);
  if (st) return st;
  int32_t r = 0;
  if (ctx->replay) {
    const int32_t* d[1] = {o.rank};
    st = replay_ints(ctx, 1, d, &r);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(&r, o.rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (rdiag && r > 0) {
    st = launch_abs_diag(ctx, o.R, c, r, rdiag);
    if (st) return st;
  }
  if (Rt && r > 0 && r <= 128) {       // callers size Rt for 128 rows (wider: no factor written)
    st = launch_rt_scatter(ctx, o.R, c, o.perm, r, c, Rt);
    if (st) return st;
  }
  st = launch_form_q(ctx, o.V, p, r, Q, ldq);
  if (st) return st;
  *r_out = r;
  return LRS_OK;
}

// Raise (never lower) a kernel's dynamic shared-memory limit.  The limit is
// process-wide state of the function (per device), so contexts running on
// other threads -- the batch executor's workers -- must never shrink it
// between another thread's occupancy check and its (cooperative) launch.
lrs_status raise_dyn_smem(lrs_ctx* ctx, const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> cur;
  std::lock_guard<std::mutex> lk(mu);
  size_t& c = cur[{func, ctx->device}];
  if (bytes <= c) return LRS_OK;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess)
    return lrs_fail(ctx, LRS_ECUDA, "cudaFuncSetAttribute(%zu B): %s", bytes, cudaGetErrorString(e));
  c = bytes;
  return LRS_OK;
}

size_t orth_ws_of(int64_t p, int64_t c, int num_sms) { return orth_ws(p, c, num_sms); }

lrs_status orth_basis(lrs_ctx* ctx, const double* M, int64_t p, int64_t c, int64_t ldi, double rtol, double* Q,
                      int64_t ldq, int64_t* r_out, int64_t kcap) {
  return orth(ctx, M, p, c, ldi, rtol, Q, ldq, r_out, false, nullptr, kcap);
}

static lrs_status gemm(lrs_ctx* ctx, int prec, int64_t M, int64_t N, int64_t K, const void* X,
                       int32_t xdt, int64_t ldx, const void* A, int32_t adt, int64_t lda, void* C,
                       int c_f64, int c_trans, int64_t ldc, double alpha = 1.0) {
  GemmArgs g{M, N, K, X, xdt, ldx, A, adt, lda, C, c_f64, c_trans, ldc, alpha};
  if (prec == LRS_PREC_FP64) return launch_gemm_simt(ctx, g, 1);
  if (prec == LRS_PREC_FP32) return launch_gemm_simt(ctx, g, 0);
  return launch_gemm_tc(ctx, g, prec);
}

}  // namespace lrs

using namespace lrs;

// ===========================================================================
extern "C" {

const char* lrs_version(void) { return "lrs 0.1 sm_103a"; }

lrs_status lrs_create(lrs_ctx** out, int device, void* cuda_stream) {
  if (!out) return LRS_EINVAL;
  *out = nullptr;
  lrs_ctx* ctx = new (std::nothrow) lrs_ctx();
  if (!ctx) return LRS_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); delete ctx; return LRS_ECUDA; }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { cudaGetLastError(); delete ctx; return LRS_ECUDA; }
  ctx->num_sms = prop.multiProcessorCount;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  ctx->coop_ok = coop;
  if (cudaMallocHost(&ctx->host_scratch, 4096) != cudaSuccess) { cudaGetLastError(); delete ctx; return LRS_ENOMEM; }
  *out = ctx;
  return LRS_OK;
}

void lrs_destroy(lrs_ctx* ctx) {
  if (!ctx) return;
  if (ctx->kev0) cudaEventDestroy(ctx->kev0);
  if (ctx->kev1) cudaEventDestroy(ctx->kev1);
  if (ctx->ws) { cudaStreamSynchronize(ctx->stream); cudaFree(ctx->ws); }
  if (ctx->aux) { cudaStreamSynchronize(ctx->stream); cudaFree(ctx->aux); }
  if (ctx->side) { cudaStreamSynchronize(ctx->side); cudaStreamDestroy(ctx->side); }
  if (ctx->side_fork) cudaEventDestroy(ctx->side_fork);
  if (ctx->side_join) cudaEventDestroy(ctx->side_join);
  if (ctx->host_scratch) cudaFreeHost(ctx->host_scratch);
  delete ctx;
}

const char* lrs_last_error(const lrs_ctx* ctx) { return ctx ? ctx->err : "NULL context"; }

int64_t lrs_launch_count(const lrs_ctx* ctx) { return ctx ? ctx->launches : 0; }

lrs_status lrs_set_kernel_timing(lrs_ctx* ctx, int32_t on) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (on && !ctx->kev0) {
    LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    LRS_CUDA_TRY(ctx, cudaEventCreate(&ctx->kev0));
    LRS_CUDA_TRY(ctx, cudaEventCreate(&ctx->kev1));
  }
  ctx->time_kernels = on ? 1 : 0;
  ctx->last_kernel_ms = -1.0;
  return LRS_OK;
}

double lrs_last_kernel_ms(const lrs_ctx* ctx) { return ctx ? ctx->last_kernel_ms : -1.0; }

lrs_status lrs_set_workspace_limit(lrs_ctx* ctx, size_t bytes) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  ctx->ws_limit = bytes;
  return LRS_OK;
}

lrs_status lrs_selftest_barrier_timeout(lrs_ctx* ctx, int64_t spin_limit) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (spin_limit < 1 || spin_limit > kSpinLimit)
    return lrs_fail(ctx, LRS_EINVAL, "selftest: spin_limit %lld not in [1, %lld]", (long long)spin_limit,
                    (long long)kSpinLimit);
  if (!ctx->coop_ok) return lrs_fail(ctx, LRS_ECUDA, "device lacks cooperative launch");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, 256);
  if (st) return st;
  return launch_barrier_selftest(ctx, spin_limit);
}

static bool dtype_ok(int32_t dt) { return dt == LRS_F64 || dt == LRS_F32 || dt == LRS_BF16; }
static bool prec_ok(int32_t p) { return p >= LRS_PREC_FP64 && p <= LRS_PREC_BF16X3; }

lrs_status lrs_sketch(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                      const lrs_grid* grid, double* Y, int64_t ldy) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  GridDev g;
  char why[256];
  if (!grid_from_abi(grid, &g, why, sizeof why)) return lrs_fail(ctx, LRS_EINVAL, "sketch: %s", why);
  if (!A || !Y) return lrs_fail(ctx, LRS_EINVAL, "sketch: NULL pointer");
  if (!dtype_ok(dtype)) return lrs_fail(ctx, LRS_EINVAL, "sketch: bad dtype %d", dtype);
  if (m < 1) return lrs_fail(ctx, LRS_EINVAL, "sketch: m=%lld < 1", (long long)m);
  if (lda < g.n || ldy < g.l) return lrs_fail(ctx, LRS_EINVAL, "sketch: lda/ldy too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, 0);
  if (st) return st;
  return launch_sketch(ctx, A, dtype, m, lda, g, Y, ldy);
}

lrs_status lrs_range_find(lrs_ctx* ctx, const double* G, int64_t m, int64_t l, int64_t ldg,
                          double rtol, double* Q, int64_t ldq, int64_t* r_out) {
  return lrs_range_find_diag(ctx, G, m, l, ldg, rtol, Q, ldq, r_out, nullptr);
}

lrs_status lrs_range_find_diag(lrs_ctx* ctx, const double* G, int64_t m, int64_t l, int64_t ldg,
                               double rtol, double* Q, int64_t ldq, int64_t* r_out, double* rdiag) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!G || !Q || !r_out) return lrs_fail(ctx, LRS_EINVAL, "range_find: NULL pointer");
  if (m < 1 || l < 1) return lrs_fail(ctx, LRS_EINVAL, "range_find: empty matrix %lldx%lld", (long long)m, (long long)l);
  if (ldg < l || ldq < (m < l ? m : l)) return lrs_fail(ctx, LRS_EINVAL, "range_find: ldg/ldq too small");
  if (!(rtol >= 0.0) || rtol >= 1.0) return lrs_fail(ctx, LRS_EINVAL, "range_find: rtol=%g not in [0,1)", rtol);
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, orth_ws(m, l, ctx->num_sms));
  if (st) return st;
  return orth(ctx, G, m, l, ldg, rtol, Q, ldq, r_out, false, rdiag);
}

}  // extern "C"

namespace lrs {

// workspace of one C-PWR pass (W, W^T and the loop buffers)
// Iterate widths: with re-orthonormalisation every iterate has at most
// min(m, l) columns (the rank of QR(Y)); without it W^T Y has l.
static int64_t cpwr_width(int64_t m, int64_t l, bool reorth_only) {
  return reorth_only ? (l < m ? l : m) : (l > m ? l : m);
}

static size_t cpwr_ws(lrs_ctx* ctx, int64_t m, int64_t l, int64_t nI, int32_t prec, bool reorth_only = false) {
  const int64_t wmax = cpwr_width(m, l, reorth_only);
  const bool tc = prec >= LRS_PREC_SPLIT_BF16;
  const size_t wsz = tc ? 4 : 8;
  size_t need = 0;
  need += 2 * align256(wsz * (size_t)(m * nI));                     // W, W^T
  need += align256(8 * (size_t)(nI * wmax)) + 2 * align256(8 * (size_t)(m * wmax));
  need += align256(8 * (size_t)(nI * wmax));                        // orthonormal T
  if (tc) need += align256(4 * (size_t)(nI * wmax)) + align256(4 * (size_t)(m * wmax));  // FP32 operands
  // the factor chain of the iterate without re-orthonormalisation: the
  // sketch's factor (at most 128 x l) and six 128 x 128 buffers
  const int64_t lc = l > 128 ? l : 128;
  need += align256(8 * (size_t)(128 * lc)) + 6 * align256(8 * 128 * 128) + 1024;
  const size_t o1 = orth_ws(m, l, ctx->num_sms), o2 = orth_ws(nI, wmax, ctx->num_sms);
  size_t inner = o1 > o2 ? o1 : o2;
  if (tc) {
    // either operand may be the prepared one (the narrow one when it is <= 256 wide)
    const size_t t1 = gemm_tc_workspace(nI > wmax ? nI : wmax, m, prec) +
                      gemm_tc_splitk_workspace(nI > wmax ? nI : wmax, nI > wmax ? nI : wmax, m, ctx->num_sms) +
                      gemm_tc_a_workspace(nI > wmax ? nI : wmax, m, prec);
    const size_t t2 = gemm_tc_workspace(wmax, nI, prec) + gemm_tc_splitk_workspace(wmax, wmax, nI, ctx->num_sms) +
                      gemm_tc_a_workspace(wmax, nI, prec);
    const size_t t = (t1 > t2 ? t1 : t2) + 4096;
    if (t > inner) inner = t;
  }
  return need + inner;
}

// The side stream: work queued there between side_fork() and the join runs
// beside the context's stream; the join makes the context's stream wait for it.
static lrs_status side_fork(lrs_ctx* ctx) {
  if (!ctx->side) {
    LRS_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    LRS_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->side_fork, cudaEventDisableTiming));
    LRS_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->side_join, cudaEventDisableTiming));
  }
  LRS_CUDA_TRY(ctx, cudaEventRecord(ctx->side_fork, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->side, ctx->side_fork, 0));
  return LRS_OK;
}

// joins the side stream back into the context's stream on every exit once armed
struct SideJoin {
  lrs_ctx* ctx;
  bool armed = false;
  explicit SideJoin(lrs_ctx* c) : ctx(c) {}
  void join() {
    if (!armed) return;
    cudaStreamWaitEvent(ctx->stream, ctx->side_join, 0);
    armed = false;
  }
  ~SideJoin() { join(); }
};

// The C-PWR loop of Alg. 7 from a given sketch Y (m x l, ldy) and the
// gathered subsample W (m x nI) and W^T (nI x m), both in wdt: q iterations
// G <- W^T G; [QR]; G <- W G; [QR].  Loop buffers come from the workspace
// above the caller's mark; the result is copied to G (ldg), *g_cols columns.
//
// Gid (optional, with reorth, q > 0): the row ID's iterate WITHOUT
// re-orthonormalisation, (W W^T)^q Y, from the factors of this
// re-orthonormalised loop.  Every QR(.) returns its factor with
// (input) = Q Rt, so
//   (W W^T)^q Y = Q_q M Rt_np,   M = Rt_g,q Rt_t,q ... Rt_g,1 Rt_t,1,
// up to the directions the rank truncation drops.  The row ID depends on the
// iterate only through the inner products of its rows, so Gid receives the
// m x r_np matrix H = Q_q M Ra^T with Ra^T Ra = Rt_np Rt_np^T (Cholesky of
// that small Gram): H H^T = (W W^T)^q Y ((W W^T)^q Y)^T, and the row ID of H
// (its CPQR on r_np instead of l rows of the transpose) is the iterate's.
// All of it runs in FP64 on r x r factors.  Products W^T G and W T in
// FP32-level arithmetic resolve each direction of an ORTHONORMAL iterate to
// FP32 accuracy relative to that direction's own scale, whereas the direct
// (W W^T)^q Y scales direction j by s_j^(2q+1) and buries every direction
// below ~1e-7 of the top under the products' rounding; squaring Rt_np in the
// Gram costs direction j a factor (s_1/s_j)^2 of FP64 rounding, relative to
// its own scale.  *gid_cols returns the columns of Gid (0 when it was not
// written: an iterate of more than 128 directions, or a Cholesky breakdown,
// is left to the caller).
static lrs_status cpwr_loop(lrs_ctx* ctx, const void* W, const void* WT, int64_t m, int64_t l, int64_t nI,
                            const double* Y, int64_t ldy, int32_t q, int32_t reorth, double rtol, int32_t prec,
                            double* G, int64_t ldg, int64_t* g_cols, double* Gid = nullptr, int64_t ldgid = 0,
                            int64_t* gid_cols = nullptr) {
  const int64_t wmax = cpwr_width(m, l, reorth != 0);
  const bool tc = prec >= LRS_PREC_SPLIT_BF16;
  const int32_t wdt = tc ? LRS_F32 : LRS_F64;
  bool chain = Gid && reorth && q > 0;
  if (gid_cols) *gid_cols = 0;
  const int64_t lc = l > 128 ? l : 128;
  const size_t sq = 8 * 128 * 128;
  double* RtY = chain ? (double*)ws_alloc(ctx, 8 * (size_t)(128 * lc)) : nullptr;   // QR(Y)'s factor
  double* Mc = chain ? (double*)ws_alloc(ctx, sq) : nullptr;                          // the product M so far
  double* Mn = chain ? (double*)ws_alloc(ctx, sq) : nullptr;
  double* Rf = chain ? (double*)ws_alloc(ctx, sq) : nullptr;                          // one factor
  double* Ga = chain ? (double*)ws_alloc(ctx, sq) : nullptr;
  double* Ra = chain ? (double*)ws_alloc(ctx, sq) : nullptr;
  double* Kf = chain ? (double*)ws_alloc(ctx, sq) : nullptr;
  int32_t* cperm = chain ? (int32_t*)ws_alloc(ctx, 4 * 128) : nullptr;
  int32_t* crank = chain ? (int32_t*)ws_alloc(ctx, 8) : nullptr;
  if (chain && (!RtY || !Mc || !Mn || !Rf || !Ga || !Ra || !Kf || !cperm || !crank))
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (power_pass chain)");
  int64_t rnp = 0, mrows = 0;          // columns of M (= rank of QR(Y)); rows of M so far
  // M <- Rf (rr x mrows) M, the first factor taken as it is
  auto chain_mul = [&](int64_t rr) -> lrs_status {
    if (mrows == 0) {
      double* t = Mc; Mc = Rf; Rf = t;
    } else {
      lrs_status s2 = spc_small_gemm(ctx, rr, rnp, mrows, Rf, mrows, 1, Mc, rnp, 1, nullptr, nullptr, Mn, rnp);
      if (s2) return s2;
      double* t = Mc; Mc = Mn; Mn = t;
    }
    mrows = rr;
    return LRS_OK;
  };
  double* Tm = (double*)ws_alloc(ctx, 8 * (size_t)(nI * wmax));
  double* To = (double*)ws_alloc(ctx, 8 * (size_t)(nI * wmax));
  double* Ga_ = (double*)ws_alloc(ctx, 8 * (size_t)(m * wmax));
  double* Gb_ = (double*)ws_alloc(ctx, 8 * (size_t)(m * wmax));
  float* T32 = tc ? (float*)ws_alloc(ctx, 4 * (size_t)(nI * wmax)) : nullptr;
  float* G32 = tc ? (float*)ws_alloc(ctx, 4 * (size_t)(m * wmax)) : nullptr;
  if (!Tm || !To || !Ga_ || !Gb_ || (tc && (!T32 || !G32)))
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (power_pass)");
  const size_t mark = ctx->ws_top;
  lrs_status st = LRS_OK;
  // starting block: Q_np = QR(A_f D) with re-orthonormalisation, else A_f D
  int64_t gc = l;
  const double* Gcur = Y;
  int64_t ldcur = ldy;
  if (reorth) {
    // Q_np only feeds W^T Q_np, which is orthonormalised again: a
    // well-conditioned basis of the same range suffices (no refinement pass)
    st = orth(ctx, Y, m, l, ldy, rtol, Ga_, wmax, &gc, /*intermediate=*/q > 0, nullptr, 0, chain ? RtY : nullptr);
    if (st) return st;
    ctx->ws_top = mark;
    Gcur = Ga_; ldcur = wmax;
    rnp = gc;                          // Y = Q_np Rt_np
    if (gc > 128) chain = false;       // no factor chain beyond 128 directions
  }
  // The chain's Cholesky, Ra^T Ra = Rt_np Rt_np^T (rnp x rnp, plain FP64),
  // needs only QR(Y)'s factor: it runs on the side stream (one block, no
  // workspace) while the loop's products and QRs run on the context's stream.
  SideJoin side(ctx);
  if (chain) {
    st = side_fork(ctx);
    if (st) return st;
    cudaStream_t main_stream = ctx->stream;
    ctx->stream = ctx->side;
    lrs_status s1 = spc_small_gemm(ctx, rnp, rnp, l, RtY, l, 1, RtY, 1, l, nullptr, nullptr, Ga, rnp);
    lrs_status s2 = s1 ? s1 : launch_pchol(ctx, Ga, (int)rnp, (int)rnp, 0.0, 0, cperm, Ra, rnp, crank);
    const cudaError_t e = cudaEventRecord(ctx->side_join, ctx->side);
    ctx->stream = main_stream;
    side.armed = true;
    if (s2) return s2;
    if (e != cudaSuccess) return lrs_fail(ctx, LRS_ECUDA, "power_pass: side stream: %s", cudaGetErrorString(e));
  }
  for (int it = 0; it < q; ++it) {
    // T = W^T G   (nI x gc)
    if (tc) {
      st = launch_to_f32(ctx, Gcur, m, gc, ldcur, G32, gc);
      if (st) return st;
      // the orthonormalisation reads FP64; the next product reads FP32.  T^T =
      // G^T W: the narrow G is the prepared operand and the wide W streams
      // through the TMA A-pass once; T is stored transposed (n-major) directly
      // (for a wide G, gc > 256, the older kernel with W prepared tiles better)
      const bool narrow = gc <= 256;
      if (reorth && narrow) st = gemm(ctx, prec, gc, nI, m, G32, LRS_F32, gc, W, wdt, nI, Tm, 1, 1, gc);
      else if (narrow) st = gemm(ctx, prec, gc, nI, m, G32, LRS_F32, gc, W, wdt, nI, T32, 0, 1, gc);
      else if (reorth) st = gemm(ctx, prec, nI, gc, m, W, wdt, nI, G32, LRS_F32, gc, Tm, 1, 0, gc);
      else st = gemm(ctx, prec, nI, gc, m, W, wdt, nI, G32, LRS_F32, gc, T32, 0, 0, gc);
    } else {
      st = gemm(ctx, prec, nI, gc, m, W, wdt, nI, Gcur, LRS_F64, ldcur, Tm, 1, 0, gc);
    }
    if (st) return st;
    ctx->ws_top = mark;
    int64_t tc_cols = gc;
    const void* Tcur = tc ? (const void*)T32 : (const void*)Tm;
    int32_t tdt = tc ? LRS_F32 : LRS_F64;
    if (reorth) {
      st = orth(ctx, Tm, nI, gc, gc, rtol, To, gc, &tc_cols, /*intermediate=*/true, nullptr, 0, chain ? Rf : nullptr);
      if (st) return st;
      ctx->ws_top = mark;
      if (chain) { st = chain_mul(tc_cols); if (st) return st; }
      if (tc) {
        st = launch_to_f32(ctx, To, nI, tc_cols, gc, T32, gc);
        if (st) return st;
        Tcur = T32; tdt = LRS_F32;
      } else {
        Tcur = To; tdt = LRS_F64;
      }
    }
    // G = W T   (m x tc_cols)  computed as (W^T)^T T; tensor-core modes form
    // G^T = T^T W^T with the narrow T prepared and W^T streamed, stored transposed
    double* Gn = (Gcur == Ga_) ? Gb_ : Ga_;
    if (tc && tc_cols <= 256) st = gemm(ctx, prec, tc_cols, m, nI, Tcur, tdt, gc, WT, wdt, m, Gn, 1, 1, wmax);
    else st = gemm(ctx, prec, m, tc_cols, nI, WT, wdt, m, Tcur, tdt, gc, Gn, 1, 0, wmax);
    if (st) return st;
    ctx->ws_top = mark;
    if (reorth) {
      double* Go = (Gn == Ga_) ? Gb_ : Ga_;
      // only the last iterate is returned as the orthonormal basis G_q
      st = orth(ctx, Gn, m, tc_cols, wmax, rtol, Go, wmax, &gc, /*intermediate=*/it + 1 < q, nullptr, 0,
                chain ? Rf : nullptr);
      if (st) return st;
      ctx->ws_top = mark;
      if (chain) { st = chain_mul(gc); if (st) return st; }
      Gcur = Go;
    } else {
      gc = tc_cols;
      Gcur = Gn;
    }
    ldcur = wmax;
  }
  LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(G, ldg * 8, Gcur, ldcur * 8, gc * 8, m, cudaMemcpyDeviceToDevice, ctx->stream));
  *g_cols = gc;
  side.join();
  if (chain && mrows == gc) {
    // Ra (from the side stream) with Ra^T Ra = Rt_np Rt_np^T
    int32_t* hr = (int32_t*)ctx->host_scratch;
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(hr + 46, crank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (hr[46] == (int32_t)rnp) {
      // H = Q_q (M Ra^T): m x rnp
      st = spc_small_gemm(ctx, gc, rnp, rnp, Mc, rnp, 1, Ra, 1, rnp, nullptr, nullptr, Kf, rnp);
      if (st) return st;
      st = spc_small_gemm(ctx, m, rnp, gc, Gcur, ldcur, 1, Kf, rnp, 1, nullptr, nullptr, Gid, ldgid);
      if (st) return st;
      if (gid_cols) *gid_cols = rnp;
    }
  }
  return LRS_OK;
}

// validation shared by lrs_power_pass and lrs_power_pass2
static lrs_status power_pass_check(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                                   const lrs_grid* sketch, const lrs_grid* gram, int32_t q, double rtol,
                                   int32_t prec, GridDev* gs, GridDev* gg) {
  char why[256];
  if (!grid_from_abi(sketch, gs, why, sizeof why)) return lrs_fail(ctx, LRS_EINVAL, "power_pass: sketch grid: %s", why);
  if (!A) return lrs_fail(ctx, LRS_EINVAL, "power_pass: NULL pointer");
  if (!dtype_ok(dtype) || !prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "power_pass: bad dtype/prec");
  if (m < 1 || q < 0 || q > 16) return lrs_fail(ctx, LRS_EINVAL, "power_pass: m=%lld q=%d", (long long)m, q);
  if (lda < gs->n) return lrs_fail(ctx, LRS_EINVAL, "power_pass: lda too small");
  if (!(rtol >= 0.0) || rtol >= 1.0) return lrs_fail(ctx, LRS_EINVAL, "power_pass: rtol=%g not in [0,1)", rtol);
  if (q > 0) {
    if (!grid_from_abi(gram, gg, why, sizeof why)) return lrs_fail(ctx, LRS_EINVAL, "power_pass: gram grid: %s", why);
    if (gg->n != gs->n) return lrs_fail(ctx, LRS_EINVAL, "power_pass: gram grid has n=%lld, sketch n=%lld", (long long)gg->n, (long long)gs->n);
  }
  return LRS_OK;
}

// the one touch of A_f: the sketch Y, and with q > 0 the subsample W and
// W^T (FP32 for the tensor-core modes, else FP64) in the workspace
static lrs_status touch(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda, const GridDev& gs,
                        const GridDev& gg, int32_t q, int32_t prec, double* Y, int64_t ldy, void** W, void** WT) {
  lrs_status st = launch_sketch(ctx, A, dtype, m, lda, gs, Y, ldy);
  if (st || q == 0) return st;
  const int64_t nI = gg.l;
  const bool tc = prec >= LRS_PREC_SPLIT_BF16;
  const size_t wsz = tc ? 4 : 8;
  *W = ws_alloc(ctx, wsz * (size_t)(m * nI));
  *WT = ws_alloc(ctx, wsz * (size_t)(m * nI));
  if (!*W || !*WT) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (power_pass)");
  if (tc) return launch_gather32_both(ctx, A, dtype, m, lda, gg, (float*)*W, nI, (float*)*WT, m);
  st = launch_gather(ctx, A, dtype, m, lda, gg, (double*)*W, nI);
  if (st) return st;
  return launch_transpose(ctx, (const double*)*W, m, nI, nI, (double*)*WT, m);
}

// Both C-PWR iterates from the touched Y, W, W^T (lrs_power_pass2 after its
// touch; lrs_power_pass_from).  The SVD's re-orthonormalised loop; its
// factors also give the ID's iterate (the same result as lrs_power_pass with
// reorth = 0).  FP64 products, or a chain wider than 128 directions: the ID's
// loop runs on its own.  The loop buffers are reused; W and W^T stay below
// the mark.
static lrs_status pass2_from(lrs_ctx* ctx, const void* W, const void* WT, int64_t m, int64_t l, int64_t nI,
                             const double* Y, int64_t ldy, int32_t q, double rtol, int32_t prec, double* G0,
                             int64_t ldg0, int64_t* g0_cols, double* G, int64_t ldg, int64_t* g_cols) {
  if (q == 0) {
    LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(G0, ldg0 * 8, Y, ldy * 8, l * 8, m, cudaMemcpyDeviceToDevice, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(G, ldg * 8, Y, ldy * 8, l * 8, m, cudaMemcpyDeviceToDevice, ctx->stream));
    *g_cols = l;
    *g0_cols = l;
    return LRS_OK;
  }
  const size_t mark = ctx->ws_top;
  int64_t gid = 0;
  lrs_status st = cpwr_loop(ctx, W, WT, m, l, nI, Y, ldy, q, 1, rtol, prec, G, ldg, g_cols,
                            prec != LRS_PREC_FP64 ? G0 : nullptr, ldg0, &gid);
  if (st) return st;
  ctx->ws_top = mark;
  *g0_cols = gid;
  if (gid == 0) {
    st = cpwr_loop(ctx, W, WT, m, l, nI, Y, ldy, q, 0, rtol, prec, G0, ldg0, g0_cols);
    if (st) return st;
  }
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

}  // namespace lrs

extern "C" {

lrs_status lrs_power_pass(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                          const lrs_grid* sketch, const lrs_grid* gram, int32_t q, int32_t reorth,
                          double rtol, int32_t prec, double* Y, int64_t ldy, double* G, int64_t ldg,
                          int64_t* g_cols) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  GridDev gs, gg;
  lrs_status st = power_pass_check(ctx, A, dtype, m, lda, sketch, gram, q, rtol, prec, &gs, &gg);
  if (st) return st;
  if (!Y || !G || !g_cols) return lrs_fail(ctx, LRS_EINVAL, "power_pass: NULL pointer");
  if (ldy < gs.l || ldg < gs.l) return lrs_fail(ctx, LRS_EINVAL, "power_pass: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int64_t l = gs.l;
  const int64_t nI = q > 0 ? gg.l : 0;
  // a re-orthonormalised pass keeps every iterate within min(m, l) columns
  st = ws_reserve(ctx, q > 0 ? cpwr_ws(ctx, m, l, nI, prec, reorth != 0) + align256(8 * (size_t)(m * l)) : 0);
  if (st) return st;
  void *W = nullptr, *WT = nullptr;
  st = touch(ctx, A, dtype, m, lda, gs, gg, q, prec, Y, ldy, &W, &WT);
  if (st) return st;
  if (q == 0) {
    LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(G, ldg * 8, Y, ldy * 8, l * 8, m, cudaMemcpyDeviceToDevice, ctx->stream));
    *g_cols = l;
    return LRS_OK;
  }
  if (!reorth && prec != LRS_PREC_FP64) {
    // the iterate without re-orthonormalisation from the factors of the
    // re-orthonormalised loop (cpwr_loop); its basis goes to scratch
    double* Gs = (double*)ws_alloc(ctx, 8 * (size_t)(m * l));
    if (!Gs) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (power_pass)");
    const size_t mark = ctx->ws_top;
    int64_t gq = 0, gid = 0;
    st = cpwr_loop(ctx, W, WT, m, l, nI, Y, ldy, q, 1, rtol, prec, Gs, l, &gq, G, ldg, &gid);
    if (st) return st;
    ctx->ws_top = mark;
    if (gid > 0) {
      *g_cols = gid;
      LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      return LRS_OK;
    }
  }
  st = cpwr_loop(ctx, W, WT, m, l, nI, Y, ldy, q, reorth, rtol, prec, G, ldg, g_cols);
  if (st) return st;
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

lrs_status lrs_power_pass2(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                           const lrs_grid* sketch, const lrs_grid* gram, int32_t q, double rtol, int32_t prec,
                           double* Y, int64_t ldy, double* G0, int64_t ldg0, int64_t* g0_cols, double* G,
                           int64_t ldg, int64_t* g_cols) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  GridDev gs, gg;
  lrs_status st = power_pass_check(ctx, A, dtype, m, lda, sketch, gram, q, rtol, prec, &gs, &gg);
  if (st) return st;
  if (!Y || !G || !G0 || !g_cols || !g0_cols) return lrs_fail(ctx, LRS_EINVAL, "power_pass2: NULL pointer");
  if (ldy < gs.l || ldg < gs.l || ldg0 < gs.l) return lrs_fail(ctx, LRS_EINVAL, "power_pass2: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int64_t l = gs.l;
  const int64_t nI = q > 0 ? gg.l : 0;
  st = ws_reserve(ctx, q > 0 ? cpwr_ws(ctx, m, l, nI, prec) : 0);
  if (st) return st;
  void *W = nullptr, *WT = nullptr;
  st = touch(ctx, A, dtype, m, lda, gs, gg, q, prec, Y, ldy, &W, &WT);
  if (st) return st;
  return lrs::pass2_from(ctx, W, WT, m, l, nI, Y, ldy, q, rtol, prec, G0, ldg0, g0_cols, G, ldg, g_cols);
}

lrs_status lrs_touch(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda, const lrs_grid* sketch,
                     const lrs_grid* gram, int32_t prec, double* Y, int64_t ldy, void* W, int64_t ldw) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  GridDev gs, gg;
  lrs_status st = power_pass_check(ctx, A, dtype, m, lda, sketch, gram, gram ? 1 : 0, 0.0, prec, &gs, &gg);
  if (st) return st;
  if (!Y || (gram && !W)) return lrs_fail(ctx, LRS_EINVAL, "touch: NULL pointer");
  if (ldy < gs.l || (gram && ldw < gg.l)) return lrs_fail(ctx, LRS_EINVAL, "touch: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  st = launch_sketch(ctx, A, dtype, m, lda, gs, Y, ldy);
  if (st || !gram) return st;
  if (prec >= LRS_PREC_SPLIT_BF16)
    return launch_gather32_both(ctx, A, dtype, m, lda, gg, (float*)W, ldw, nullptr, 0);
  return launch_gather(ctx, A, dtype, m, lda, gg, (double*)W, ldw);
}

lrs_status lrs_power_pass_from(lrs_ctx* ctx, const double* Y, int64_t ldy, const void* W, int64_t ldw, int64_t m,
                               int64_t l, int64_t nI, int32_t q, double rtol, int32_t prec, double* G0,
                               int64_t ldg0, int64_t* g0_cols, double* G, int64_t ldg, int64_t* g_cols) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!Y || !G || !G0 || !g_cols || !g0_cols || (q > 0 && !W))
    return lrs_fail(ctx, LRS_EINVAL, "power_pass_from: NULL pointer");
  if (!prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "power_pass_from: bad prec");
  if (m < 1 || l < 1 || q < 0 || q > 16 || (q > 0 && nI < 1))
    return lrs_fail(ctx, LRS_EINVAL, "power_pass_from: m=%lld l=%lld |I|=%lld q=%d", (long long)m, (long long)l,
                    (long long)nI, q);
  if (!(rtol >= 0.0) || rtol >= 1.0) return lrs_fail(ctx, LRS_EINVAL, "power_pass_from: rtol=%g not in [0,1)", rtol);
  if (ldy < l || ldg < l || ldg0 < l || (q > 0 && ldw < nI))
    return lrs_fail(ctx, LRS_EINVAL, "power_pass_from: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, q > 0 ? cpwr_ws(ctx, m, l, nI, prec) : 0);
  if (st) return st;
  const void* Wc = W;
  void* WT = nullptr;
  if (q > 0) {
    // the loop takes W with row stride |I| and its transpose
    const bool tc = prec >= LRS_PREC_SPLIT_BF16;
    const size_t wsz = tc ? 4 : 8;
    if (ldw != nI) {
      void* Wd = ws_alloc(ctx, wsz * (size_t)(m * nI));
      if (!Wd) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (power_pass_from)");
      LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(Wd, nI * wsz, W, ldw * wsz, nI * wsz, m, cudaMemcpyDeviceToDevice,
                                          ctx->stream));
      Wc = Wd;
    }
    WT = ws_alloc(ctx, wsz * (size_t)(m * nI));
    if (!WT) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (power_pass_from)");
    st = tc ? launch_transpose32(ctx, (const float*)Wc, m, nI, nI, (float*)WT, m)
            : launch_transpose(ctx, (const double*)Wc, m, nI, nI, (double*)WT, m);
    if (st) return st;
  }
  return lrs::pass2_from(ctx, Wc, WT, m, l, nI, Y, ldy, q, rtol, prec, G0, ldg0, g0_cols, G, ldg, g_cols);
}

}  // extern "C"

namespace lrs {

__global__ void k_unpermute_r(const double* __restrict__ R, const int32_t* __restrict__ perm, int64_t rank, int64_t r,
                              double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * r) return;
  const int64_t i = e / r, j = e - i * r;                 // out(i, perm[j]) = R(i, j)
  out[i * r + perm[j]] = i < rank ? R[i * r + j] : 0.0;
}

// R (r x r, row-major) with B^T = Q R for B (r x n FP64 row-major): the
// cooperative pivoted QR of B^T (column-major B^T is B's row-major storage)
// run to r steps, its columns returned to their original order
static lrs_status r_of_bt_cpqr(lrs_ctx* ctx, const double* B, int64_t r, int64_t n, double* Rout) {
  if (n < r) return LRS_ERANK;
  double* Mc = (double*)ws_alloc(ctx, 8 * (size_t)(n * r));
  CpqrOut o{};
  o.perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)r);
  o.R = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
  o.V = (double*)ws_alloc(ctx, 8 * (size_t)(n * r));
  o.tail2 = (double*)ws_alloc(ctx, 8);
  o.rank = (int32_t*)ws_alloc(ctx, 8);
  if (!Mc || !o.perm || !o.R || !o.V || !o.tail2 || !o.rank) return LRS_ERANK;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(Mc, B, 8 * (size_t)(n * r), cudaMemcpyDeviceToDevice, ctx->stream));
  lrs_status st = launch_cpqr(ctx, Mc, n, r, n, r, 0.0, o);
  if (st) return st;
  int32_t rank = 0;
  if (ctx->replay) {
    const int32_t* d[1] = {o.rank};
    st = replay_ints(ctx, 1, d, &rank);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(&rank, o.rank, 4, cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  k_unpermute_r<<<(unsigned)((r * r + 255) / 256), 256, 0, ctx->stream>>>(o.R, o.perm, rank, r, Rout);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// The rest of the SVD once B's right singular structure is known: Vr (r x r,
// row-major, columns = U_B) and sv (r, descending).  U = Q U_B(:, :kk) with
// the sign convention, S, V = B^T U_B(:, :kk) S^-1 for B r x n (row stride n;
// FP64 when prec is FP64, else FP32), err_est from the tail of sv and fro2.
static lrs_status svd_finish(lrs_ctx* ctx, double* Vr, const double* sv, int64_t r, int64_t kk, const double* Q,
                             int64_t ldq, int64_t m, const void* B, int64_t n, int32_t prec, double* U, int64_t ldu,
                             double* S, void* V, int64_t ldv, const double* fro2, double* err_est) {
  const int f64 = prec == LRS_PREC_FP64;
  double* Wk = (double*)ws_alloc(ctx, 8 * (size_t)(r * kk));
  double* sgn = (double*)ws_alloc(ctx, 8 * (size_t)kk);
  if (!Wk || !sgn) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd)");
  // U = Q Vr(:, :kk): m x kk x r in FP64, 16 x 16 output tiles over the SMs
  lrs_status st = spc_small_gemm(ctx, m, kk, r, Q, ldq, 1, Vr, r, 1, nullptr, nullptr, U, ldu);
  if (st) return st;
  // sign convention on U, then V = B^T Vr_k diag(sign) S_k^{-1} carries the same signs
  st = launch_sign_fix(ctx, U, m, kk, ldu, sgn);
  if (st) return st;
  st = launch_scale_cols(ctx, Vr, r, r, sv, sgn, kk, Wk, kk);
  if (st) return st;
  if (prec >= LRS_PREC_SPLIT_BF16 && !f64) {
    // V^T (kk x n) = Wk^T B on the tensor cores (B streamed once, V stored
    // n-major), three BF16 pieces per operand: V carries the reconstruction,
    // so it keeps FP32-level accuracy whatever the A-pass precision
    GemmArgs gv{kk, n, r, Wk, LRS_F64, kk, B, LRS_F32, n, V, 0, 1, ldv, 1.0};
    st = apass_eligible(gv, LRS_PREC_BF16X3) ? launch_gemm_tc(ctx, gv, LRS_PREC_BF16X3)
                                             : gemm(ctx, LRS_PREC_FP32, n, kk, r, B, LRS_F32, n, Wk, LRS_F64, kk,
                                                    V, 0, 0, ldv);
  } else {
    st = gemm(ctx, f64 ? LRS_PREC_FP64 : LRS_PREC_FP32, n, kk, r, B, f64 ? LRS_F64 : LRS_F32, n, Wk,
              LRS_F64, kk, V, f64, 0, ldv);
  }
  if (st) return st;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(S, sv, 8 * (size_t)kk, cudaMemcpyDeviceToDevice, ctx->stream));
  if (err_est && ctx->replay == kReplayCapture) {
    // captured: computed on the device into the decomposition's slot
    *err_est = 0.0;
    st = launch_err_tail(ctx, sv, r, kk, fro2, ctx->cap_err);
    if (st) return st;
  } else if (err_est) {
    double* h = (double*)ctx->host_scratch;
    if (fro2) LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h, fro2, 8, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<double> s_h((size_t)r);
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(s_h.data(), sv, 8 * (size_t)r, cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    // energy of B beyond rank k, summed smallest first
    double tail = 0.0;
    for (int64_t i = r - 1; i >= kk; --i) tail += s_h[(size_t)i] * s_h[(size_t)i];
    const double f = fro2 ? h[0] : 0.0;
    *err_est = f > 0.0 ? sqrt(tail / f) : 0.0;
  }
  return LRS_OK;
}

// The TSQR tree halves its height per level only while a leaf tile holds at
// least 2r rows; wider, it degenerates into many levels of nearly the full
// height (the same rows again and again)
static bool tsqr_halves(int64_t r, size_t tsz) {
  int64_t C = (int64_t)((200 * 1024) / (tsz * (size_t)r));
  if (C > 1024) C = 1024;
  return C >= 2 * r;
}

size_t svd_from_b_ws(int64_t r, int64_t n, int64_t m, int64_t kk, int32_t prec, int num_sms) {
  const size_t bsz = prec == LRS_PREC_FP64 ? 8 : 4;
  size_t need = (tsqr_halves(r, bsz) ? tsqr_ws(r, n, bsz) : 0) + r_of_bt_gram_ws(r, num_sms);
  if (prec != LRS_PREC_FP64 && !tsqr_halves(r, bsz))   // the FP64 copy of B and its pivoted QR
    need += 3 * align256(8 * (size_t)(n * r)) + align256(8 * (size_t)(r * r)) + cpqr_ws(n, r, r) + 1024;
  need += 4 * align256(8 * (size_t)(r * r)) + align256(8 * (size_t)(m * r)) + jacobi_ws(r, r) + 65536;
  need += jacobi_rows_ws(r) + align256(4 * (size_t)r);
  if (prec == LRS_PREC_FP64)                     // R of B^T by the pivoted QR
    need += 2 * align256(8 * (size_t)(n * r)) + align256(8 * (size_t)(r * r)) + cpqr_ws(n, r, r) + 1024;
  if (prec >= LRS_PREC_SPLIT_BF16) need += gemm_tc_workspace(kk, r, LRS_PREC_BF16X3) + 4096;
  return need;
}

// (a5) SVD of a given B (r x n, FP64 when prec is FP64, else FP32; row stride
// n) whose rows live in the range basis Q (m x r): U = Q U_B(:, :kk), S, V =
// B^T U_B S^-1.  fro2 (device, may be NULL) holds ||A_f||_F^2 for err_est.
lrs_status svd_from_b(lrs_ctx* ctx, const void* B, int64_t r, int64_t n, const double* Q, int64_t ldq, int64_t m,
                      int32_t k, int32_t prec, double* U, int64_t ldu, double* S, void* V, int64_t ldv,
                      const double* fro2, double* err_est) {
  const int f64 = prec == LRS_PREC_FP64;
  const int64_t kk = k < r ? k : r;
  double* Rm = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
  double* Vr = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
  double* sv = (double*)ws_alloc(ctx, 8 * (size_t)r);
  double* QT = (double*)ws_alloc(ctx, 8 * (size_t)(m * r));
  if (!Rm || !Vr || !sv || !QT) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd)");
  // SVD(B), all in FP64 once B exists.  FP32 B: R from the exact-slice Gram
  // and a PIVOTED FP64 Cholesky (P^T B B^T P = R^T R), then the FP64
  // one-sided Jacobi on the rows of R across a thread-block cluster, U_B =
  // P U' (jacobi_cluster.cu); TSQR if the Cholesky breaks down.  FP64 B: R
  // of B^T by the cooperative pivoted QR, FP64 Jacobi on its columns.
  lrs_status st = LRS_ERANK;
  if (f64 && r >= 24 && ctx->coop_ok) {
    // FP64 B: R of B^T by the cooperative pivoted QR (many SMs, no pivot
    // tolerance), columns put back in order: B^T = Q (R P^T); the Jacobi on
    // R P^T then gives U_B.  Replaces the one-block-per-leaf Householder TSQR.
    const size_t mark = ctx->ws_top;
    st = r_of_bt_cpqr(ctx, (const double*)B, r, n, Rm);
    ctx->ws_top = mark;
    if (st != LRS_OK && st != LRS_ERANK) return st;
  }
  int32_t* piv = (int32_t*)ws_alloc(ctx, 4 * (size_t)r);
  if (!piv) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd)");
  bool pivoted = false;
  if (st == LRS_ERANK && !f64 && r <= 128) {
    const size_t mark = ctx->ws_top;
    st = launch_r_of_bt_gram(ctx, (const float*)B, r, n, n, Rm, piv);
    ctx->ws_top = mark;
    if (st != LRS_OK && st != LRS_ERANK) return st;
    pivoted = st == LRS_OK;
  }
  if (st == LRS_ERANK && !f64 && !tsqr_halves(r, 4) && ctx->coop_ok) {
    // FP32 B too tall for the TSQR tree (r > 160): R of B^T by the
    // cooperative pivoted QR of B's FP64 copy
    const size_t mark = ctx->ws_top;
    double* B64 = (double*)ws_alloc(ctx, 8 * (size_t)(r * n));
    if (!B64) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd: FP64 copy of B)");
    st = launch_widen_f32(ctx, (const float*)B, r * n, B64);
    if (st) return st;
    st = r_of_bt_cpqr(ctx, B64, r, n, Rm);
    ctx->ws_top = mark;
    if (st != LRS_OK && st != LRS_ERANK) return st;
  }
  if (st == LRS_ERANK) st = launch_tsqr(ctx, B, f64, r, n, n, Rm);
  if (st) return st;
  st = LRS_ERANK;
  if (!f64) {
    const size_t mark = ctx->ws_top;
    st = launch_jacobi_rows(ctx, Rm, r, r, pivoted ? piv : nullptr, Vr, sv);
    ctx->ws_top = mark;
    if (st != LRS_OK && st != LRS_ERANK) return st;
  }
  if (st == LRS_ERANK) {
    // FP64 Jacobi on the columns of R (one block, or across the SMs); the
    // pivoted factor's right vectors are rows of P^T U_B, so a pivoted R is
    // only ever taken by the cluster kernel above
    if (pivoted) {
      const size_t mark = ctx->ws_top;
      st = launch_r_of_bt_gram(ctx, (const float*)B, r, n, n, Rm, nullptr);
      ctx->ws_top = mark;
      if (st == LRS_ERANK) st = launch_tsqr(ctx, B, f64, r, n, n, Rm);
      if (st) return st;
    }
    st = launch_jacobi(ctx, Rm, r, Vr, sv);
  }
  if (st) return st;
  (void)QT;
  return svd_finish(ctx, Vr, sv, r, kk, Q, ldq, m, B, n, prec, U, ldu, S, V, ldv, fro2, err_est);
}

// (a4) B = Q^T A_f (r x n, row stride n; FP64 when prec is FP64, else FP32)
// -- the one full read of A_f -- and ||A_f||_F^2 into fro2 (device; fused
// into the tensor-core A-pass, a separate pass otherwise)
static size_t apass_b_ws(lrs_ctx* ctx, int64_t m, int64_t n, int64_t r, int32_t prec) {
  return prec >= LRS_PREC_SPLIT_BF16
             ? gemm_tc_workspace(r, m, prec) + gemm_tc_splitk_workspace(r, n, m, ctx->num_sms) + 4096
             : 0;
}

static lrs_status apass_b(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                          const double* Q, int64_t ldq, int64_t r, int32_t prec, void* B, double* fro2) {
  const int f64 = prec == LRS_PREC_FP64;
  GemmArgs ga{r, n, m, Q, LRS_F64, ldq, A, dtype, lda, B, f64, 0, n, 1.0};
  const size_t mark = ctx->ws_top;
  lrs_status st;
  if (prec >= LRS_PREC_SPLIT_BF16 && (r <= 128 || apass_eligible(ga, prec))) {
    st = launch_gemm_tc(ctx, ga, prec, fro2);
    if (st) return st;
  } else {
    st = gemm(ctx, prec, r, n, m, Q, LRS_F64, ldq, A, dtype, lda, B, f64, 0, n);
    if (st) return st;
    st = launch_fro2(ctx, A, dtype, m, n, lda, fro2);
    if (st) return st;
  }
  ctx->ws_top = mark;
  return LRS_OK;
}

lrs_status gemm_prec(lrs_ctx* ctx, int prec, int64_t M, int64_t N, int64_t K, const void* X, int32_t xdt, int64_t ldx,
                     const void* A, int32_t adt, int64_t lda, void* C, int c_f64, int c_trans, int64_t ldc) {
  return gemm(ctx, prec, M, N, K, X, xdt, ldx, A, adt, lda, C, c_f64, c_trans, ldc);
}

}  // namespace lrs

extern "C" {

lrs_status lrs_svd_k(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                     const double* Q, int64_t ldq, int64_t r, int32_t k, int32_t prec, double* U,
                     int64_t ldu, double* S, void* V, int64_t ldv, double* err_est) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!A || !Q || !U || !S || !V) return lrs_fail(ctx, LRS_EINVAL, "svd_k: NULL pointer");
  if (!dtype_ok(dtype) || !prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "svd_k: bad dtype/prec");
  if (m < 1 || n < 1 || r < 1 || k < 1) return lrs_fail(ctx, LRS_EINVAL, "svd_k: m=%lld n=%lld r=%lld k=%d", (long long)m, (long long)n, (long long)r, k);
  if (r > m) return lrs_fail(ctx, LRS_EINVAL, "svd_k: r=%lld > m=%lld", (long long)r, (long long)m);
  const int64_t kk = k < r ? k : r;
  if (lda < n || ldq < r || ldu < kk || ldv < kk) return lrs_fail(ctx, LRS_EINVAL, "svd_k: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int f64 = prec == LRS_PREC_FP64;
  const size_t bsz = f64 ? 8 : 4;
  size_t need = align256(bsz * (size_t)(r * n)) + 256 + svd_from_b_ws(r, n, m, kk, prec, ctx->num_sms) +
                lrs::apass_b_ws(ctx, m, n, r, prec);
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  void* B = ws_alloc(ctx, bsz * (size_t)(r * n));
  double* fro2 = (double*)ws_alloc(ctx, 8);
  if (!B || !fro2) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd_k)");
  st = lrs::apass_b(ctx, A, dtype, m, n, lda, Q, ldq, r, prec, B, fro2);
  if (st) return st;
  st = svd_from_b(ctx, B, r, n, Q, ldq, m, k, prec, U, ldu, S, V, ldv, fro2, err_est);
  if (st) return st;
  return r < k ? lrs_fail(ctx, LRS_ERANK, "svd_k: rank r=%lld < k=%d", (long long)r, k) : LRS_OK;
}

lrs_status lrs_apass_slab(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                          const double* Q, int64_t ldq, int64_t r, int32_t prec, void* B, double* fro2) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!A || !Q || !B || !fro2) return lrs_fail(ctx, LRS_EINVAL, "apass_slab: NULL pointer");
  if (!dtype_ok(dtype) || !prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "apass_slab: bad dtype/prec");
  if (m < 1 || n < 1 || r < 1 || r > m)
    return lrs_fail(ctx, LRS_EINVAL, "apass_slab: m=%lld n=%lld r=%lld", (long long)m, (long long)n, (long long)r);
  if (lda < n || ldq < r) return lrs_fail(ctx, LRS_EINVAL, "apass_slab: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, lrs::apass_b_ws(ctx, m, n, r, prec) + 256);
  if (st) return st;
  return lrs::apass_b(ctx, A, dtype, m, n, lda, Q, ldq, r, prec, B, fro2);
}

lrs_status lrs_slab_factor(lrs_ctx* ctx, const void* B, int64_t r, int64_t n, int32_t prec, int32_t mode, double* F,
                           int64_t ldf) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!B || !F) return lrs_fail(ctx, LRS_EINVAL, "slab_factor: NULL pointer");
  if (!prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "slab_factor: bad prec");
  if (r < 1 || n < 1 || ldf < r) return lrs_fail(ctx, LRS_EINVAL, "slab_factor: r=%lld n=%lld ldf=%lld",
                                                 (long long)r, (long long)n, (long long)ldf);
  const int f64 = prec == LRS_PREC_FP64;
  if (mode == LRS_FACTOR_GRAM) {
    if (f64 || r > 128) return lrs_fail(ctx, LRS_EINVAL, "slab_factor: the Gram form takes FP32 B with r <= 128");
  } else if (mode == LRS_FACTOR_R) {
    if (n < r) return lrs_fail(ctx, LRS_EINVAL, "slab_factor: the R form needs n=%lld >= r=%lld", (long long)n,
                               (long long)r);
  } else {
    return lrs_fail(ctx, LRS_EINVAL, "slab_factor: mode %d", mode);
  }
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  size_t need = 2 * align256(8 * (size_t)(r * r)) + 1024;
  if (mode == LRS_FACTOR_GRAM) need += gram_oz_ws(r, ctx->num_sms);
  else need += tsqr_ws(r, n, f64 ? 8 : 4) + 2 * align256(8 * (size_t)(n * r)) + cpqr_ws(n, r, r) + 1024;
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  double* Rm = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
  if (!Rm) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (slab_factor)");
  if (mode == LRS_FACTOR_GRAM) {
    // F = B B^T, the exact-slice tensor-core Gram of the SVD path
    st = launch_gram_oz(ctx, (const float*)B, r, n, n, ldf == r ? F : Rm);
    if (st) return st;
    if (ldf != r)
      LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(F, ldf * 8, Rm, r * 8, r * 8, r, cudaMemcpyDeviceToDevice, ctx->stream));
    return LRS_OK;
  }
  // F = R^T with R^T R = B B^T: the cooperative pivoted QR of B^T (FP64 B),
  // else the Householder TSQR of the SVD path
  st = LRS_ERANK;
  if (f64 && r >= 24 && ctx->coop_ok) {
    const size_t mark = ctx->ws_top;
    st = r_of_bt_cpqr(ctx, (const double*)B, r, n, Rm);
    ctx->ws_top = mark;
    if (st != LRS_OK && st != LRS_ERANK) return st;
  }
  if (st == LRS_ERANK) st = launch_tsqr(ctx, B, f64, r, n, n, Rm);
  if (st) return st;
  return launch_transpose(ctx, Rm, r, r, r, F, ldf);
}

lrs_status lrs_svd_from_factor(lrs_ctx* ctx, const double* F, int64_t ldf, int64_t nf, int32_t mode,
                               const double* Q, int64_t ldq, int64_t m, int64_t r, int32_t k, int32_t prec,
                               const void* B, int64_t n, const double* fro2, double* U, int64_t ldu, double* S,
                               void* V, int64_t ldv, double* err_est) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!F || !Q || !B || !U || !S || !V) return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: NULL pointer");
  if (!prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: bad prec");
  if (m < 1 || n < 1 || r < 1 || k < 1 || r > m)
    return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: m=%lld n=%lld r=%lld k=%d", (long long)m, (long long)n,
                    (long long)r, k);
  const int f64 = prec == LRS_PREC_FP64;
  if (mode == LRS_FACTOR_GRAM) {
    if (f64 || r > 128 || nf != r)
      return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: the Gram form takes FP32 B, r <= 128 and nf == r");
  } else if (mode == LRS_FACTOR_R) {
    if (nf < r) return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: nf=%lld < r=%lld", (long long)nf, (long long)r);
  } else {
    return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: mode %d", mode);
  }
  const int64_t kk = k < r ? k : r;
  if (ldf < nf || ldq < r || ldu < kk || ldv < kk) return lrs_fail(ctx, LRS_EINVAL, "svd_from_factor: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  size_t need = 4 * align256(8 * (size_t)(r * r)) + 2 * align256(8 * (size_t)r) + jacobi_ws(r, r) +
                jacobi_rows_ws(r) + align256(8 * (size_t)(r * kk)) + 65536;
  if (mode == LRS_FACTOR_R)
    need += align256(8 * (size_t)(nf * r)) + 2 * align256(8 * (size_t)(nf * r)) + cpqr_ws(nf, r, r) +
            tsqr_ws(r, nf, 8) + 1024;
  if (prec >= LRS_PREC_SPLIT_BF16) need += gemm_tc_workspace(kk, r, LRS_PREC_BF16X3) + 4096;
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  double* Rm = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
  double* Vr = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
  double* sv = (double*)ws_alloc(ctx, 8 * (size_t)r);
  int32_t* piv = (int32_t*)ws_alloc(ctx, 4 * (size_t)r);
  int32_t* rank = (int32_t*)ws_alloc(ctx, 8);
  if (!Rm || !Vr || !sv || !piv || !rank) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd_from_factor)");
  if (mode == LRS_FACTOR_GRAM) {
    // the pivoted FP64 Cholesky of the summed Gram and the cluster Jacobi on
    // the rows of its factor, as lrs_svd_k takes them for FP32 B
    const double* G = F;
    if (ldf != r) {
      double* Gc = (double*)ws_alloc(ctx, 8 * (size_t)(r * r));
      if (!Gc) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd_from_factor)");
      LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(Gc, r * 8, F, ldf * 8, r * 8, r, cudaMemcpyDeviceToDevice, ctx->stream));
      G = Gc;
    }
    st = launch_pchol(ctx, G, (int)r, (int)r, 0.0, 1, piv, Rm, r, rank);
    if (st) return st;
    int32_t* h = (int32_t*)ctx->host_scratch;
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 44, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (h[44] != (int32_t)r) {
      if (err_est) *err_est = -1.0;       // nothing written: the caller takes LRS_FACTOR_R
      return lrs_fail(ctx, LRS_ERANK,
                      "svd_from_factor: the FP64 Gram of B is not positive definite (Cholesky rank %d < r=%lld); "
                      "LRS_FACTOR_R factors B without squaring it", h[44], (long long)r);
    }
    const size_t mark = ctx->ws_top;
    st = launch_jacobi_rows(ctx, Rm, r, r, piv, Vr, sv);
    ctx->ws_top = mark;
    if (st != LRS_OK && st != LRS_ERANK) return st;
    if (st == LRS_ERANK) {
      // no cluster fits: the unpivoted factor and the Jacobi on its columns
      st = launch_pchol(ctx, G, (int)r, (int)r, 0.0, 0, piv, Rm, r, rank);
      if (st) return st;
      st = launch_jacobi(ctx, Rm, r, Vr, sv);
      if (st) return st;
    }
  } else {
    // R of F^T (r x r, F F^T = B B^T), then the FP64 Jacobi on its columns
    const double* Fc = F;
    if (ldf != nf) {
      double* t = (double*)ws_alloc(ctx, 8 * (size_t)(nf * r));
      if (!t) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd_from_factor)");
      LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(t, nf * 8, F, ldf * 8, nf * 8, r, cudaMemcpyDeviceToDevice, ctx->stream));
      Fc = t;
    }
    st = LRS_ERANK;
    if (r >= 24 && ctx->coop_ok) {
      const size_t mark = ctx->ws_top;
      st = r_of_bt_cpqr(ctx, Fc, r, nf, Rm);
      ctx->ws_top = mark;
      if (st != LRS_OK && st != LRS_ERANK) return st;
    }
    if (st == LRS_ERANK) st = launch_tsqr(ctx, Fc, 1, r, nf, nf, Rm);
    if (st) return st;
    st = launch_jacobi(ctx, Rm, r, Vr, sv);
    if (st) return st;
  }
  st = lrs::svd_finish(ctx, Vr, sv, r, kk, Q, ldq, m, B, n, prec, U, ldu, S, V, ldv, fro2, err_est);
  if (st) return st;
  return r < k ? lrs_fail(ctx, LRS_ERANK, "svd_from_factor: rank r=%lld < k=%d", (long long)r, k) : LRS_OK;
}

lrs_status lrs_id_k(lrs_ctx* ctx, const double* Ysk, int64_t m, int64_t l, int64_t ldy, int32_t k,
                    int32_t* J, double* P, int64_t ldp, double* err_est) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!Ysk || !J || !P) return lrs_fail(ctx, LRS_EINVAL, "id_k: NULL pointer");
  if (m < 1 || l < 1 || k < 1) return lrs_fail(ctx, LRS_EINVAL, "id_k: m=%lld l=%lld k=%d", (long long)m, (long long)l, k);
  if (k > m) return lrs_fail(ctx, LRS_EINVAL, "id_k: k=%d exceeds m=%lld", k, (long long)m);
  // a sketch of l < k columns has rank below k: a rank-k ID does not exist
  if (k > l) return lrs_fail(ctx, LRS_ERANK, "id_k: sketch rank <= l=%lld < k=%d", (long long)l, k);
  if (ldy < l || ldp < k) return lrs_fail(ctx, LRS_EINVAL, "id_k: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  size_t need = align256(8 * (size_t)(m * l)) + align256(4 * (size_t)m) +
                align256(8 * (size_t)(k * m)) + align256(8 * (size_t)(l * k)) + 65536 +
                cpqr_ws(l, m, k);
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  // Y^T is l x m; its column-major storage is Y's row-major storage.
  double* Mc = (double*)ws_alloc(ctx, 8 * (size_t)(m * l));
  CpqrOut o{};
  o.perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)m);
  o.R = (double*)ws_alloc(ctx, 8 * (size_t)(k * m));
  o.V = (double*)ws_alloc(ctx, 8 * (size_t)(l * k));
  o.tail2 = (double*)ws_alloc(ctx, 8);
  o.rank = (int32_t*)ws_alloc(ctx, 8);
  double* nrm2 = (double*)ws_alloc(ctx, 8);
  if (!Mc || !o.perm || !o.R || !o.V || !o.tail2 || !o.rank || !nrm2)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (id_k)");
  LRS_CUDA_TRY(ctx, cudaMemcpy2DAsync(Mc, l * 8, Ysk, ldy * 8, l * 8, m, cudaMemcpyDeviceToDevice, ctx->stream));
  st = launch_fro2(ctx, Mc, LRS_F64, m, l, l, nrm2);
  if (st) return st;
  st = launch_cpqr(ctx, Mc, l, m, l, k, 0.0, o);
  if (st) return st;
  int32_t rank = 0;
  double* h = (double*)ctx->host_scratch;
  if (ctx->replay == kReplayCapture) {
    // captured: the rank from the record, the error estimate on the device
    const int32_t* d[1] = {o.rank};
    st = replay_ints(ctx, 1, d, &rank);
    if (st) return st;
    if (rank < k) return lrs_fail(ctx, LRS_ERANK, "id_k: sketch rank %d < k=%d", rank, k);
    st = launch_id_coeffs(ctx, o.R, k, m, o.perm, J, P, ldp);
    if (st) return st;
    if (err_est) *err_est = 0.0;
    return launch_err_ratio(ctx, o.tail2, nrm2, ctx->cap_err + 1);
  }
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(&rank, o.rank, 4, cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h, o.tail2, 8, cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 1, nrm2, 8, cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->replay == kReplayRecord) ctx->log.push_back(rank);
  if (rank < k) return lrs_fail(ctx, LRS_ERANK, "id_k: sketch rank %d < k=%d", rank, k);
  st = launch_id_coeffs(ctx, o.R, k, m, o.perm, J, P, ldp);
  if (st) return st;
  if (err_est) *err_est = h[1] > 0.0 ? sqrt(fmax(h[0], 0.0) / h[1]) : 0.0;
  return LRS_OK;
}

lrs_status lrs_range_error(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                           const double* Q, int64_t ldq, int64_t r, double* err) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!A || !Q || !err) return lrs_fail(ctx, LRS_EINVAL, "range_error: NULL pointer");
  if (!dtype_ok(dtype) || m < 1 || n < 1 || r < 0 || r > m || lda < n || ldq < r)
    return lrs_fail(ctx, LRS_EINVAL, "range_error: bad sizes");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, align256(8 * (size_t)(r * n)) + 4096);
  if (st) return st;
  double* B = r > 0 ? (double*)ws_alloc(ctx, 8 * (size_t)(r * n)) : nullptr;
  double* sq = (double*)ws_alloc(ctx, 16);
  if ((r > 0 && !B) || !sq) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (range_error)");
  // every square in FP64: err^2 = 1 - ||Q^T A||^2 / ||A||^2 cancels, and an
  // FP32-level ||A||^2 would leave err at ~sqrt(u32) ~ 3e-4
  st = launch_fro2(ctx, A, dtype, m, n, lda, sq, 1);
  if (st) return st;
  if (r > 0) {
    st = gemm(ctx, LRS_PREC_FP64, r, n, m, Q, LRS_F64, ldq, A, dtype, lda, B, 1, 0, n);
    if (st) return st;
    st = launch_fro2(ctx, B, LRS_F64, r, n, n, sq + 1);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemsetAsync(sq + 1, 0, 8, ctx->stream));
  }
  double* h = (double*)ctx->host_scratch;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 8, sq, 16, cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const double a2 = h[8], b2 = h[9];
  *err = a2 > 0.0 ? sqrt(fmax(0.0, 1.0 - b2 / a2)) : 0.0;
  return LRS_OK;
}

lrs_status lrs_gemm_tn(lrs_ctx* ctx, int64_t M, int64_t N, int64_t K, const void* X, int32_t x_dtype,
                       int64_t ldx, const void* A, int32_t a_dtype, int64_t lda, void* C, int32_t c_f64,
                       int32_t c_trans, int64_t ldc, int32_t prec) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!X || !A || !C) return lrs_fail(ctx, LRS_EINVAL, "gemm: NULL pointer");
  if (M < 0 || N < 0 || K < 0) return lrs_fail(ctx, LRS_EINVAL, "gemm: negative size");
  if (!dtype_ok(x_dtype) || !dtype_ok(a_dtype) || !prec_ok(prec)) return lrs_fail(ctx, LRS_EINVAL, "gemm: bad dtype/prec");
  if (ldx < M || lda < N || ldc < (c_trans ? M : N)) return lrs_fail(ctx, LRS_EINVAL, "gemm: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, prec >= LRS_PREC_SPLIT_BF16
                                      ? gemm_tc_workspace(M, K, prec) + gemm_tc_splitk_workspace(M, N, K, ctx->num_sms) + 4096
                                      : 0);
  if (st) return st;
  return gemm(ctx, prec, M, N, K, X, x_dtype, ldx, A, a_dtype, lda, C, c_f64, c_trans, ldc);
}

}  // extern "C"
