// Householder QR with column pivoting in FP64 (paper Sec. 4: the rank-k
// column-pivoted QR behind the row ID; also the rank-revealing "QR(.)" of
// Algs. 2/3/7), the explicit Q factor, and the ID coefficients
// C = R_1^{-1} R_2, P = ([I | C] Z^T)^T.
//
// Pivoting rule: the remaining column of largest 2-norm, norms recomputed
// from the updated columns at every step (no down-dating); ties go to the
// lowest current position.  Reflector: R_jj = -sign(x_0) ||x||, v = x +
// sign(x_0)||x|| e_1 normalised, H = I - 2 v v^T.
//
// One persistent cooperative launch runs all steps.  Each block owns a
// contiguous range of physical columns; a step is
//   (1) every block reduces the per-block best (norm^2, position) -> pivot,
//   (2) the pivot's owner builds v, block 0 records the position swap,
//       -- grid barrier --
//   (3) every block applies H to its live columns, records row j of R and
//       the new norms, and publishes its best candidate,
//       -- grid barrier --
// The barriers are bounded (common.cuh) and report LRS_ETIMEOUT.
#include "common.cuh"
#include "internal.h"

#include <cooperative_groups.h>

namespace lrs {

struct CpqrState {
  double* M; int64_t p, c, ldm;
  int64_t kmax; double rtol;
  // outputs
  int32_t* perm; double* R; double* V; double* tail2; int32_t* rank;
  // scratch
  double* norm2;        // c
  int32_t* pos_of;      // c  (physical -> position)
  int32_t* phys_at;     // c  (position -> physical)
  uint8_t* done;        // c
  double* Rphys;        // kmax x c (row j, physical column)
  double* best_val;     // nblocks
  int32_t* best_pos;    // nblocks
  int32_t* best_phys;   // nblocks
  double* vbuf;         // p   (current reflector)
  double* pivinfo;      // [0] = R_jj, [1] = top
  GridBarrier bar;
  int v_in_smem;
};

__device__ __forceinline__ bool better(double a, int pa, double b, int pb) {
  return (a > b) || (a == b && pa < pb);
}

// block-local argmax over (val, pos, phys); writes the winner to thread 0
__device__ void block_best(double& val, int& pos, int& phys, double* sv, int* sp, int* sf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, val, o);
    int op = __shfl_xor_sync(0xffffffffu, pos, o);
    int of = __shfl_xor_sync(0xffffffffu, phys, o);
    if (better(ov, op, val, pos)) { val = ov; pos = op; phys = of; }
  }
  __syncthreads();
  if (lane == 0) { sv[wid] = val; sp[wid] = pos; sf[wid] = phys; }
  __syncthreads();
  if (wid == 0) {
    val = lane < nw ? sv[lane] : -1.0; pos = lane < nw ? sp[lane] : 0x7fffffff;
    phys = lane < nw ? sf[lane] : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, val, o);
      int op = __shfl_xor_sync(0xffffffffu, pos, o);
      int of = __shfl_xor_sync(0xffffffffu, phys, o);
      if (better(ov, op, val, pos)) { val = ov; pos = op; phys = of; }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(512, 1) k_cpqr(CpqrState s) {
  extern __shared__ double smem_v[];
  __shared__ double sv[32];
  __shared__ int sp[32], sf[32];
  __shared__ int s_piv_pos, s_piv_phys, s_stop;

  const int nb = gridDim.x;
  const int64_t per = (s.c + nb - 1) / nb;
  const int64_t c_lo = (int64_t)blockIdx.x * per;
  const int64_t c_hi = min(s.c, c_lo + per);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // ---- init: norms of all columns, positions = identity ----------------------
  {
    double bv = -1.0; int bp = 0x7fffffff, bf = -1;
    for (int64_t cc = c_lo + wid; cc < c_hi; cc += nw) {
      const double* col = s.M + cc * s.ldm;
      double a = 0.0;
      for (int64_t i = lane; i < s.p; i += 32) a = fma(col[i], col[i], a);
      a = warp_sum(a);
      if (lane == 0) {
        s.norm2[cc] = a; s.pos_of[cc] = (int)cc; s.phys_at[cc] = (int)cc; s.done[cc] = 0;
      }
      if (better(a, (int)cc, bv, bp)) { bv = a; bp = (int)cc; bf = (int)cc; }
    }
    block_best(bv, bp, bf, sv, sp, sf);
    if (threadIdx.x == 0) { s.best_val[blockIdx.x] = bv; s.best_pos[blockIdx.x] = bp; s.best_phys[blockIdx.x] = bf; }
  }
  if (!grid_sync(s.bar)) return;

  double top = 0.0;
  int64_t j = 0;
  for (; j < s.kmax; ++j) {
    // (1) global pivot (every block reduces the same data)
    {
      double bv = -1.0; int bp = 0x7fffffff, bf = -1;
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double v = __ldcg(s.best_val + b);
        const int p = __ldcg(s.best_pos + b);
        if (better(v, p, bv, bp)) { bv = v; bp = p; bf = __ldcg(s.best_phys + b); }
      }
      block_best(bv, bp, bf, sv, sp, sf);
      if (threadIdx.x == 0) {
        s_piv_pos = bp; s_piv_phys = bf;
        const double nrm = sqrt(fmax(bv, 0.0));
        if (j == 0) top = nrm;
        s_stop = (bf < 0 || bv <= 0.0 || (j > 0 && nrm <= s.rtol * top)) ? 1 : 0;
      }
      __syncthreads();
    }
    if (s_stop) break;
    const int piv = s_piv_phys;

    // (2) reflector by the owner of the pivot column; position swap by block 0
    if (piv >= c_lo && piv < c_hi) {
      double* col = s.M + (int64_t)piv * s.ldm;
      double a = 0.0;
      for (int64_t i = j + threadIdx.x; i < s.p; i += blockDim.x) a = fma(col[i], col[i], a);
      a = block_sum(a, sv);
      const double alpha = sqrt(a);
      const double x0 = col[j];
      const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
      const double v0 = x0 + sgn * alpha;
      double b = 0.0;
      for (int64_t i = j + threadIdx.x; i < s.p; i += blockDim.x) {
        const double vi = (i == j) ? v0 : col[i];
        b = fma(vi, vi, b);
      }
      b = block_sum(b, sv);
      const double inv = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
      for (int64_t i = threadIdx.x; i < s.p; i += blockDim.x) {
        const double vi = i < j ? 0.0 : ((i == j) ? v0 : col[i]) * inv;
        s.vbuf[i] = vi;
        s.V[(int64_t)j * s.p + i] = vi;
      }
      if (threadIdx.x == 0) {
        s.done[piv] = 1;
        s.Rphys[j * s.c + piv] = -sgn * alpha;
        s.pivinfo[0] = -sgn * alpha;
      }
      // the pivot column becomes R's column: rows > j are zero (after every
      // thread has read it above: the two loops map rows to threads differently)
      __syncthreads();
      for (int64_t i = j + threadIdx.x; i < s.p; i += blockDim.x) col[i] = (i == j) ? -sgn * alpha : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const int pj = __ldcg(s.phys_at + j);  // physical column now at position j
      const int pp = s_piv_pos;             // position of the pivot
      s.phys_at[j] = piv; s.phys_at[pp] = pj;
      s.pos_of[piv] = (int)j; s.pos_of[pj] = pp;
    }
    if (!grid_sync(s.bar)) return;

    // (3) apply H_j = I - 2 v v^T to the live columns of this block
    const double* v = s.vbuf;
    if (s.v_in_smem) {
      for (int64_t i = threadIdx.x; i < s.p; i += blockDim.x) smem_v[i] = __ldcg(s.vbuf + i);
      __syncthreads();
      v = smem_v;
    }
    double bv = -1.0; int bp = 0x7fffffff, bf = -1;
    for (int64_t cc = c_lo + wid; cc < c_hi; cc += nw) {
      if (s.done[cc]) continue;
      double* col = s.M + cc * s.ldm;
      double w = 0.0;
      if (s.v_in_smem) {
        for (int64_t i = j + lane; i < s.p; i += 32) w = fma(v[i], col[i], w);
      } else {
        for (int64_t i = j + lane; i < s.p; i += 32) w = fma(__ldcg(v + i), col[i], w);
      }
      w = warp_sum(w);
      const double tw = 2.0 * w;
      double a = 0.0;
      for (int64_t i = j + lane; i < s.p; i += 32) {
        const double vi = s.v_in_smem ? v[i] : __ldcg(v + i);
        const double x = fma(-tw, vi, col[i]);
        col[i] = x;
        if (i > j) a = fma(x, x, a);
      }
      a = warp_sum(a);
      if (lane == 0) {
        s.Rphys[j * s.c + cc] = col[j];
        s.norm2[cc] = a;
      }
      const int pc = __ldcg(s.pos_of + cc);
      if (better(a, pc, bv, bp)) { bv = a; bp = pc; bf = (int)cc; }
    }
    block_best(bv, bp, bf, sv, sp, sf);
    if (threadIdx.x == 0) { s.best_val[blockIdx.x] = bv; s.best_pos[blockIdx.x] = bp; s.best_phys[blockIdx.x] = bf; }
    if (!grid_sync(s.bar)) return;
  }

  // ---- epilogue: rank, permutation, R in pivoted order, trailing norm ------
  const int64_t r = j;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) *s.rank = (int32_t)r;
    for (int64_t q = threadIdx.x; q < s.c; q += blockDim.x) s.perm[q] = __ldcg(s.phys_at + q);
    double t = 0.0;
    for (int64_t cc = threadIdx.x; cc < s.c; cc += blockDim.x)
      if (!__ldcg(s.done + cc)) t += __ldcg(s.norm2 + cc);
    t = block_sum(t, sv);
    if (threadIdx.x == 0) *s.tail2 = (r < min(s.p, s.c)) ? t : 0.0;
  }
  // R[i, q] = Rphys[i, phys_at[q]] for i < r, zero below the diagonal
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * s.c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / s.c, q = e - i * s.c;
    s.R[i * s.c + q] = (q < i) ? 0.0 : __ldcg(s.Rphys + i * s.c + __ldcg(s.phys_at + q));
  }
}

lrs_status launch_cpqr(lrs_ctx* ctx, double* M, int64_t p, int64_t c, int64_t ldm,
                       int64_t kmax, double rtol, const CpqrOut& o) {
  if (!ctx->coop_ok) return lrs_fail(ctx, LRS_ECUDA, "device lacks cooperative launch");
  CpqrState s{};
  s.M = M; s.p = p; s.c = c; s.ldm = ldm; s.kmax = kmax; s.rtol = rtol;
  s.perm = o.perm; s.R = o.R; s.V = o.V; s.tail2 = o.tail2; s.rank = o.rank;
  const int threads = 512;
  const size_t vbytes = sizeof(double) * (size_t)p;
  s.v_in_smem = vbytes <= 160 * 1024 ? 1 : 0;
  const size_t dyn = s.v_in_smem ? vbytes : 0;
  if (dyn > 48 * 1024)
    LRS_CUDA_TRY(ctx, cudaFuncSetAttribute(k_cpqr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int per_sm = 0;
  LRS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cpqr, threads, dyn));
  if (per_sm < 1) return lrs_fail(ctx, LRS_ECUDA, "cpqr: kernel does not fit on an SM");
  int64_t nb = ctx->num_sms;                       // one block per SM
  const int64_t want = (c + 15) / 16;              // at least ~16 columns per block
  if (nb > want) nb = want < 1 ? 1 : want;

  s.norm2 = (double*)ws_alloc(ctx, sizeof(double) * c);
  s.pos_of = (int32_t*)ws_alloc(ctx, sizeof(int32_t) * c);
  s.phys_at = (int32_t*)ws_alloc(ctx, sizeof(int32_t) * c);
  s.done = (uint8_t*)ws_alloc(ctx, c);
  s.Rphys = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(kmax > 0 ? kmax : 1) * c);
  s.best_val = (double*)ws_alloc(ctx, sizeof(double) * nb);
  s.best_pos = (int32_t*)ws_alloc(ctx, sizeof(int32_t) * nb);
  s.best_phys = (int32_t*)ws_alloc(ctx, sizeof(int32_t) * nb);
  s.vbuf = (double*)ws_alloc(ctx, vbytes);
  s.pivinfo = (double*)ws_alloc(ctx, sizeof(double) * 2);
  unsigned* bar = (unsigned*)ws_alloc(ctx, 256);
  if (!s.norm2 || !s.pos_of || !s.phys_at || !s.done || !s.Rphys || !s.best_val || !s.best_pos ||
      !s.best_phys || !s.vbuf || !s.pivinfo || !bar)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpqr)");
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, 256, ctx->stream));
  s.bar.count = bar; s.bar.gen = bar + 1; s.bar.err = (int*)(bar + 2);
  void* args[] = {&s};
  LRS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_cpqr, dim3((unsigned)nb), dim3(threads),
                                                args, dyn, ctx->stream));
  ctx->launches++;
  // the barrier's error word is checked by the caller through lrs::check_device_error
  int err_h = 0;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(&err_h, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (err_h != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "cpqr: grid barrier wait gave up");
  return LRS_OK;
}

// ---------------------------------------------------------------------------
// Q = H_0 ... H_{r-1} [I_r; 0]: column c only sees H_c .. H_0 (reflectors
// with index > c leave e_c untouched), so each block builds one column.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_form_q(const double* __restrict__ V, int64_t p, int64_t r,
                                                double* __restrict__ Q, int64_t ldq) {
  extern __shared__ double q[];
  __shared__ double red[32];
  const int64_t c = blockIdx.x;
  for (int64_t i = threadIdx.x; i < p; i += blockDim.x) q[i] = (i == c) ? 1.0 : 0.0;
  __syncthreads();
  for (int64_t jj = c; jj >= 0; --jj) {
    const double* v = V + jj * p;
    double w = 0.0;
    for (int64_t i = jj + threadIdx.x; i < p; i += blockDim.x) w = fma(v[i], q[i], w);
    w = block_sum(w, red);
    const double tw = 2.0 * w;
    for (int64_t i = jj + threadIdx.x; i < p; i += blockDim.x) q[i] = fma(-tw, v[i], q[i]);
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < p; i += blockDim.x) Q[i * ldq + c] = q[i];
}

lrs_status launch_form_q(lrs_ctx* ctx, const double* V, int64_t p, int64_t r, double* Q, int64_t ldq) {
  if (r <= 0) return LRS_OK;
  const size_t dyn = sizeof(double) * (size_t)p;
  if (dyn > 200 * 1024) return lrs_fail(ctx, LRS_EINVAL, "form_q: p=%lld too large", (long long)p);
  if (dyn > 48 * 1024)
    LRS_CUDA_TRY(ctx, cudaFuncSetAttribute(k_form_q, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  k_form_q<<<(unsigned)r, 256, dyn, ctx->stream>>>(V, p, r, Q, ldq);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// ---------------------------------------------------------------------------
// ID coefficients.  R is k x m (pivoted order, row stride m).  Column q >= k
// of R_2 gives C[:, q-k] = R_1^{-1} R[:, q] by back substitution; then
// P[perm[i], :] = e_i (i < k) and P[perm[q], :] = C[:, q-k]^T.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_id_coeffs(const double* __restrict__ R, int64_t k, int64_t m,
                                                   const int32_t* __restrict__ perm,
                                                   int32_t* __restrict__ J, double* __restrict__ P,
                                                   int64_t ldp) {
  extern __shared__ double R1[];   // k x k
  for (int64_t e = threadIdx.x; e < k * k; e += blockDim.x) R1[e] = R[(e / k) * m + (e % k)];
  __syncthreads();
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0) {
    for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
      J[i] = perm[i];
      double* prow = P + (int64_t)perm[i] * ldp;
      for (int64_t t = 0; t < k; ++t) prow[t] = (t == i) ? 1.0 : 0.0;
    }
  }
  if (q >= m - k) return;
  const int64_t col = k + q;
  double* prow = P + (int64_t)perm[col] * ldp;
  // back substitution, writing the solution straight into P's row
  for (int64_t i = k - 1; i >= 0; --i) {
    double acc = R[i * m + col];
    for (int64_t t = i + 1; t < k; ++t) acc = fma(-R1[i * k + t], prow[t], acc);
    prow[i] = acc / R1[i * k + i];
  }
}

lrs_status launch_id_coeffs(lrs_ctx* ctx, const double* R, int64_t k, int64_t m,
                            const int32_t* perm, int32_t* J, double* P, int64_t ldp) {
  const size_t dyn = sizeof(double) * (size_t)(k * k);
  if (dyn > 200 * 1024) return lrs_fail(ctx, LRS_EINVAL, "id: k=%lld too large", (long long)k);
  if (dyn > 48 * 1024)
    LRS_CUDA_TRY(ctx, cudaFuncSetAttribute(k_id_coeffs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  const int64_t cols = m - k;
  const unsigned nb = (unsigned)((cols + 127) / 128 > 0 ? (cols + 127) / 128 : 1);
  k_id_coeffs<<<nb, 128, dyn, ctx->stream>>>(R, k, m, perm, J, P, ldp);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
