// FP64 SVD of the small triangular factor of B^T on one thread-block cluster
// (paper Alg. 2, "SVD(B)"), for the FP32-data path of lrs_svd_k.
//
// Input: R (r x r, upper triangular) with P^T B B^T P = R^T R from the
// pivoted Cholesky of the Gram (P: perm[pos] = row of B), so P^T B = R^T Z^T
// with Z^T Z = I.  One-sided (Hestenes) Jacobi on the COLUMNS OF R^T (the rows
// of R): X W = U' diag(s) with X = R^T, W orthogonal; then
//   B = (P U') diag(s) (Z W)^T,
// so the left singular vectors of B are U_B = P U', where U' holds the
// normalised columns of the rotated X, and s are its column norms.  The
// right factor W is never accumulated.  Pivoting makes R graded (|R_jj|
// non-increasing, each row dominated by its diagonal), which is the
// preconditioning under which one-sided Jacobi on R^T converges in few
// sweeps (Drmac & Veselic, "New fast and accurate Jacobi SVD algorithm",
// SIAM J. Matrix Anal. Appl. 29, 2008).
//
// Parallel ordering: block-cyclic Jacobi over a cluster of NC CTAs.  The
// columns form 2 NC blocks of b columns (the last padded with zero columns,
// which never rotate).  A sweep is a round-robin tournament of the blocks
// (2 NC - 1 rounds, every block pair meets once; the blocks' internal pairs
// are taken in the first round of the sweep): CTA i holds the blocks at
// tournament positions i and 2 NC - 1 - i in its shared memory, rotates the
// b x b cross pairs in b conflict-free sub-rounds (a warp per pair, FP64
// data throughout), then sends each block it gives up straight into the
// shared memory of the CTA that takes it next (distributed shared memory),
// double-buffered by round parity, with one cluster barrier per round.
// On GB300 an SM retires 2 FP64 FMAs per clock, so spreading the sweep over
// up to 16 SMs with a hardware barrier is what makes FP64 affordable here.
// The kernel has no spin-wait: the cluster barrier is a hardware barrier of
// co-scheduled CTAs, and every CTA takes the same number of them.
#include "common.cuh"
#include "internal.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace lrs {

namespace {

constexpr int kMaxSweeps = 40;
// A sweep whose largest rotated pair had |x.y| <= kStopRatio ||x|| ||y||
// ends the iteration: one-sided Jacobi converges quadratically, so the next
// sweep would start near (kStopRatio)^2 times a constant that grows as
// singular values cluster -- under the rotation threshold r u64 for
// well-separated values (it would only confirm convergence), and ~1e-12 in a
// host model with ten values equal to 1e-10, whose columns are then
// orthogonal to that level.
constexpr float kStopRatio = 3e-9f;

struct JacRowsArgs {
  const double* R;      // r x r row-major (ldr), upper triangular
  int64_t ldr;
  int r, rs;            // columns / column length; rs = r rounded up to even
  int b;                // columns per block
  double* Wg;           // out: rotated columns, column c at Wg + c * rs
  int* sweeps;          // out: sweeps taken (for tests and tuning)
};

// One warp per column pair.  The FP64 pipe of a GB300 SM retires 2 FMAs per
// clock, shared by its four schedulers (a warp instruction holds a
// scheduler's share for ~64 cycles, also the latency of a dependent one), so
// a CTA keeps b = 4 warps (one pair each) busy per sub-round and each pair
// step issues as few FP64 instructions as possible: the dot product g = x.y
// (one FMA per element and a shuffle tree) and the rotation (four per
// element) run in FP64; the control arithmetic runs on the FP32 pipe.
//   * The squared column norms a, b are tracked through the rotations in
//     double-float (a' = (a - 2 t g + t^2 b) / (1 + t^2)), recomputed from the
//     columns in FP64 at the start of every sweep.
//   * The angle t = tan(theta) is solved in double-float from them and g.
//   * c and s are built in FP64 from the FP32 c~ = (1 + t^2)^-1/2: with
//     kappa = c~^2 (1 + t^2) (FP64; c~^2 is an exact product), c = c~ rho,
//     s = c~ t rho, rho = kappa^-1/2 = 1 - d/2 + 3 d^2 / 8 for d = kappa - 1
//     ~ 1e-7, so c^2 + s^2 = 1 to FP64 rounding: the rotation is orthogonal
//     whatever the accuracy of t (a less accurate angle only leaves a smaller
//     off-diagonal for the next sweep).
//
// shared layout per CTA: buf[parity][slot] = b columns of rs doubles,
// nrm[parity][slot][b] (tracked squared norms, double-float), ids[parity]
// [slot][b] (global column index, -1 for pad), per-sweep rotation counters
__global__ void __launch_bounds__(256, 1) k_jacobi_rows_cl(JacRowsArgs a) {
  extern __shared__ double jsm[];
  cg::cluster_group cl = cg::this_cluster();
  const int NC = (int)cl.num_blocks();
  const int me = (int)cl.block_rank();
  const int b = a.b, rs = a.rs, r = a.r;
  const int blk = b * rs;                               // doubles per block
  double* buf = jsm;                                    // [2][2][blk]
  float2* nrm = reinterpret_cast<float2*>(buf + 4 * blk);   // [2][2][b] (hi, lo)
  int* ids = reinterpret_cast<int*>(nrm + 4 * b);       // [2][2][b]
  int* rotc = ids + 4 * b;                              // [kMaxSweeps] (CTA 0's copy is the sum)
  unsigned* rmx = reinterpret_cast<unsigned*>(rotc + kMaxSweeps);   // [kMaxSweeps] largest pair ratio (float bits)
  __shared__ int s_rot;
  __shared__ unsigned s_rmx;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  const int nb2 = 2 * NC;

  // ---- round 0: CTA i holds block i (slot 0) and block 2 NC - 1 - i (slot 1)
  for (int e = tid; e < 2 * blk; e += nth) {
    const int slot = e / blk, w = e - slot * blk;
    const int j = w / rs, i = w - j * rs;
    const int blockid = slot == 0 ? me : nb2 - 1 - me;
    const int c = blockid * b + j;                       // column c of X = row c of R
    buf[slot * blk + w] = (c < r && i < r) ? a.R[(int64_t)c * a.ldr + i] : 0.0;
  }
  for (int e = tid; e < 2 * b; e += nth) {
    const int slot = e / b, j = e - slot * b;
    const int blockid = slot == 0 ? me : nb2 - 1 - me;
    const int c = blockid * b + j;
    ids[slot * b + j] = c < r ? c : -1;
  }
  for (int e = tid; e < kMaxSweeps; e += nth) { rotc[e] = 0; rmx[e] = 0u; }
  cl.sync();                                            // every CTA started; DSMEM usable

  // a pair is orthogonal once |x.y| <= tol ||x|| ||y||
  const float tolf = 1.1102230246251565e-16f * (float)(r > 16 ? r : 16);

  float mxr = 0.f;                                      // this warp's largest rotated pair ratio this sweep
  // rotate the pair (x, y) with tracked squared norms (na, nb) in place (one warp)
  auto rotate = [&](double* x, double* y, float2* na, float2* nb) -> int {
    double gg = 0.0;
    for (int i = lane; i < rs; i += 32) gg = fma(x[i], y[i], gg);
    gg = warp_sum(gg);
    const df32 g = df_from_f64(gg);
    const float2 av = *na, bv = *nb;
    const df32 aa{av.x, av.y}, bb{bv.x, bv.y};
    if (g.hi == 0.0f || fabsf(g.hi) <= tolf * (sqrtf(aa.hi) * sqrtf(bb.hi))) return 0;
    mxr = fmaxf(mxr, fabsf(g.hi) / (sqrtf(aa.hi) * sqrtf(bb.hi)));
    // zeta = (b - a) / (2 g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
    // in double-float: an angle accurate to ~1e-14 keeps the convergence of
    // the last sweeps quadratic
    const df32 dd = df_add(bb, df_neg(aa));
    const df32 zeta = df_div(dd, df32{2.0f * g.hi, 2.0f * g.lo});
    df32 t;
    if (fabsf(zeta.hi) > 1e18f) {
      t = df_div(df_from_f(0.5f), zeta);                 // 1 / (2 zeta): 1 + zeta^2 overflows
    } else {
      const df32 w = df_sqrt(df_add(df_from_f(1.0f), df_mul(zeta, zeta)));
      const df32 den = df_add(zeta.hi < 0.0f ? df_neg(zeta) : zeta, w);
      t = df_div(df_from_f(zeta.hi < 0.0f ? -1.0f : 1.0f), den);
    }
    const float tf = t.hi;
    if (!(tf != 0.0f)) return 0;
    const float cf = rsqrtf(fmaf(tf, tf, 1.0f));
    const double td = widen_f32(tf) + widen_f32(t.lo), cd = widen_f32(cf);
    const double sd = cd * td;
    const double kap = (cd * cd) * fma(td, td, 1.0);     // c~^2 exact, one rounding each after
    const double dlt = kap - 1.0;                        // exact (kappa ~ 1)
    const double rho = fma(dlt, fma(dlt, 0.375, -0.5), 1.0);
    const double cs = cd * rho, sn = sd * rho;           // cs^2 + sn^2 = rho^2 kappa = 1 + O(u64)
    for (int i = lane; i < rs; i += 32) {
      const double u = x[i], v = y[i];
      x[i] = fma(-sn, v, cs * u);
      y[i] = fma(sn, u, cs * v);
    }
    if (lane == 0) {
      // a' = (a - 2 t g + t^2 b) / (1 + t^2), b' = (b + 2 t g + t^2 a) / (1 + t^2),
      // 1 / (1 + t^2) = c~^2 / kappa = c~^2 (1 - d + d^2)
      const df32 tg2 = df_mul(g, df32{2.0f * t.hi, 2.0f * t.lo});
      const df32 t2df = df_mul(t, t);
      const df32 na2 = df_add(df_add(aa, df_neg(tg2)), df_mul(t2df, bb));
      const df32 nb2v = df_add(df_add(bb, tg2), df_mul(t2df, aa));
      const float c2 = __fmul_rn(cf, cf);
      const df32 q0{c2, __fmaf_rn(cf, cf, -c2)};
      float dh, dl;
      split_f64_f2(dlt, dh, dl);
      const df32 rho2 = df_add(df_from_f(1.0f), df32{-dh, -dl + dh * dh});
      const df32 q = df_mul(q0, rho2);
      const df32 ra = df_mul(na2, q), rb = df_mul(nb2v, q);
      *na = make_float2(ra.hi, ra.lo);
      *nb = make_float2(rb.hi, rb.lo);
    }
    __syncwarp();
    return 1;
  };
  // squared norms of the columns this CTA holds (start of every sweep), FP64
  auto renorm = [&](int p) {
    for (int q = wid; q < 2 * b; q += nw) {
      const int slot = q / b, j = q - slot * b;
      const double* x = buf + (p * 2 + slot) * blk + j * rs;
      double t = 0.0;
      for (int i = lane; i < rs; i += 32) t = fma(x[i], x[i], t);
      t = warp_sum(t);
      if (lane == 0) {
        float h, l;
        split_f64_f2(t, h, l);
        nrm[(p * 2 + slot) * b + j] = make_float2(h, l);
      }
    }
  };

  int par = 0, sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) { s_rot = 0; s_rmx = 0u; }
    mxr = 0.f;
    renorm(par);
    __syncthreads();
    int nrot = 0;                                       // lane 0 of each warp counts
    for (int round = 0; round < nb2 - 1; ++round) {
      double* A0 = buf + (par * 2 + 0) * blk;
      double* B0 = buf + (par * 2 + 1) * blk;
      float2* nA = nrm + (par * 2 + 0) * b;
      float2* nB = nrm + (par * 2 + 1) * b;
      const int* idA = ids + (par * 2 + 0) * b;
      const int* idB = ids + (par * 2 + 1) * b;
      if (round == 0) {
        // internal pairs of both blocks: round-robin within a block, b' = b
        // rounded up to even, pairs (u, b' - 1 - u) with slot 0 fixed
        const int bp = (b + 1) & ~1;
        for (int sr = 0; sr < bp - 1; ++sr) {
          for (int pr = wid; pr < bp; pr += nw) {        // bp / 2 pairs per block, 2 blocks
            const int which = pr / (bp / 2), u = pr % (bp / 2);
            auto slotpos = [&](int sidx) -> int {
              if (sidx == 0) return 0;
              int v = sidx - 1 + sr;
              if (v >= bp - 1) v -= bp - 1;
              return 1 + v;
            };
            int p = slotpos(u), q = slotpos(bp - 1 - u);
            if (p > q) { const int tt = p; p = q; q = tt; }
            if (q >= b) continue;
            const int* id = which == 0 ? idA : idB;
            if (id[p] < 0 || id[q] < 0) continue;
            double* base = which == 0 ? A0 : B0;
            float2* nn = which == 0 ? nA : nB;
            nrot += rotate(base + p * rs, base + q * rs, nn + p, nn + q);
          }
          __syncthreads();
        }
      }
      // cross pairs: sub-round u pairs column j of A with column (j + u) mod b of B
      for (int u = 0; u < b; ++u) {
        for (int j = wid; j < b; j += nw) {
          int q = j + u;
          if (q >= b) q -= b;
          if (idA[j] < 0 || idB[q] < 0) continue;
          nrot += rotate(A0 + j * rs, B0 + q * rs, nA + j, nB + q);
        }
        __syncthreads();
      }
      // ---- hand the blocks on (tournament rotation of positions 1 .. 2NC-1) ----
      // slot 0 of CTA i is position i, slot 1 is position 2NC-1-i.  Position p
      // moves to p + 1 (2NC-1 wraps to 1); position 0 stays.
      const int npar = par ^ 1;
      for (int slot = 0; slot < 2; ++slot) {
        const int pos = slot == 0 ? me : nb2 - 1 - me;
        int dpos = pos == 0 ? 0 : (pos == nb2 - 1 ? 1 : pos + 1);
        const int dcta = dpos < NC ? dpos : nb2 - 1 - dpos;
        const int dslot = dpos < NC ? 0 : 1;
        double* dst = cl.map_shared_rank(buf + (npar * 2 + dslot) * blk, dcta);
        float2* dnr = cl.map_shared_rank(nrm + (npar * 2 + dslot) * b, dcta);
        int* did = cl.map_shared_rank(ids + (npar * 2 + dslot) * b, dcta);
        const double* src = buf + (par * 2 + slot) * blk;
        for (int e = tid; e < blk; e += nth) dst[e] = src[e];
        const float2* snr = nrm + (par * 2 + slot) * b;
        const int* sid = ids + (par * 2 + slot) * b;
        for (int e = tid; e < b; e += nth) { dnr[e] = snr[e]; did[e] = sid[e]; }
      }
      if (round == nb2 - 2) {
        if (lane == 0 && nrot) atomicAdd(&s_rot, nrot);
        if (lane == 0 && mxr > 0.f) atomicMax(&s_rmx, __float_as_uint(mxr));
        __syncthreads();                                 // s_rot, s_rmx complete
        if (tid == 0 && s_rot) atomicAdd(cl.map_shared_rank(rotc + sweep, 0), s_rot);
        if (tid == 0 && s_rmx) atomicMax(cl.map_shared_rank(rmx + sweep, 0), s_rmx);
      }
      cl.sync();
      par = npar;
    }
    // every CTA reads the same sum, after the barrier that ordered the adds
    const int total = *cl.map_shared_rank(rotc + sweep, 0);
    const float biggest = __uint_as_float(*cl.map_shared_rank(rmx + sweep, 0));
    if (total == 0 || biggest <= kStopRatio) { ++sweep; break; }
  }
  // rotated columns out, by global column index
  for (int slot = 0; slot < 2; ++slot) {
    const double* src = buf + (par * 2 + slot) * blk;
    const int* sid = ids + (par * 2 + slot) * b;
    for (int e = tid; e < blk; e += nth) {
      const int j = e / rs, i = e - j * rs;
      const int c = sid[j];
      if (c >= 0) a.Wg[(int64_t)c * rs + i] = src[e];
    }
  }
  if (me == 0 && tid == 0) *a.sweeps = sweep;
  cl.sync();                                            // no CTA leaves while others may read its memory
}

// s_k = column norms of W (descending, ties by index) and U_B[perm[i]][k] =
// W[order[k]][i] / s_k (zero column when s_k = 0).  The norms are ranked by
// their bit patterns as 64-bit integers (the order of non-negative doubles;
// a total order on any bits, so the ranks are always a permutation) on the
// integer pipe, and each column is scaled by one reciprocal: FP64 compares
// and divides issue over ~64 cycles per warp instruction on this part.
__global__ void __launch_bounds__(1024) k_jacobi_rows_finish(const double* __restrict__ W, int r, int rs,
                                                             const int32_t* __restrict__ perm,
                                                             double* __restrict__ Ub, double* __restrict__ s_out) {
  __shared__ double s_norm[1024];
  __shared__ long long s_key[1024];
  __shared__ double s_inv[1024];
  __shared__ int order[1024];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < r; c += nw) {
    double t = 0.0;
    for (int i = lane; i < r; i += 32) t = fma(W[(int64_t)c * rs + i], W[(int64_t)c * rs + i], t);
    t = warp_sum(t);
    if (lane == 0) {
      const double sv = sqrt(t);
      s_norm[c] = sv;
      s_key[c] = __double_as_longlong(sv);
      s_inv[c] = sv > 0.0 ? 1.0 / sv : 0.0;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    int rank = 0;
    const long long v = s_key[c];
    for (int d = 0; d < r; ++d) {
      const long long u = s_key[d];
      rank += (u > v || (u == v && d < c)) ? 1 : 0;
    }
    order[rank] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, k = e - i * r;               // position i, singular index k
    const int c = order[k];
    const int row = perm ? perm[i] : i;
    const double w = W[(int64_t)c * rs + i], sv = s_norm[c];
    // the reciprocal is finite down to 2^-1000 (far below any kept norm)
    Ub[(int64_t)row * r + k] = sv >= 0x1p-1000 ? w * s_inv[c] : (sv > 0.0 ? w / sv : 0.0);
  }
  for (int k = threadIdx.x; k < r; k += blockDim.x) s_out[k] = s_norm[order[k]];
}

struct ClusterPlan {
  int nc = 0, b = 0, threads = 0;
  size_t smem = 0;
};

size_t rows_smem(int b, int rs) {
  return sizeof(double) * (size_t)(4 * b * rs) + sizeof(float2) * (size_t)(4 * b) +
         sizeof(int) * (size_t)(4 * b + 2 * kMaxSweeps) + 64;
}

bool cluster_fits(int nc, int threads, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nc);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, (const void*)k_jacobi_rows_cl, &cfg);
  if (e != cudaSuccess) { cudaGetLastError(); return false; }
  return nclusters >= 1;
}

// Blocks of 4 columns give each CTA four pairs per sub-round (a warp each, one
// per scheduler), and as many CTAs as that leaves (r / 8, at most 16): the
// per-SM FP64 throughput is the bound, so the sweep is spread as widely as
// the pair count allows while every CTA still fills its four schedulers.
ClusterPlan plan_for(int r) {
  ClusterPlan pl;
  const int rs = (r + 1) & ~1;
  int b = 4;
  int nc = (r + 2 * b - 1) / (2 * b);
  if (nc > 16) { nc = 16; b = (r + 31) / 32; }
  if (nc < 2) { nc = 2; b = (r + 3) / 4; }
  for (; nc >= 2; --nc) {
    const int bb = (r + 2 * nc - 1) / (2 * nc);
    if (bb > 8) break;                                   // 8 warps per CTA at most
    const int bp = (bb + 1) & ~1;
    const int threads = 32 * (bp > 2 ? bp : 2);
    const size_t smem = rows_smem(bb, rs);
    if (cluster_fits(nc, threads, smem)) {
      pl.nc = nc; pl.b = bb; pl.threads = threads; pl.smem = smem;
      return pl;
    }
  }
  return pl;
}

}  // namespace

size_t jacobi_rows_ws(int64_t r) {
  const int64_t rs = (r + 1) & ~int64_t(1);
  return ((sizeof(double) * (size_t)(r * rs) + 255) & ~size_t(255)) + 512;
}

lrs_status launch_jacobi_rows(lrs_ctx* ctx, const double* R, int64_t r, int64_t ldr, const int32_t* perm,
                              double* Ub, double* s) {
  if (r < 8 || r > 1024) return LRS_ERANK;
  static int attr_set[64] = {0};
  if (ctx->device >= 0 && ctx->device < 64 && !attr_set[ctx->device]) {
    // clusters above 8 CTAs are opt-in
    const cudaError_t e = cudaFuncSetAttribute((const void*)k_jacobi_rows_cl,
                                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();
    attr_set[ctx->device] = 1;
  }
  const int ri = (int)r;
  ClusterPlan pl = plan_for(ri);
  if (pl.nc < 2) return LRS_ERANK;
  if (pl.smem > 48 * 1024) {
    const lrs_status st = raise_dyn_smem(ctx, (const void*)k_jacobi_rows_cl, pl.smem);
    if (st) return st;
  }
  const int rs = (ri + 1) & ~1;
  double* Wg = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(r * rs));
  int* sweeps = (int*)ws_alloc(ctx, 256);
  if (!Wg || !sweeps) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cluster Jacobi)");
  JacRowsArgs a{R, ldr, ri, rs, pl.b, Wg, sweeps};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)pl.nc);
  cfg.blockDim = dim3((unsigned)pl.threads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)pl.nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  LRS_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, k_jacobi_rows_cl, a));
  k_jacobi_rows_finish<<<1, 1024, 0, ctx->stream>>>(Wg, ri, rs, perm, Ub, s);
  ctx->launches += 2;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
