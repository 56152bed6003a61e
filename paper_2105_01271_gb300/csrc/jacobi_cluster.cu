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
// b x b cross pairs in b conflict-free sub-rounds (a team of kTeam lanes per
// pair, FP64 throughout), then sends each block it gives up straight into
// the shared memory of the CTA that takes it next (distributed shared memory),
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

constexpr int kTeam = 8;             // lanes per column pair
constexpr int kMaxSweeps = 40;

struct JacRowsArgs {
  const double* R;      // r x r row-major (ldr), upper triangular
  int64_t ldr;
  int r, rs;            // columns / column length; rs = r rounded up to even
  int b;                // columns per block
  double* Wg;           // out: rotated columns, column c at Wg + c * rs
  int* sweeps;          // out: sweeps taken (for tests and tuning)
};

// shared layout per CTA: buf[parity][slot] = b columns of rs doubles, then
// ids[parity][slot][b] (global column index, -1 for pad), counters
__global__ void __launch_bounds__(256, 1) k_jacobi_rows_cl(JacRowsArgs a) {
  extern __shared__ double jsm[];
  cg::cluster_group cl = cg::this_cluster();
  const int NC = (int)cl.num_blocks();
  const int me = (int)cl.block_rank();
  const int b = a.b, rs = a.rs, r = a.r;
  const int blk = b * rs;                               // doubles per block
  double* buf = jsm;                                    // [2][2][blk]
  int* ids = reinterpret_cast<int*>(buf + 4 * blk);     // [2][2][b]
  int* rotc = ids + 4 * b;                              // [kMaxSweeps] (CTA 0's copy is the sum)
  __shared__ int s_rot;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lg = tid % kTeam, team = tid / kTeam, nteam = nth / kTeam;
  const int lane = tid & 31;
  const unsigned gmask = ((1u << kTeam) - 1u) << (lane & (32 - kTeam));
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
  for (int e = tid; e < kMaxSweeps; e += nth) rotc[e] = 0;
  cl.sync();                                            // every CTA started; DSMEM usable

  const double eps = 1.1102230246251565e-16;
  const double tol = eps * (double)(r > 16 ? r : 16);   // |x.y| <= tol ||x|| ||y||: orthogonal
  const double tol2 = tol * tol;

  // rotate the pair (x, y) of columns in place (a team of kTeam lanes)
  auto rotate = [&](double* x, double* y) -> int {
    double aa = 0.0, bb = 0.0, gg = 0.0;
    for (int i = lg; i < rs; i += kTeam) {
      const double u = x[i], v = y[i];
      aa = fma(u, u, aa); bb = fma(v, v, bb); gg = fma(u, v, gg);
    }
#pragma unroll
    for (int o = kTeam / 2; o > 0; o >>= 1) {
      aa += __shfl_xor_sync(gmask, aa, o);
      bb += __shfl_xor_sync(gmask, bb, o);
      gg += __shfl_xor_sync(gmask, gg, o);
    }
    if (gg == 0.0 || gg * gg <= tol2 * (aa * bb)) return 0;
    const double zeta = (bb - aa) / (2.0 * gg);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    const double cs = 1.0 / sqrt(1.0 + t * t);
    const double sn = cs * t;
    for (int i = lg; i < rs; i += kTeam) {
      const double u = x[i], v = y[i];
      x[i] = cs * u - sn * v;
      y[i] = sn * u + cs * v;
    }
    return 1;
  };

  int par = 0, sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < nb2 - 1; ++round) {
      double* A0 = buf + (par * 2 + 0) * blk;
      double* B0 = buf + (par * 2 + 1) * blk;
      const int* idA = ids + (par * 2 + 0) * b;
      const int* idB = ids + (par * 2 + 1) * b;
      int nrot = 0;
      if (round == 0) {
        // internal pairs of both blocks: round-robin within a block, b' = b
        // rounded up to even, pairs (u, b' - 1 - u) with slot 0 fixed
        const int bp = (b + 1) & ~1;
        for (int sr = 0; sr < bp - 1; ++sr) {
          for (int pr = team; pr < bp; pr += nteam) {      // bp / 2 pairs per block, 2 blocks
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
            const int did = rotate(base + p * rs, base + q * rs);
            if (lg == 0) nrot += did;
          }
          __syncthreads();
        }
      }
      // cross pairs: sub-round u pairs column j of A with column (j + u) mod b of B
      for (int u = 0; u < b; ++u) {
        for (int j = team; j < b; j += nteam) {
          int q = j + u;
          if (q >= b) q -= b;
          if (idA[j] < 0 || idB[q] < 0) continue;
          const int did = rotate(A0 + j * rs, B0 + q * rs);
          if (lg == 0) nrot += did;
        }
        __syncthreads();
      }
      if (lg == 0 && nrot) atomicAdd(&s_rot, nrot);
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
        int* did = cl.map_shared_rank(ids + (npar * 2 + dslot) * b, dcta);
        const double* src = buf + (par * 2 + slot) * blk;
        for (int e = tid; e < blk; e += nth) dst[e] = src[e];
        const int* sid = ids + (par * 2 + slot) * b;
        for (int e = tid; e < b; e += nth) did[e] = sid[e];
      }
      if (round == nb2 - 2) {
        __syncthreads();                                 // s_rot complete
        if (tid == 0 && s_rot) atomicAdd(cl.map_shared_rank(rotc + sweep, 0), s_rot);
      }
      cl.sync();
      par = npar;
    }
    // every CTA reads the same sum, after the barrier that ordered the adds
    const int total = *cl.map_shared_rank(rotc + sweep, 0);
    if (total == 0) { ++sweep; break; }
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
// W[order[k]][i] / s_k (zero column when s_k = 0)
__global__ void __launch_bounds__(1024) k_jacobi_rows_finish(const double* __restrict__ W, int r, int rs,
                                                             const int32_t* __restrict__ perm,
                                                             double* __restrict__ Ub, double* __restrict__ s_out) {
  __shared__ double s_norm[1024];
  __shared__ int order[1024];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < r; c += nw) {
    double t = 0.0;
    for (int i = lane; i < r; i += 32) t = fma(W[(int64_t)c * rs + i], W[(int64_t)c * rs + i], t);
    t = warp_sum(t);
    if (lane == 0) s_norm[c] = sqrt(t);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    int rank = 0;
    const double v = s_norm[c];
    for (int d = 0; d < r; ++d) {
      const double u = s_norm[d];
      if (u > v || (u == v && d < c)) ++rank;
    }
    order[rank] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, k = e - i * r;               // position i, singular index k
    const int c = order[k];
    const double sv = s_norm[c];
    const int row = perm ? perm[i] : i;
    Ub[(int64_t)row * r + k] = sv > 0.0 ? W[(int64_t)c * rs + i] / sv : 0.0;
  }
  for (int k = threadIdx.x; k < r; k += blockDim.x) s_out[k] = s_norm[order[k]];
}

struct ClusterPlan {
  int nc = 0, b = 0, threads = 0;
  size_t smem = 0;
};

size_t rows_smem(int b, int rs) {
  return sizeof(double) * (size_t)(4 * b * rs) + sizeof(int) * (size_t)(4 * b + kMaxSweeps) + 64;
}

// cluster size: the padded column count 2 NC b should stay close to r (pad
// columns cost pairs) while NC is as large as the hardware schedules
// (per-SM FP64 throughput is the bound); estimate the sweep cost as the
// per-CTA pair work plus a barrier term per round
ClusterPlan plan_for(lrs_ctx* ctx, int r) {
  ClusterPlan best;
  double best_cost = 1e300;
  const int rs = (r + 1) & ~1;
  for (int nc = 16; nc >= 2; --nc) {
    const int b = (r + 2 * nc - 1) / (2 * nc);
    if (b < 1) continue;
    const int cols = 2 * nc * b;
    const double pairs_per_cta = (double)cols * (cols - 1) / 2.0 / nc;
    const double cost = pairs_per_cta * (double)rs / kTeam + 120.0 * (2 * nc - 1);
    if (cost < best_cost) {
      // can the device schedule a cluster of this size with this shared memory?
      int threads = ((b * kTeam + 31) / 32) * 32;
      if (threads < 64) threads = 64;
      if (threads > 256) threads = 256;
      const size_t smem = rows_smem(b, rs);
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
      if (e != cudaSuccess) { cudaGetLastError(); continue; }
      if (nclusters < 1) continue;
      best_cost = cost;
      best.nc = nc; best.b = b; best.threads = threads; best.smem = smem;
    }
  }
  return best;
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
  ClusterPlan pl = plan_for(ctx, ri);
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
