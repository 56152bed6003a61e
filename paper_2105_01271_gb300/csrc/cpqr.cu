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
// One persistent cooperative launch runs all steps.  The matrix is split by
// ROWS: block b keeps rows [r_lo, r_hi) of every column (in shared memory
// when the slab fits), so all SMs share the FP64 work whatever the aspect
// ratio.  Column sums (norms^2, Householder dot products) are reduced across
// blocks through per-block partials; block b owns the final sum of a
// contiguous range of columns.  One step j:
//   (F) every block updates its rows >= j of the live columns with the
//       previous reflector, records row j-1 of R if it owns that row, writes
//       partial norms^2 over rows >= j, and the owner of row j publishes row j
//                                                          -- grid barrier --
//   (N) column owners sum the norms^2 and their local best (norm^2, position)
//                                                          -- grid barrier --
//   (P) every block picks the pivot, forms its rows of v (needs only
//       ||x||, x_0 and its own rows of x) and writes partial dots v^T M(:, c)
//                                                          -- grid barrier --
//   (D) column owners sum the dots                         -- grid barrier --
// The barriers are bounded (common.cuh) and report LRS_ETIMEOUT.
#include "common.cuh"
#include "internal.h"

namespace lrs {

struct CpqrState {
  double* M; int64_t p, c, ldm;          // column-major input (column j at M + j*ldm), read once
  int64_t kmax; double rtol;
  // outputs
  int32_t* perm; double* R; double* V; double* tail2; int32_t* rank;
  // scratch
  double* slab_g;       // global per-block regions when shared memory is too small
  double* part_n;       // nb x c partial norms^2
  double* part_d;       // nb x c partial dot products
  double* colsum;       // c: reduced sums (owner mode)
  double* rowbuf;       // c: the current row j
  double* Rphys;        // kmax x c (row j, physical column)
  double* best_val;     // nb
  int32_t* best_pos;    // nb
  int32_t* best_phys;   // nb
  GridBarrier bar;
  int64_t rows_b;       // rows per block
  int64_t lds;          // slab column stride (odd: no shared-memory bank conflicts)
  int64_t region;       // doubles per block region: lds*c (slab) + rows_b (v) + c (sums)
  int slab_in_smem;
  int redundant;        // 1: every block reduces every column (2 barriers per step)
  int team;             // threads per column in the update and dot phases (1..8, power of 2)
};

__device__ __forceinline__ bool better(double a, int pa, double b, int pb) { return pivot_better(a, pa, b, pb); }

// block-wide argmax over (val, pos, phys); thread 0 ends with the winner
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

constexpr int kCpqrThreads = 512;
constexpr int kCpqrMaxBlocks = 160;

// One warp sums part[b * c + cc] over the nb blocks (lane-strided, fixed
// shuffle tree: the same order in every block and every run).
__device__ __forceinline__ double warp_sum_blocks(const double* part, int64_t c, int64_t cc, int nb, int lane) {
  double a = 0.0;
  for (int bb = lane; bb < nb; bb += 32) a += __ldcg(part + (int64_t)bb * c + cc);
  return warp_sum(a);
}

// The same for up to 4 columns cc0 + k*stride at once: every load is issued
// before the first add, so the L2 latency is paid once, not once per column.
template <int NC>
__device__ __forceinline__ void warp_sum_blocks_n(const double* part, int64_t c, int64_t cc0, int64_t stride,
                                                  int ncol, int nb, int lane, double (&out)[NC]) {
  double acc[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) acc[k] = 0.0;
  for (int bb = lane; bb < nb; bb += 32) {
    double v[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) v[k] = k < ncol ? __ldcg(part + (int64_t)bb * c + cc0 + k * stride) : 0.0;
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] += v[k];
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) out[k] = warp_sum(acc[k]);
}

// Sum of part[bb * c + cc] over the nb blocks by the 4 lanes (q4 = 0..3) of
// one column: lane q4 takes bb = q4, q4+4, ... with four loads in flight, then
// two shuffles.  nb - 1 FP64 additions per column, the same order everywhere.
// All 32 lanes of the warp must call it (the shuffles use the full mask).
__device__ __forceinline__ double sum4_blocks(const double* part, int64_t c, int64_t cc, bool valid, int nb,
                                              int q4) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (valid) {
    int bb = q4;
    for (; bb + 12 < nb; bb += 16) {
      a0 += __ldcg(part + (int64_t)bb * c + cc);
      a1 += __ldcg(part + (int64_t)(bb + 4) * c + cc);
      a2 += __ldcg(part + (int64_t)(bb + 8) * c + cc);
      a3 += __ldcg(part + (int64_t)(bb + 12) * c + cc);
    }
    for (; bb < nb; bb += 4) a0 += __ldcg(part + (int64_t)bb * c + cc);
  }
  double a = (a0 + a1) + (a2 + a3);
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  a += __shfl_xor_sync(0xffffffffu, a, 2);
  return a;
}

// Sum of part[bb * c + cc] over the nb (<= 160) blocks by one warp: every
// lane issues its (at most 5) loads before the first add, so the L2 latency is
// paid once; then a fixed shuffle tree (the same order in every block and
// run).  Used in owner mode, where a block owns only a few columns.
__device__ __forceinline__ double warp_sum_blocks_wide(const double* part, int64_t c, int64_t cc, int nb,
                                                       int lane) {
  double v[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int bb = lane + 32 * k;
    v[k] = bb < nb ? __ldcg(part + (int64_t)bb * c + cc) : 0.0;
  }
  double a = ((v[0] + v[1]) + (v[2] + v[3])) + v[4];
  return warp_sum(a);
}

__global__ void __launch_bounds__(kCpqrThreads, 1) k_cpqr(CpqrState s) {
  extern __shared__ double smem_d[];
  __shared__ double sv[32];
  __shared__ int sp[32], sf[32];
  __shared__ int s_piv, s_pivpos, s_stop;
  __shared__ double s_alpha, s_sgn, s_inv, s_x0;

  const int nb = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t r_lo = (int64_t)b * s.rows_b;
  const int64_t r_hi = min(s.p, r_lo + s.rows_b);
  const int64_t nr = r_hi > r_lo ? r_hi - r_lo : 0;      // rows of this block
  const int64_t cpb = (s.c + nb - 1) / nb;                // columns owned per block (owner mode)
  const int64_t o_lo = min(s.c, (int64_t)b * cpb), o_hi = min(s.c, o_lo + cpb);
  const int64_t c_lo = s.redundant ? 0 : o_lo, c_hi = s.redundant ? s.c : o_hi;
  double* slab = s.slab_in_smem ? smem_d : s.slab_g + (int64_t)b * s.region;   // column cc at slab + cc*lds
  double* vloc = slab + s.lds * s.c;                      // this block's rows of the reflector
  double* sums = vloc + s.rows_b;                         // reduced column sums (redundant mode)
  // every block keeps its own copy of the pivoting bookkeeping: all blocks
  // reach the same pivot decision, so the copies stay identical
  int32_t* pos_of = reinterpret_cast<int32_t*>(sums + s.c);   // physical -> position
  int32_t* phys_at = pos_of + s.c;                            // position -> physical
  uint8_t* done = reinterpret_cast<uint8_t*>(phys_at + s.c);
  double* pn = s.part_n + (int64_t)b * s.c;
  double* pd = s.part_d + (int64_t)b * s.c;

  for (int64_t e = threadIdx.x; e < nr * s.c; e += blockDim.x) {
    const int64_t cc = e / nr, i = e - cc * nr;
    slab[cc * s.lds + i] = s.M[cc * s.ldm + r_lo + i];
  }
  for (int64_t cc = threadIdx.x; cc < s.c; cc += blockDim.x) {
    pos_of[cc] = (int)cc; phys_at[cc] = (int)cc; done[cc] = 0;
  }
  __syncthreads();

  // Threads of one column "team" share its rows in (F) and (P); teams live
  // inside one warp (T divides 32), so team shuffles and syncs use a team mask.
  const int T = s.team;
  const int tm = threadIdx.x & (T - 1);
  const int team = threadIdx.x / T, nteams = blockDim.x / T;
  const unsigned tmask = (T == 32 ? 0xffffffffu : ((1u << T) - 1u)) << (lane & ~(T - 1));
  auto team_sum = [&](double v) {
    for (int o = 1; o < T; o <<= 1) v += __shfl_xor_sync(tmask, v, o);
    return v;
  };

  int64_t j = 0;
  double top = 0.0;
  for (;; ++j) {
    // ---- (F) apply H_{j-1}; row j-1 of R; partial norms^2 over rows >= j ---
    {
      const int64_t i0 = max(r_lo, j - 1) - r_lo;
      const int64_t in = max(r_lo, j) - r_lo;
      const bool upd = j > 0;
      const int64_t lprev = (upd && (j - 1) >= r_lo && (j - 1) < r_hi) ? (j - 1) - r_lo : -1;
      const int64_t lcur = (j >= r_lo && j < r_hi) ? j - r_lo : -1;
      for (int64_t cc = team; cc < s.c; cc += nteams) {
        double nrm = 0.0;
        double* col = slab + cc * s.lds;
        if (!done[cc]) {
          if (upd) {
            const double tw = 2.0 * (s.redundant ? sums[cc] : __ldcg(s.colsum + cc));
            for (int64_t i = i0 + tm; i < nr; i += T) {
              const double x = fma(-tw, vloc[i], col[i]);
              col[i] = x;
              if (i == lprev) s.Rphys[(j - 1) * s.c + cc] = x;
            }
            __syncwarp(tmask);
          }
          for (int64_t i = in + tm; i < nr; i += T) nrm = fma(col[i], col[i], nrm);
        }
        nrm = team_sum(nrm);
        if (tm == 0) {
          pn[cc] = nrm;
          if (lcur >= 0) s.rowbuf[cc] = col[lcur];
        }
      }
    }
    if (!grid_sync(s.bar)) return;

    // ---- (N) norms^2 and the best candidate -------------------------------
    {
      double bv = -1.0; int bp = 0x7fffffff, bf = -1;
      if (s.redundant) {
        // every block reduces every column: 4 lanes per column keep the FP64 adds few
        const int q4 = lane & 3, slot = lane >> 2;
        for (int64_t base = c_lo + wid * 8; base < c_hi; base += (int64_t)nw * 8) {
          const int64_t cc = base + slot;
          const double a = sum4_blocks(s.part_n, s.c, cc, cc < c_hi, nb, q4);
          if (cc < c_hi && !done[cc]) {
            if (q4 == 0) sums[cc] = a;
            const int pc = pos_of[cc];
            if (better(a, pc, bv, bp)) { bv = a; bp = pc; bf = (int)cc; }
          }
        }
      } else {
        // a block owns a few columns: a whole warp per column
        for (int64_t cc = c_lo + wid; cc < c_hi; cc += nw) {
          if (done[cc]) continue;
          const double a = warp_sum_blocks_wide(s.part_n, s.c, cc, nb, lane);
          if (lane == 0) {
            s.colsum[cc] = a;
            const int pc = pos_of[cc];
            if (better(a, pc, bv, bp)) { bv = a; bp = pc; bf = (int)cc; }
          }
        }

      }
      block_best(bv, bp, bf, sv, sp, sf);
      if (!s.redundant) {
        if (threadIdx.x == 0) { s.best_val[b] = bv; s.best_pos[b] = bp; s.best_phys[b] = bf; }
        if (!grid_sync(s.bar)) return;
        bv = -1.0; bp = 0x7fffffff; bf = -1;
        for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) {
          const double v = __ldcg(s.best_val + bb);
          const int pp = __ldcg(s.best_pos + bb);
          if (better(v, pp, bv, bp)) { bv = v; bp = pp; bf = __ldcg(s.best_phys + bb); }
        }
        block_best(bv, bp, bf, sv, sp, sf);
      }
      // thread 0 holds the global winner
      if (threadIdx.x == 0) {
        const double nrm = bv > 0.0 ? bv * rsqrt_fast(bv) : 0.0;
        if (j == 0) top = nrm;
        const bool stop = (j >= s.kmax) || bf < 0 || bv <= 0.0 || (j > 0 && nrm <= s.rtol * top);
        s_stop = stop ? 1 : 0;
        s_piv = bf; s_pivpos = bp;
        if (!stop) {
          const double x0 = __ldcg(s.rowbuf + bf);
          const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
          const double vn2 = 2.0 * nrm * (nrm + fabs(x0));     // ||x + sgn ||x|| e_j||^2
          s_alpha = nrm; s_sgn = sgn; s_x0 = x0;
          s_inv = vn2 > 0.0 ? rsqrt_fast(vn2) : 0.0;
        }
      }
      __syncthreads();
    }
    if (s_stop) break;

    // ---- (P) this block's rows of v and partial dots v^T M(:, c) ------------
    {
      const int piv = s_piv;
      const double inv = s_inv;
      const double* xcol = slab + (int64_t)piv * s.lds;
      for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) {
        const int64_t gi = r_lo + i;
        double vi = 0.0;
        if (gi == j) vi = (s_x0 + s_sgn * s_alpha) * inv;
        else if (gi > j) vi = xcol[i] * inv;
        vloc[i] = vi;
        s.V[j * s.p + gi] = vi;
      }
      if (threadIdx.x == 0) {
        const int pj = phys_at[j];
        const int pp = s_pivpos;
        phys_at[j] = piv; phys_at[pp] = pj;
        pos_of[piv] = (int)j; pos_of[pj] = pp;
        done[piv] = 1;
        if (b == 0) s.Rphys[j * s.c + piv] = -s_sgn * s_alpha;
      }
      __syncthreads();
      const int64_t i0 = max(r_lo, j) - r_lo;
      for (int64_t cc = team; cc < s.c; cc += nteams) {
        double d = 0.0;
        if (!done[cc]) {
          const double* col = slab + cc * s.lds;
          for (int64_t i = i0 + tm; i < nr; i += T) d = fma(vloc[i], col[i], d);
        }
        d = team_sum(d);
        if (tm == 0) pd[cc] = d;
      }
    }
    if (!grid_sync(s.bar)) return;

    // ---- (D) dots ------------------------------------------------------------
    {
      if (s.redundant) {
        const int q4 = lane & 3, slot = lane >> 2;
        for (int64_t base = c_lo + wid * 8; base < c_hi; base += (int64_t)nw * 8) {
          const int64_t cc = base + slot;
          const double a = sum4_blocks(s.part_d, s.c, cc, cc < c_hi, nb, q4);
          if (cc < c_hi && q4 == 0) sums[cc] = a;
        }
      } else {
        for (int64_t cc = c_lo + wid; cc < c_hi; cc += nw) {
          if (done[cc]) continue;
          const double a = warp_sum_blocks_wide(s.part_d, s.c, cc, nb, lane);
          if (lane == 0) s.colsum[cc] = a;
        }
      }
    }
    if (!s.redundant) {
      if (!grid_sync(s.bar)) return;
    } else {
      __syncthreads();
    }
  }

  // ---- epilogue: rank, permutation, R in pivoted order, trailing norm ------
  const int64_t r = j;
  if (b == 0) {
    if (threadIdx.x == 0) *s.rank = (int32_t)r;
    double t = 0.0;
    for (int64_t cc = threadIdx.x; cc < s.c; cc += blockDim.x)
      if (!done[cc]) t += s.redundant ? sums[cc] : __ldcg(s.colsum + cc);
    t = block_sum(t, sv);
    if (threadIdx.x == 0) *s.tail2 = (r < min(s.p, s.c)) ? t : 0.0;
    for (int64_t q = threadIdx.x; q < s.c; q += blockDim.x) s.perm[q] = phys_at[q];
  }
  for (int64_t e = (int64_t)b * blockDim.x + threadIdx.x; e < r * s.c; e += (int64_t)nb * blockDim.x) {
    const int64_t i = e / s.c, q = e - i * s.c;
    s.R[i * s.c + q] = (q < i) ? 0.0 : __ldcg(s.Rphys + i * s.c + phys_at[q]);
  }
}

// ---------------------------------------------------------------------------
// Column-owner form of the same factorisation, for c >= 128 columns whose
// owned slabs fit in shared memory.  Block b owns a contiguous range of
// physical columns with all their rows, so the Householder dot products and
// the norms are block-local and a step needs ONE grid barrier:
//   every block: v_j from the pivot column (read from the winner's slot),
//     H_j applied to its live columns (dot, update, row j of R), norms^2 over
//     rows > j, its best candidate published with a copy of that column
//                                                          -- grid barrier --
//   every block: the winner among the candidates (block order, so the same
//     decision everywhere), stop test, the position swap in its own copy of
//     the permutation.
// Candidates and candidate columns are double-buffered by step parity: a
// block still reading step j's slots never sees step j+1's writes.  Pivot,
// tie, reflector and stop rules are those of k_cpqr.
// ---------------------------------------------------------------------------
struct CpqrColsState {
  const double* M; int64_t p, c, ldm;    // column-major input, read once
  int64_t kmax; double rtol; int64_t cpb;
  int32_t* perm; double* R; double* V; double* tail2; int32_t* rank;
  double* Rphys;                         // kmax x c by physical column
  PivotCand* cand;                       // 2 x nb
  double* cand_col;                      // 2 x nb x p
  double* tail_part;                     // nb
  GridBarrier bar;
};

constexpr int kColsThreads = 512;

__global__ void __launch_bounds__(kColsThreads, 1) k_cpqr_cols(CpqrColsState s) {
  extern __shared__ double csm[];
  const int nb = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t p = s.p;
  const int64_t o_lo = min(s.c, (int64_t)b * s.cpb), o_hi = min(s.c, o_lo + s.cpb);
  const int nown = (int)(o_hi - o_lo);
  double* slab = csm;                         // nown x p (column cc at slab + cc * p)
  double* vv = slab + s.cpb * p;              // p: the reflector (rows >= j), first the pivot column
  double* nrm2 = vv + p;                      // cpb: remaining norms^2 of the owned columns
  int32_t* pos_of = reinterpret_cast<int32_t*>(nrm2 + s.cpb);
  int32_t* phys_at = pos_of + s.c;
  uint8_t* done = reinterpret_cast<uint8_t*>(phys_at + s.c);   // cpb
  __shared__ double sv[32];
  __shared__ int sp[32], sf[32];
  __shared__ int s_piv, s_stop;
  __shared__ double s_alpha, s_sgn, s_inv, s_top;

  for (int64_t e = threadIdx.x; e < (int64_t)nown * p; e += blockDim.x) {
    const int64_t cc = e / p, i = e - cc * p;
    slab[cc * p + i] = s.M[(o_lo + cc) * s.ldm + i];
  }
  for (int64_t q = threadIdx.x; q < s.c; q += blockDim.x) { pos_of[q] = (int)q; phys_at[q] = (int)q; }
  for (int64_t cc = threadIdx.x; cc < s.cpb; cc += blockDim.x) done[cc] = 0;
  __syncthreads();

  // norms^2 over rows >= r0 of the owned live columns (a warp per column)
  auto norms = [&](int64_t r0) {
    for (int cc = wid; cc < nown; cc += nw) {
      double a = 0.0;
      if (!done[cc]) {
        const double* col = slab + (int64_t)cc * p;
        for (int64_t i = r0 + lane; i < p; i += 32) a = fma(col[i], col[i], a);
      }
      a = warp_sum(a);
      if (lane == 0) nrm2[cc] = a;
    }
  };
  // best owned candidate -> buffer `buf`, with a copy of its column
  auto publish = [&](int buf) {
    __syncthreads();
    if (wid == 0) {
      double bv = -1.0; int bp = 0x7fffffff, bf = -1;
      for (int cc = lane; cc < nown; cc += 32) {
        if (done[cc]) continue;
        const int ph = (int)(o_lo + cc);
        if (pivot_better(nrm2[cc], pos_of[ph], bv, bp)) { bv = nrm2[cc]; bp = pos_of[ph]; bf = ph; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int of = __shfl_xor_sync(0xffffffffu, bf, o);
        if (pivot_better(ov, op, bv, bp)) { bv = ov; bp = op; bf = of; }
      }
      if (lane == 0) {
        cand_store(s.cand + buf * nb + b, bv, bp, bf);
        sf[0] = bf;
      }
    }
    __syncthreads();
    const int bf = sf[0];
    if (bf >= 0) {
      const double* col = slab + (bf - o_lo) * p;
      double* dst = s.cand_col + ((int64_t)buf * nb + b) * p;
      for (int64_t i = threadIdx.x; i < p; i += blockDim.x) dst[i] = col[i];
    }
  };

  norms(0);
  publish(0);
  if (!grid_sync(s.bar)) return;
  int64_t j = 0;
  for (;; ++j) {
    const int buf = (int)(j & 1);
    // ---- decide: the winner of buffer buf (every block, block order) -------
    {
      double bv = -1.0; int bp = 0x7fffffff, bf = -1;
      for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) {
        double v; int pp, pf;
        cand_load(s.cand + buf * nb + bb, v, pp, pf);
        if (pivot_better(v, pp, bv, bp)) { bv = v; bp = pp; bf = pf; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int of = __shfl_xor_sync(0xffffffffu, bf, o);
        if (pivot_better(ov, op, bv, bp)) { bv = ov; bp = op; bf = of; }
      }
      __syncthreads();
      if (lane == 0) { sv[wid] = bv; sp[wid] = bp; sf[wid] = bf; }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
          if (pivot_better(sv[w], sp[w], bv, bp)) { bv = sv[w]; bp = sp[w]; bf = sf[w]; }
        const double nrm = bv > 0.0 ? bv * rsqrt_fast(bv) : 0.0;
        if (j == 0) s_top = nrm;
        const bool stop = (j >= s.kmax) || bf < 0 || !(bv > 0.0) || (j > 0 && nrm <= s.rtol * s_top);
        s_stop = stop ? 1 : 0;
        if (!stop) {
          const int pj = phys_at[j];
          phys_at[j] = bf; phys_at[bp] = pj;
          pos_of[bf] = (int)j; pos_of[pj] = bp;
          if (bf >= o_lo && bf < o_hi) done[bf - o_lo] = 1;
          s_piv = bf; s_alpha = nrm;
        }
      }
      __syncthreads();
    }
    if (s_stop) break;
    const int piv = s_piv;
    // ---- the reflector from the winner's column (rows >= j) -----------------
    {
      const int64_t owner = piv / s.cpb;
      const double* src = s.cand_col + ((int64_t)buf * nb + owner) * p;
      for (int64_t i = j + threadIdx.x; i < p; i += blockDim.x) vv[i] = __ldcg(src + i);
      __syncthreads();
      if (threadIdx.x == 0) {
        const double x0 = vv[j], nrm = s_alpha;
        const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
        const double vn2 = 2.0 * nrm * (nrm + fabs(x0));
        s_sgn = sgn;
        s_inv = vn2 > 0.0 ? rsqrt_fast(vn2) : 0.0;
      }
      __syncthreads();
      const double inv = s_inv;
      for (int64_t i = j + threadIdx.x; i < p; i += blockDim.x)
        vv[i] = (i == j) ? (vv[i] + s_sgn * s_alpha) * inv : vv[i] * inv;
      __syncthreads();
      if (b == 0) {
        for (int64_t i = threadIdx.x; i < p; i += blockDim.x) s.V[j * p + i] = i < j ? 0.0 : vv[i];
        if (threadIdx.x == 0) s.Rphys[j * s.c + piv] = -s_sgn * s_alpha;
      }
    }
    // ---- H_j on the owned live columns, row j of R, norms over rows > j -----
    for (int cc = wid; cc < nown; cc += nw) {
      double a = 0.0;
      if (!done[cc]) {
        double* col = slab + (int64_t)cc * p;
        // four interleaved partial sums per lane (the FP64 latency chains)
        double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
        int64_t i = j + lane;
        for (; i + 96 < p; i += 128) {
          d0 = fma(vv[i], col[i], d0);
          d1 = fma(vv[i + 32], col[i + 32], d1);
          d2 = fma(vv[i + 64], col[i + 64], d2);
          d3 = fma(vv[i + 96], col[i + 96], d3);
        }
        for (; i < p; i += 32) d0 = fma(vv[i], col[i], d0);
        const double tw = 2.0 * warp_sum((d0 + d1) + (d2 + d3));
        if (lane == 0) {                              // row j of R
          const double x = fma(-tw, vv[j], col[j]);
          col[j] = x;
          s.Rphys[j * s.c + o_lo + cc] = x;
        }
        double n0 = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;
        i = j + 1 + lane;
        for (; i + 96 < p; i += 128) {
          const double x0 = fma(-tw, vv[i], col[i]), x1 = fma(-tw, vv[i + 32], col[i + 32]);
          const double x2 = fma(-tw, vv[i + 64], col[i + 64]), x3 = fma(-tw, vv[i + 96], col[i + 96]);
          col[i] = x0; col[i + 32] = x1; col[i + 64] = x2; col[i + 96] = x3;
          n0 = fma(x0, x0, n0); n1 = fma(x1, x1, n1); n2 = fma(x2, x2, n2); n3 = fma(x3, x3, n3);
        }
        for (; i < p; i += 32) {
          const double x = fma(-tw, vv[i], col[i]);
          col[i] = x;
          n0 = fma(x, x, n0);
        }
        a = (n0 + n1) + (n2 + n3);
      }
      a = warp_sum(a);
      if (lane == 0) nrm2[cc] = a;
    }
    publish((int)((j + 1) & 1));
    if (!grid_sync(s.bar)) return;
  }

  // ---- epilogue: rank, permutation, R in pivoted order, trailing norm --------
  const int64_t r = j;
  {
    double t = 0.0;
    for (int cc = threadIdx.x; cc < nown; cc += blockDim.x)
      if (!done[cc]) t += nrm2[cc];
    t = block_sum(t, sv);
    if (threadIdx.x == 0) s.tail_part[b] = t;
  }
  if (!grid_sync(s.bar)) return;
  if (b == 0) {
    if (threadIdx.x == 0) *s.rank = (int32_t)r;
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int bb = 0; bb < nb; ++bb) t += __ldcg(s.tail_part + bb);
    if (threadIdx.x == 0) *s.tail2 = (r < min(s.p, s.c)) ? t : 0.0;
    for (int64_t q = threadIdx.x; q < s.c; q += blockDim.x) s.perm[q] = phys_at[q];
  }
  for (int64_t e = (int64_t)b * blockDim.x + threadIdx.x; e < r * s.c; e += (int64_t)nb * blockDim.x) {
    const int64_t i = e / s.c, q = e - i * s.c;
    s.R[i * s.c + q] = (q < i) ? 0.0 : __ldcg(s.Rphys + i * s.c + phys_at[q]);
  }
}

struct ColsGeom { int64_t nb, cpb; size_t smem; };

ColsGeom cols_geom(int64_t p, int64_t c, int num_sms) {
  ColsGeom g{};
  g.cpb = (c + num_sms - 1) / num_sms;
  if (g.cpb < 1) g.cpb = 1;
  g.nb = (c + g.cpb - 1) / g.cpb;
  g.smem = sizeof(double) * (size_t)(g.cpb * p + p + g.cpb) + sizeof(int32_t) * (size_t)(2 * c) + (size_t)g.cpb + 16;
  return g;
}

bool cpqr_cols_eligible(int64_t p, int64_t c, int num_sms) {
  if (c < 128 || p < 1) return false;
  return cols_geom(p, c, num_sms).smem <= 200 * 1024;
}

size_t cpqr_cols_scratch_bytes(int64_t p, int64_t c, int64_t kmax, int num_sms) {
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const ColsGeom g = cols_geom(p, c, num_sms);
  size_t b = 0;
  b += a256(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1) * c);
  b += a256(sizeof(PivotCand) * (size_t)(2 * g.nb));
  b += a256(sizeof(double) * (size_t)(2 * g.nb * p));
  b += a256(sizeof(double) * (size_t)g.nb);
  b += 256;
  return b;
}

lrs_status launch_cpqr_cols(lrs_ctx* ctx, double* M, int64_t p, int64_t c, int64_t ldm,
                            int64_t kmax, double rtol, const CpqrOut& o) {
  const ColsGeom g = cols_geom(p, c, ctx->num_sms);
  CpqrColsState s{};
  s.M = M; s.p = p; s.c = c; s.ldm = ldm; s.kmax = kmax; s.rtol = rtol; s.cpb = g.cpb;
  s.perm = o.perm; s.R = o.R; s.V = o.V; s.tail2 = o.tail2; s.rank = o.rank;
  s.Rphys = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(kmax > 0 ? kmax : 1) * c);
  s.cand = (PivotCand*)ws_alloc(ctx, sizeof(PivotCand) * (size_t)(2 * g.nb));
  s.cand_col = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(2 * g.nb * p));
  s.tail_part = (double*)ws_alloc(ctx, sizeof(double) * (size_t)g.nb);
  unsigned* bar = (unsigned*)ws_alloc(ctx, 256);
  if (!s.Rphys || !s.cand || !s.cand_col || !s.tail_part || !bar)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpqr_cols)");
  if (g.smem > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_cpqr_cols, g.smem); if (_s) return _s; }
  int per_sm = 0;
  LRS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cpqr_cols, kColsThreads, g.smem));
  if (per_sm < 1 || g.nb > (int64_t)per_sm * ctx->num_sms)
    return lrs_fail(ctx, LRS_ECUDA, "cpqr_cols: %lld blocks do not fit", (long long)g.nb);
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, 256, ctx->stream));
  s.bar.count = bar; s.bar.gen = bar + 1; s.bar.err = (int*)(bar + 2);
  void* args[] = {&s};
  LRS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_cpqr_cols, dim3((unsigned)g.nb),
                                                dim3(kColsThreads), args, g.smem, ctx->stream));
  ctx->launches++;
  int* h = (int*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {(const int32_t*)(bar + 2)};
    const lrs_status rs = replay_ints(ctx, 1, d, h + 33);
    if (rs) return rs;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 33, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[33] != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "cpqr_cols: grid barrier wait gave up");
  return LRS_OK;
}

// Bytes launch_cpqr takes from the workspace for these sizes (the same block
// count, slab placement and 256-byte rounding as the launch below).
size_t cpqr_scratch_bytes(int64_t p, int64_t c, int64_t kmax, int num_sms) {
  if (cpqr_cols_eligible(p, c, num_sms)) return cpqr_cols_scratch_bytes(p, c, kmax, num_sms);
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  int64_t nb = (p * c + 2047) / 2048;
  if (nb > num_sms) nb = num_sms;
  if (nb > kCpqrMaxBlocks) nb = kCpqrMaxBlocks;
  if (nb > (p + 3) / 4) nb = (p + 3) / 4;
  if (nb < 1) nb = 1;
  const int64_t rows_b = (p + nb - 1) / nb;
  nb = (p + rows_b - 1) / rows_b;
  const int64_t lds = rows_b | 1;
  const int64_t region = lds * c + rows_b + c + (c + (c * 8 + 7) / 8 + 1);
  size_t b = 0;
  if (sizeof(double) * (size_t)region > 200 * 1024) b += a256(sizeof(double) * (size_t)(nb * region));
  b += 2 * a256(sizeof(double) * (size_t)(nb * c));
  b += 2 * a256(sizeof(double) * (size_t)c);
  b += a256(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1) * c);
  b += a256(sizeof(double) * (size_t)nb) + 2 * a256(sizeof(int32_t) * (size_t)nb);
  b += 256;
  return b;
}

lrs_status launch_cpqr(lrs_ctx* ctx, double* M, int64_t p, int64_t c, int64_t ldm,
                       int64_t kmax, double rtol, const CpqrOut& o) {
  if (!ctx->coop_ok) return lrs_fail(ctx, LRS_ECUDA, "device lacks cooperative launch");
  if (cpqr_cols_eligible(p, c, ctx->num_sms)) return launch_cpqr_cols(ctx, M, p, c, ldm, kmax, rtol, o);
  CpqrState s{};
  s.M = M; s.p = p; s.c = c; s.ldm = ldm; s.kmax = kmax; s.rtol = rtol;
  s.perm = o.perm; s.R = o.R; s.V = o.V; s.tail2 = o.tail2; s.rank = o.rank;
  // blocks: about 2048 matrix elements each (the FP64 work of one step per
  // block), at most one per SM, at least 4 rows each
  int64_t nb = (p * c + 2047) / 2048;
  if (nb > ctx->num_sms) nb = ctx->num_sms;
  if (nb > kCpqrMaxBlocks) nb = kCpqrMaxBlocks;   // the owner sums load <= 5 partials per lane
  if (nb > (p + 3) / 4) nb = (p + 3) / 4;
  if (nb < 1) nb = 1;
  s.rows_b = (p + nb - 1) / nb;
  nb = (p + s.rows_b - 1) / s.rows_b;
  s.lds = s.rows_b | 1;
  // per block: slab, v rows, column sums, then pos_of/phys_at (int32) and done (bytes)
  s.region = s.lds * c + s.rows_b + c + (c + (c * 8 + 7) / 8 + 1);
  s.redundant = (nb * c <= 24576) ? 1 : 0;
  s.team = c >= 512 ? 1 : (c >= 256 ? 2 : (c >= 128 ? 4 : 8));
  const size_t slab_bytes = sizeof(double) * (size_t)s.region;
  s.slab_in_smem = slab_bytes <= 200 * 1024 ? 1 : 0;
  const size_t dyn = s.slab_in_smem ? slab_bytes : 0;
  if (dyn > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_cpqr, (size_t)(dyn)); if (_s) return _s; }
  int per_sm = 0;
  LRS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cpqr, kCpqrThreads, dyn));
  if (per_sm < 1) return lrs_fail(ctx, LRS_ECUDA, "cpqr: kernel does not fit on an SM");
  if (!s.slab_in_smem) {
    s.slab_g = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(nb * s.region));
    if (!s.slab_g) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpqr slab)");
  }
  s.part_n = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(nb * c));
  s.part_d = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(nb * c));
  s.colsum = (double*)ws_alloc(ctx, sizeof(double) * c);
  s.rowbuf = (double*)ws_alloc(ctx, sizeof(double) * c);
  s.Rphys = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(kmax > 0 ? kmax : 1) * c);
  s.best_val = (double*)ws_alloc(ctx, sizeof(double) * nb);
  s.best_pos = (int32_t*)ws_alloc(ctx, sizeof(int32_t) * nb);
  s.best_phys = (int32_t*)ws_alloc(ctx, sizeof(int32_t) * nb);
  unsigned* bar = (unsigned*)ws_alloc(ctx, 256);
  if (!s.part_n || !s.part_d || !s.colsum || !s.rowbuf || !s.Rphys || !s.best_val || !s.best_pos || !s.best_phys || !bar)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (cpqr)");
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, 256, ctx->stream));
  s.bar.count = bar; s.bar.gen = bar + 1; s.bar.err = (int*)(bar + 2);
  void* args[] = {&s};
  LRS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_cpqr, dim3((unsigned)nb), dim3(kCpqrThreads),
                                                args, dyn, ctx->stream));
  ctx->launches++;
  int* h = (int*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {(const int32_t*)(bar + 2)};
    const lrs_status rs = replay_ints(ctx, 1, d, h + 32);
    if (rs) return rs;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 32, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[32] != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "cpqr: grid barrier wait gave up");
  return LRS_OK;
}

// ---------------------------------------------------------------------------
// Q = H_0 ... H_{r-1} [I_r; 0]: column c only sees H_c .. H_0 (reflectors
// with index > c leave e_c untouched), so each block builds one column.
// ---------------------------------------------------------------------------
// work NULL: the column lives in shared memory (p doubles); else in work +
// c p (global memory, for columns longer than shared memory holds)
__global__ void __launch_bounds__(512) k_form_q(const double* __restrict__ V, int64_t p, int64_t r,
                                                double* __restrict__ Q, int64_t ldq, double* __restrict__ work) {
  extern __shared__ double qs[];
  __shared__ double red[32];
  const int64_t c = blockIdx.x;
  double* q = work ? work + c * p : qs;
  const int64_t bs = blockDim.x;
  for (int64_t i = threadIdx.x; i < p; i += bs) q[i] = (i == c) ? 1.0 : 0.0;
  __syncthreads();
  for (int64_t jj = c; jj >= 0; --jj) {
    const double* v = V + jj * p;
    // four independent loads in flight per thread (the loop is latency-bound otherwise)
    double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
    int64_t i = jj + threadIdx.x;
    for (; i + 3 * bs < p; i += 4 * bs) {
      const double a0 = __ldg(v + i), a1 = __ldg(v + i + bs), a2 = __ldg(v + i + 2 * bs), a3 = __ldg(v + i + 3 * bs);
      w0 = fma(a0, q[i], w0); w1 = fma(a1, q[i + bs], w1);
      w2 = fma(a2, q[i + 2 * bs], w2); w3 = fma(a3, q[i + 3 * bs], w3);
    }
    for (; i < p; i += bs) w0 = fma(__ldg(v + i), q[i], w0);
    const double w = block_sum((w0 + w1) + (w2 + w3), red);
    const double tw = 2.0 * w;
    i = jj + threadIdx.x;
    for (; i + 3 * bs < p; i += 4 * bs) {
      const double a0 = __ldg(v + i), a1 = __ldg(v + i + bs), a2 = __ldg(v + i + 2 * bs), a3 = __ldg(v + i + 3 * bs);
      q[i] = fma(-tw, a0, q[i]); q[i + bs] = fma(-tw, a1, q[i + bs]);
      q[i + 2 * bs] = fma(-tw, a2, q[i + 2 * bs]); q[i + 3 * bs] = fma(-tw, a3, q[i + 3 * bs]);
    }
    for (; i < p; i += bs) q[i] = fma(-tw, __ldg(v + i), q[i]);
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < p; i += bs) Q[i * ldq + c] = q[i];
}

lrs_status launch_form_q(lrs_ctx* ctx, const double* V, int64_t p, int64_t r, double* Q, int64_t ldq) {
  if (r <= 0) return LRS_OK;
  size_t dyn = sizeof(double) * (size_t)p;
  double* work = nullptr;
  if (dyn > 200 * 1024) {
    // columns too long for shared memory: each block works in its own
    // column of global scratch (form_q_ws bytes, from the caller's reserve)
    work = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(p * r));
    if (!work) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (form_q, p=%lld)", (long long)p);
    dyn = 0;
  }
  if (dyn > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_form_q, (size_t)(dyn)); if (_s) return _s; }
  k_form_q<<<(unsigned)r, 512, dyn, ctx->stream>>>(V, p, r, Q, ldq, work);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// ---------------------------------------------------------------------------
// ID coefficients.  R is k x m (pivoted order, row stride m).  Column q >= k
// of R_2 gives C[:, q-k] = R_1^{-1} R[:, q] by back substitution; then
// P[perm[i], :] = e_i (i < k) and P[perm[q], :] = C[:, q-k]^T.  A team of T
// threads (a power of two dividing 32) solves one column: for each unknown i
// the team splits R_1[i, i+1:] . c[i+1:] by index mod T and reduces it with
// shuffles, then one lane applies 1 / R_ii (precomputed per block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_id_coeffs(const double* __restrict__ R, int64_t k, int64_t m,
                                                   const int32_t* __restrict__ perm,
                                                   int32_t* __restrict__ J, double* __restrict__ P,
                                                   int64_t ldp, int T) {
  extern __shared__ double R1[];   // k x k, then 1 / R_ii (k), then one solution vector per team
  double* dinv = R1 + k * k;
  double* cs = dinv + k;
  for (int64_t e = threadIdx.x; e < k * k; e += blockDim.x) R1[e] = R[(e / k) * m + (e % k)];
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) dinv[i] = 1.0 / R[i * m + i];
  if (blockIdx.x == 0) {
    for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
      J[i] = perm[i];
      double* prow = P + (int64_t)perm[i] * ldp;
      for (int64_t t = 0; t < k; ++t) prow[t] = (t == i) ? 1.0 : 0.0;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tm = threadIdx.x & (T - 1);
  const int team = threadIdx.x / T, nteams = blockDim.x / T;
  const unsigned tmask = (T == 32 ? 0xffffffffu : ((1u << T) - 1u)) << (lane & ~(T - 1));
  const int64_t q = (int64_t)blockIdx.x * nteams + team;
  if (q >= m - k) return;                          // whole teams leave together
  const int64_t col = k + q;
  double* c = cs + (int64_t)team * k;
  for (int64_t i = tm; i < k; i += T) c[i] = R[i * m + col];
  __syncwarp(tmask);
  for (int64_t i = k - 1; i >= 0; --i) {
    double a = 0.0;
    for (int64_t t = i + 1 + tm; t < k; t += T) a = fma(R1[i * k + t], c[t], a);
    for (int o = 1; o < T; o <<= 1) a += __shfl_xor_sync(tmask, a, o);
    if (tm == 0) c[i] = (c[i] - a) * dinv[i];
    __syncwarp(tmask);
  }
  double* prow = P + (int64_t)perm[col] * ldp;
  for (int64_t t = tm; t < k; t += T) prow[t] = c[t];
}

lrs_status launch_id_coeffs(lrs_ctx* ctx, const double* R, int64_t k, int64_t m,
                            const int32_t* perm, int32_t* J, double* P, int64_t ldp) {
  const int64_t cols = m - k;
  // team size: about 8 warps' worth of threads per SM, at most half a warp
  const int64_t want = (int64_t)ctx->num_sms * 8 * 32;
  int T = 1;
  while (T < 16 && cols * T < want) T <<= 1;
  // larger teams (fewer solution vectors) when k x k leaves little shared memory
  while (T < 32 && sizeof(double) * (size_t)(k * k + k + (256 / T) * k) > 200 * 1024) T <<= 1;
  const int nteams = 256 / T;
  const size_t dyn = sizeof(double) * (size_t)(k * k + k + nteams * k);
  if (dyn > 200 * 1024) return lrs_fail(ctx, LRS_EINVAL, "id: k=%lld too large", (long long)k);
  if (dyn > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_id_coeffs, (size_t)(dyn)); if (_s) return _s; }
  const unsigned nb = (unsigned)((cols + nteams - 1) / nteams > 0 ? (cols + nteams - 1) / nteams : 1);
  k_id_coeffs<<<nb, 256, dyn, ctx->stream>>>(R, k, m, perm, J, P, ldp, T);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
