/*
 * lrs.h -- C ABI of the GB300 deterministic-sketch low-rank library.
 *
 * Method: Dunton & Doostan, "Deterministic matrix sketches for low-rank
 * compression of high-dimensional simulation data" (arXiv 2105.01271).
 * A_f (m x n) holds one simulation snapshot per row (Sec. 2); the library
 * sketches it onto a coarse grid without forming D (Sec. 2, Table 1), runs the
 * coarse-grid power iteration C-PWR (Sec. 5, Alg. 7), finds the range (the
 * "QR(.)" of Algs. 2/3/7), projects B = Q^T A_f and takes the SVD of B
 * (Sec. 3.1, Alg. 2), and computes the row interpolative decomposition on the
 * sketch (Sec. 4, Alg. 4).
 *
 * Conventions for every call
 *  - Matrices are ROW-MAJOR with an explicit row stride (ld*, in elements,
 *    >= the number of columns).  "Column-major X" below means the row-major
 *    storage of X^T.
 *  - Every data pointer is a DEVICE pointer on the context's device, owned by
 *    the caller; the library never frees or keeps it.  Pointers to scalar
 *    outputs (r_out, err_est, ...) are HOST pointers.
 *  - Calls are stream-ordered on the context's stream.  A call that returns a
 *    host scalar synchronises that stream before returning.
 *  - Errors are status codes; nothing is thrown across the ABI.  Arguments
 *    are validated on the host before any launch (LRS_EINVAL, with a message
 *    from lrs_last_error).  LRS_ECUDA reports a CUDA error;  LRS_ETIMEOUT a
 *    device-side wait that gave up (bounded spins, never an endless loop);
 *    LRS_ENOMEM a failed workspace allocation.  After LRS_ECUDA/LRS_ETIMEOUT
 *    the context stays usable only if the CUDA context is.
 *  - The library owns one workspace per context, grown on demand with
 *    cudaMalloc and released by lrs_destroy.
 */
#ifndef LRS_H_
#define LRS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRS_OK = 0,
  LRS_EINVAL = 1,
  LRS_ENOMEM = 2,
  LRS_ECUDA = 3,
  LRS_ERANK = 4,     /* numerical rank r < k: outputs valid at rank r */
  LRS_ETIMEOUT = 5
} lrs_status;

/* storage type of A_f */
typedef enum { LRS_F64 = 0, LRS_F32 = 1, LRS_BF16 = 2 } lrs_dtype;

/* Sec. 2 sketches.  Per axis the coarse point j sits at fine index
 * c_j = s*j + s/2 (integer division).
 *  LRS_INJECT      D = 1 at c_j                           (direct injection)
 *  LRS_FULLWEIGHT  1/4, 1/2, 1/4 at c_j-1, c_j, c_j+1;     (nearest neighbour,
 *                  a neighbour outside the grid is zero    d = 1; needs s >= 2)
 *  LRS_BLOCKAVG    1/s on s*j .. s*j+s-1                   (global sketch)
 * Multi-dimensional grids use the tensor product of the per-axis operators. */
typedef enum { LRS_INJECT = 0, LRS_FULLWEIGHT = 1, LRS_BLOCKAVG = 2 } lrs_stencil;

/* arithmetic of the dense products that read A_f or its projection
 *  LRS_PREC_FP64        FP64 FMA on CUDA cores (for FP64 data)
 *  LRS_PREC_FP32        FP32 FMA on CUDA cores (the plain FP32 method)
 *  LRS_PREC_SPLIT_BF16  tcgen05 tensor cores, BF16 hi+lo split of both
 *                       operands (3 products), FP32 accumulation
 *  LRS_PREC_BF16X3      tcgen05, 3-piece BF16 split (6 products), FP32-level */
typedef enum {
  LRS_PREC_FP64 = 0,
  LRS_PREC_FP32 = 1,
  LRS_PREC_SPLIT_BF16 = 2,
  LRS_PREC_BF16X3 = 3
} lrs_prec;

/* Cartesian fine grid: N[0] is x (fastest), then y, z.  n = prod N[d];
 * coarse grid N[d]/s[d] (N[d] % s[d] == 0), l = prod N[d]/s[d].  Dof index of
 * (x,y,z) is (z*N[1] + y)*N[0] + x; coarse index likewise. */
typedef struct {
  int32_t ndim;       /* 1, 2 or 3 */
  int32_t kind;       /* lrs_stencil */
  int64_t N[3];
  int32_t s[3];
} lrs_grid;

typedef struct lrs_ctx lrs_ctx;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
lrs_status lrs_create(lrs_ctx** out, int device, void* cuda_stream);
void lrs_destroy(lrs_ctx* ctx);
/* Message of the last failed call on ctx (never NULL; "" if none). */
const char* lrs_last_error(const lrs_ctx* ctx);
/* Build identification, e.g. "lrs sm_103a". */
const char* lrs_version(void);

/*
 * lrs_sketch -- A_c = A_f D (Sec. 2, Table 1), D never formed.
 *   A   m x n in `dtype` (n = grid->N product), row stride lda.
 *   Y   m x l FP64, row stride ldy.  Accumulated in FP64; injection is an
 *       exact copy.
 * EINVAL: m < 1, N[d] % s[d] != 0, s[d] < 1, full weighting with s[d] < 2,
 * lda < n, ldy < l, NULL pointers.
 */
lrs_status lrs_sketch(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                      const lrs_grid* grid, double* Y, int64_t ldy);

/*
 * lrs_power_pass -- C-PWR (Sec. 5, Alg. 7) from one touch of A_f.
 *   Reads the sketch points (grid `sketch`) and the Gram subsample
 *   W = A_f(:, I) (grid `gram`, injection points; |I| > k, Sec. 5 Remark),
 *   then runs q iterations  G <- W^T G; [G <- QR(G)]; G <- W G; [G <- QR(G)]
 *   with the bracketed re-orthonormalisations when reorth != 0.  QR(.) is the
 *   rank-revealing range finder of lrs_range_find with tolerance rtol.  With
 *   reorth the loop starts from QR(A_f D) (Alg. 7's Q_np), which has the same
 *   range as A_f D up to the truncated directions.
 *   Without reorth (the iterate (W W^T)^q A_f D, which the row ID takes) and
 *   prec other than LRS_PREC_FP64, the iterate is formed from the factors of
 *   the re-orthonormalised loop: each QR(.) there gives (input) = Q Rt, so
 *   (W W^T)^q Y = Q_q M Rt_np with M = Rt_g,q Rt_t,q ... Rt_g,1 Rt_t,1, in
 *   exact arithmetic up to the directions the rank truncation drops.  Since
 *   the row ID (lrs_id_k) depends only on the inner products of the rows,
 *   G then holds the m x r matrix H = Q_q M Ra^T (Ra^T Ra = Rt_np Rt_np^T,
 *   r = the rank of QR(A_f D), *g_cols = r <= 128), whose rows have the
 *   iterate's inner products: lrs_id_k(H) is the iterate's row ID, its
 *   pivoted QR taking r rows instead of l.  All of it runs in FP64 on r x r
 *   factors, so every retained direction keeps the products' accuracy
 *   relative to its own scale, where the direct product scales direction j
 *   by s_j^(2q+1) and loses all below the products' rounding of the top one.
 *   Wider iterates (and LRS_PREC_FP64) take the direct form, *g_cols = l.
 *   Y   m x l FP64 (row stride ldy): the sketch A_f D.
 *   G   m x l FP64 (row stride ldg): G_q in its first *g_cols columns (the
 *       rank after truncation when reorth != 0; without reorth l, or r for
 *       the row-Gram form below).
 *   q = 0 returns G = Y.  `gram` may be NULL when q = 0.
 *   prec: arithmetic of the W^T G and W G products (lrs_prec).
 */
lrs_status lrs_power_pass(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                          const lrs_grid* sketch, const lrs_grid* gram, int32_t q,
                          int32_t reorth, double rtol, int32_t prec,
                          double* Y, int64_t ldy, double* G, int64_t ldg, int64_t* g_cols);

/*
 * lrs_power_pass2 -- both C-PWR iterates of one matrix from one touch of A_f
 * (Sec. 5, Alg. 7): the sketch points and the Gram subsample W are read once,
 * then the q iterations run twice on them, first without the optional
 * re-orthonormalisations (G0: the iterate the row ID takes, as the paper's
 * ID experiments run C-PWR) and then with them (G: the orthonormal basis the
 * SVD takes).  Equal to lrs_power_pass(reorth = 0) -> G0 and
 * lrs_power_pass(reorth = 1) -> G on the same arguments, bit for bit, with
 * one sketch launch and one subsample gather instead of two of each.
 *   Y   m x l FP64 (row stride ldy): the sketch A_f D.
 *   G0  m x l FP64 (row stride ldg0): G_q without re-orthonormalisation in
 *       its first *g0_cols columns, in the form lrs_power_pass gives it
 *       (the row-Gram form H of r columns, or the iterate itself).
 *   G   m x l FP64 (row stride ldg): the re-orthonormalised G_q in its first
 *       *g_cols columns.  q = 0 returns G0 = G = Y (*g_cols = *g0_cols = l).
 * The re-orthonormalised loop runs once: its factors give G0.
 */
lrs_status lrs_power_pass2(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda,
                           const lrs_grid* sketch, const lrs_grid* gram, int32_t q, double rtol, int32_t prec,
                           double* Y, int64_t ldy, double* G0, int64_t ldg0, int64_t* g0_cols, double* G,
                           int64_t ldg, int64_t* g_cols);

/*
 * lrs_range_find -- orthonormal basis of the numerical range of G (the
 * "QR(A_c)" of Algs. 2/3 and "QR(G_q)" of Alg. 7), by Householder QR with
 * column pivoting in FP64, stopped before the first step whose largest
 * remaining column norm is <= rtol * |R_00|.  For rtol >= 1e-6 the same
 * pivots and stop (in exact arithmetic) come from a pivoted Cholesky of the
 * FP64 Gram G^T G (one pivot column at a time for wide G), followed by the
 * triangular solve and one Cholesky-QR2 pass; Q then differs from the
 * Householder Q by column signs and rounding only.
 *   G   m x l FP64 (row stride ldg), not modified.
 *   Q   m x r FP64 (row stride ldq >= min(m,l)); caller allocates min(m,l)
 *       columns.  *r_out = r.
 */
lrs_status lrs_range_find(lrs_ctx* ctx, const double* G, int64_t m, int64_t l, int64_t ldg,
                          double rtol, double* Q, int64_t ldq, int64_t* r_out);
/* lrs_range_find that also writes |R_ii| (i < r, non-increasing: the pivoted
 * factor's diagonal, which reveals the numerical rank) into rdiag (device,
 * min(m,l) doubles; entries from r on are left as they were).  rdiag NULL is
 * lrs_range_find. */
lrs_status lrs_range_find_diag(lrs_ctx* ctx, const double* G, int64_t m, int64_t l, int64_t ldg,
                               double rtol, double* Q, int64_t ldq, int64_t* r_out, double* rdiag);

/*
 * lrs_svd_k -- TPC-SVD from a range basis (Sec. 3.1, Alg. 2):
 *   B = Q^T A_f (r x n; the one full read of A_f; ||A_f||_F^2 fused),
 *   SVD(B) via the R factor of B^T (FP32 B: the Gram B B^T as an exact-slice
 *   product on the tensor cores, ~2^-46 relative, and an FP64 Cholesky; FP64 B: the pivoted QR of B^T) and one-sided Jacobi,
 *   U_k = Q U_B(:,1:k), S_k, V_k = B^T U_B(:,1:k) S_k^{-1}.
 *   A   m x n in dtype, row stride lda.    Q  m x r FP64, row stride ldq.
 *   U   m x k FP64 (row stride ldu).       S  k FP64.
 *   V   n x k (row stride ldv), FP64 when prec == LRS_PREC_FP64, else FP32.
 *   err_est (host, may be NULL): sqrt(sum_{i>k} s_i(B)^2 / ||A_f||_F^2), the
 *       energy of B beyond rank k.  U_k S_k V_k^T is the orthogonal projection
 *       U_k U_k^T A_f, whose squared error is this term plus the energy of A_f
 *       outside range(Q); err_est is therefore exact when range(Q) holds A_f
 *       and a lower bound otherwise.  Computed from the tail singular values
 *       (no cancellation against ||A_f||_F^2).
 * Sign convention: the largest-magnitude entry of each U column is positive.
 * Returns LRS_ERANK when r < k; then only the first r columns are written.
 */
lrs_status lrs_svd_k(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                     const double* Q, int64_t ldq, int64_t r, int32_t k, int32_t prec,
                     double* U, int64_t ldu, double* S, void* V, int64_t ldv, double* err_est);

/*
 * lrs_id_k -- rank-k row ID of a sketch (Sec. 4, Algs. 4/5): Householder
 * CPQR of Ysk^T in FP64 for k steps (pivot = largest remaining column norm,
 * norms recomputed each step, ties to the lowest position), C = R_1^{-1} R_2,
 * P = ([I | C] Z^T)^T.
 *   Ysk m x l FP64 (row stride ldy), not modified.
 *   J   k int32: skeleton snapshot (row) indices, in pivot order.
 *   P   m x k FP64 (row stride ldp) with P(J,:) = I exactly.
 *   err_est (host, may be NULL): ||R_22||_F / ||Ysk||_F, the relative error of
 *       the coarse ID.  Lift: A_f ~ P A_f(J, :) (Alg. 4).
 * Returns LRS_ERANK if the sketch has a zero column norm before step k, or
 * fewer than k columns (l < k; nothing written).
 */
lrs_status lrs_id_k(lrs_ctx* ctx, const double* Ysk, int64_t m, int64_t l, int64_t ldy, int32_t k,
                    int32_t* J, double* P, int64_t ldp, double* err_est);

/*
 * Column split of one matrix over several devices (data parallel over
 * slabs of A_f's columns).  The sketch A_f D and the subsample A_f(:, I)
 * (Sec. 2, Alg. 7) act on each coarse cell's own fine points, and Alg. 2's
 * B = Q^T A_f and B B^T are sums over column slabs, so a device that holds
 * the columns of whole coarse cells needs no other device's columns.  The
 * calls below are the per-device steps; the caller runs the two exchanges
 * between them (sums over devices, e.g. NCCL all-reduce):
 *   1. lrs_touch on the device's slab, into its columns of a zero-filled
 *      m x l sketch Y and m x |I| subsample W            -> sum Y, W (exact:
 *      the devices' columns are disjoint)
 *   2. lrs_power_pass_from(Y, W) -> G0, G (the same on every device)
 *   3. Q = G (q > 0), else lrs_range_find(G) (the same on every device)
 *   4. lrs_apass_slab: B_p = Q^T A_p for the slab's columns, ||A_p||_F^2
 *   5. lrs_slab_factor: F_p with F_p F_p^T = B_p B_p^T    -> sum the r x r
 *      Grams (LRS_FACTOR_GRAM), or place the F_p side by side in a
 *      zero-filled r x (P r) matrix and sum (LRS_FACTOR_R); sum the fro2
 *   6. lrs_svd_from_factor: U, S (the same on every device) and V_p, the
 *      slab's rows of V
 *   7. lrs_id_k(G0): J, P (the same on every device)
 * A slab is a range of the slowest axis (y in 2-D, z in 3-D) whose ends are
 * multiples of both grids' s on that axis; with full weighting that s must
 * be >= 3 (the 3-point stencil then stays inside its cell).  The slab's
 * grids are the full grids with that axis cut to the slab; its dof, coarse
 * and subsample indices are then contiguous ranges of the full ones.
 */
#define LRS_FACTOR_GRAM 0   /* F = B B^T (r x r): FP32 B, r <= 128 */
#define LRS_FACTOR_R 1      /* F = R^T (r x r), R^T R = B B^T: any B with n >= r */

/*
 * lrs_touch -- the touch of A_f alone (the first step of lrs_power_pass):
 * the sketch Y = A_f D (m x l FP64, row stride ldy) and, when gram is not
 * NULL, the subsample W = A_f(:, I) (m x |I|, row stride ldw) at the
 * injection points of `gram`.  W's type follows prec: FP32 for
 * LRS_PREC_SPLIT_BF16 and LRS_PREC_BF16X3 (exact: A_f's values), FP64
 * otherwise.  Asynchronous (no host read-back).
 * EINVAL as lrs_sketch, and gram's n differing from sketch's.
 */
lrs_status lrs_touch(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t lda, const lrs_grid* sketch,
                     const lrs_grid* gram, int32_t prec, double* Y, int64_t ldy, void* W, int64_t ldw);

/*
 * lrs_power_pass_from -- lrs_power_pass2 from a given sketch and subsample:
 * Y (m x l FP64, row stride ldy) and W (m x |I| = nI, row stride ldw, typed
 * as lrs_touch writes it for prec).  Same outputs (G0, *g0_cols; G,
 * *g_cols) and the same bits as lrs_power_pass2 on the A_f they came from.
 * W may be NULL when q = 0.  Synchronises.
 */
lrs_status lrs_power_pass_from(lrs_ctx* ctx, const double* Y, int64_t ldy, const void* W, int64_t ldw, int64_t m,
                               int64_t l, int64_t nI, int32_t q, double rtol, int32_t prec, double* G0,
                               int64_t ldg0, int64_t* g0_cols, double* G, int64_t ldg, int64_t* g_cols);

/*
 * lrs_apass_slab -- B = Q^T A (Alg. 2; the A-pass of lrs_svd_k) for the
 * columns a device holds, and ||A||_F^2 of them into fro2 (device, one
 * double).  A m x n in dtype (row stride lda); Q m x r FP64 (row stride
 * ldq); B r x n, row stride n, FP64 when prec == LRS_PREC_FP64, else FP32.
 * Asynchronous.
 */
lrs_status lrs_apass_slab(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                          const double* Q, int64_t ldq, int64_t r, int32_t prec, void* B, double* fro2);

/*
 * lrs_slab_factor -- F (r x r FP64, row stride ldf) with F F^T = B B^T for
 * B from lrs_apass_slab (r x n, row stride n, typed by prec).
 *   LRS_FACTOR_GRAM  F = B B^T by the exact-slice tensor-core Gram of
 *                    lrs_svd_k (FP32 B, r <= 128; B cut into six BF16
 *                    slices per row, slice products summed exactly); the
 *                    devices' F add up to the full Gram.
 *   LRS_FACTOR_R     F = R^T, R the R factor of B^T (pivoted QR for FP64 B,
 *                    Householder TSQR otherwise; n >= r); [F_1 ... F_P]
 *                    then has the full Gram as its Gram, without squaring
 *                    B's condition number.
 * Synchronises (the Gram's error flag; the pivoted QR's rank).
 */
lrs_status lrs_slab_factor(lrs_ctx* ctx, const void* B, int64_t r, int64_t n, int32_t prec, int32_t mode, double* F,
                           int64_t ldf);

/*
 * lrs_svd_from_factor -- the rest of lrs_svd_k from the summed factor:
 *   LRS_FACTOR_GRAM  F r x r (nf = r): pivoted FP64 Cholesky, then the FP64
 *                    one-sided Jacobi on the rows of its factor.  LRS_ERANK
 *                    with *err_est = -1 (nothing written) when the Cholesky
 *                    stops early: the caller then takes LRS_FACTOR_R.
 *   LRS_FACTOR_R     F r x nf (nf >= r, e.g. [F_1 ... F_P]): the R factor of
 *                    F^T, then the FP64 Jacobi on its columns.
 * U = Q U_B(:,1:k) (m x k, row stride ldu), S (k), and V = B^T U_B S^-1 for
 * this device's B (r x n, row stride n, typed by prec): the device's rows of
 * V (n x k, row stride ldv; FP64 when prec == LRS_PREC_FP64, else FP32).
 * fro2 (device): ||A_f||_F^2 of the WHOLE matrix, for err_est (host, may be
 * NULL) as lrs_svd_k.  Signs as lrs_svd_k.  Returns LRS_ERANK when r < k.
 * Synchronises.
 */
lrs_status lrs_svd_from_factor(lrs_ctx* ctx, const double* F, int64_t ldf, int64_t nf, int32_t mode,
                               const double* Q, int64_t ldq, int64_t m, int64_t r, int32_t k, int32_t prec,
                               const void* B, int64_t n, const double* fro2, double* U, int64_t ldu, double* S,
                               void* V, int64_t ldv, double* err_est);

/*
 * lrs_sketch_svd -- the leading r singular triplets of a sketch Y = A_c
 * (m x l FP64), the SVD step of SPC-ID (Alg. 5: U_c, S_c, V_c of A_c).
 *   The pivoted QR of lrs_range_find (tolerance rtol), stopped after at most
 *   112 steps (the FP64 Jacobi tile of lrs_svd_k), gives Q and *rank_out =
 *   min(numerical rank, 112).  When it stops at 112 with directions left, Q
 *   is refined by two steps of subspace iteration Q <- orth(Y Y^T Q); the SVD
 *   of Q^T Y (Rayleigh-Ritz) gives the triplets, whose error then shrinks as
 *   (s_113 / s_r)^4.
 *   Q   caller scratch, m x min(m,l) FP64 (row stride ldq); on return it holds
 *       the basis used.
 *   U   m x r, S r, V l x r (FP64; row strides ldu, ldv >= r); 1 <= r <= 112.
 * ERANK (nothing written) when the numerical rank is below r.
 */
lrs_status lrs_sketch_svd(lrs_ctx* ctx, const double* Y, int64_t m, int64_t l, int64_t ldy, double rtol, double* Q,
                          int64_t ldq, int32_t r, double* U, int64_t ldu, double* S, double* V, int64_t ldv,
                          int64_t* rank_out);

/*
 * lrs_spc_lift -- the lifted row skeleton of SPC-ID (Sec. 4, Alg. 5):
 *   S_f = A_c(J,:) T_r  (k x n),   T_r = A_c^+ U_r U_r^T A_f,
 * so that A_f ~ P S_f with (J, P) the rank-k row ID of the sketch A_c = Y
 * (lrs_id_k).  T_r is Alg. 5's lifting operator after its H^T = A_c^T A_f is
 * substituted.  U_r (m x r), S_r (r), V_r (l x r) are the leading r singular
 * triplets of Y (lrs_sketch_svd); k <= r <= min(m, l) and s_r > 0.  Computed as
 *   X = U_r S_r^-1 V_r^T Y(J,:)^T (m x k, FP64),  S_f = X^T A_f,
 * the second product being one read of A_f by the A-pass kernel in `prec`.
 *   A   m x n in dtype (row stride lda).   Y  m x l FP64 (row stride ldy).
 *   U   row stride ldu >= r;  V  row stride ldv >= r;  S, J device.
 *   Sf  k x n (row stride ldsf >= n): FP64 when prec == LRS_PREC_FP64, else FP32.
 * EINVAL: sizes or strides out of range, s_r <= 0 (read back: synchronises once).
 */
lrs_status lrs_spc_lift(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                        const double* Y, int64_t l, int64_t ldy, const double* U, int64_t ldu, const double* S,
                        const double* V, int64_t ldv, int64_t r, const int32_t* J, int32_t k, int32_t prec,
                        void* Sf, int64_t ldsf);

/*
 * lrs_spc_err -- SPC-ID-ERR (Sec. 4, Alg. 6): with every c-th snapshot kept,
 * B_f = A_f(J,:) and B_c = Y(J,:) for the 0-based rows J = c-1, 2c-1, ...
 * (m_c = floor(m / c) of them, 1 <= m_c <= 128),
 *   eps_hat[i] = c * lambda_max(B_f B_f^T - taus[i] B_c B_c^T),  i < ntau,
 * the estimate of eps(tau) in the SPC-ID error bound, for each tau >= 0 of the
 * caller's grid (the bound minimises over tau together with its other terms).
 * Grams in FP64 (FP32 data: the exact-slice tensor-core Gram); lambda_max by
 * Householder tridiagonalisation and Sturm-count bisection (one block per tau).
 *   A  m x n in dtype (row stride lda).   Y  m x l FP64 (row stride ldy).
 *   taus, eps_hat: HOST arrays of ntau doubles.  Synchronises.
 */
lrs_status lrs_spc_err(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                       const double* Y, int64_t l, int64_t ldy, int32_t c, const double* taus, int32_t ntau,
                       double* eps_hat);

/*
 * Single-read SPC over streamed snapshots (Sec. 3.2, Alg. 3; Sec. 4, Algs. 5
 * and 6).  The rows of A_f arrive in blocks, from host memory or from device
 * memory, and each block is read once:
 *   A_c(rows,:) = a_f D,   H^T += A_c(rows,:)^T a_f   (l x n on the device,
 *   FP32, FP64 when prec == LRS_PREC_FP64),   ||A_f||_F^2 += ||a_f||_F^2,
 * and, with err_c > 0, the rows c-1, 2c-1, ... are kept for SPC-ID-ERR.
 * Host blocks are copied on the stream's own copy stream into two staging
 * buffers, each guarded by a "copied" and a "free" event, so the copy of one
 * block overlaps the work on the previous one.
 *
 *   lrs_spc_stream_create  ctx (borrowed; must outlive the stream), storage
 *       dtype, m rows in all, sketch grid, block_rows (staging size),
 *       err_c (0: keep no rows; else 1 <= m / err_c <= 128), prec of the
 *       H^T products.  Allocates A_c (8 m l bytes), H^T (4 or 8 l n bytes),
 *       2 staging blocks and the kept rows.
 *   lrs_spc_stream_push    nrows rows of A_f (row stride ld >= n), host
 *       (on_device = 0; pinned memory overlaps best) or device (1; read in
 *       place); returns once the work is queued on ctx's stream.  The rows
 *       must total m before a finisher runs.
 *   lrs_spc_stream_svd     SPC-SVD (Alg. 3) with Q_c = the leading r left
 *       singular vectors of A_c (lrs_sketch_svd, tolerance rtol; r <= 112):
 *       B = S_r^-1 V_r^T H^T = U_r^T A_f, then as lrs_svd_k: U (m x k FP64),
 *       S (k), V (n x k; FP64 for FP64 prec, else FP32); err_est (host, may
 *       be NULL) as lrs_svd_k's.
 *   lrs_spc_stream_id      SPC-ID (Alg. 5): (J, P) = lrs_id_k of A_c, and the
 *       lifted skeleton S_f = A_c(J,:) T_r (k x n; FP64 for FP64 prec, else
 *       FP32) with T_r = V_r S_r^-2 V_r^T H^T, the operator as printed.
 *   lrs_spc_stream_err     SPC-ID-ERR (Alg. 6) on the kept rows: as
 *       lrs_spc_err with c = err_c (host taus / eps_hat).
 *   lrs_spc_stream_sketch  A_c (device, m x l FP64, row stride l).
 *   lrs_spc_stream_reset   start a new matrix of the same shape in the same
 *       buffers (waits for the stream's queued work).
 */
typedef struct lrs_spc_stream lrs_spc_stream;
lrs_status lrs_spc_stream_create(lrs_ctx* ctx, int32_t dtype, int64_t m, const lrs_grid* sketch, int64_t block_rows,
                                 int32_t err_c, int32_t prec, lrs_spc_stream** out);
lrs_status lrs_spc_stream_push(lrs_spc_stream* s, const void* rows, int64_t nrows, int64_t ld, int32_t on_device);
lrs_status lrs_spc_stream_svd(lrs_spc_stream* s, double rtol, int32_t r, int32_t k, double* U, int64_t ldu, double* S,
                              void* V, int64_t ldv, double* err_est);
lrs_status lrs_spc_stream_id(lrs_spc_stream* s, double rtol, int32_t r, int32_t k, int32_t* J, double* P, int64_t ldp,
                             void* Sf, int64_t ldsf, double* err_est);
lrs_status lrs_spc_stream_err(lrs_spc_stream* s, const double* taus, int32_t ntau, double* eps_hat);
const double* lrs_spc_stream_sketch(const lrs_spc_stream* s);
lrs_status lrs_spc_stream_reset(lrs_spc_stream* s);
void lrs_spc_stream_destroy(lrs_spc_stream* s);

/*
 * C-PWR in the same single read (Sec. 5, Alg. 7 with re-orthonormalisation).
 * lrs_spc_stream_cpwr (before the first push) makes every pushed block also
 * gather its rows of the subsample W = A_f(:, I) (grid `gram`, injection
 * points; m x |I| FP64) and accumulate Z^T += W(rows,:)^T a_f (|I| x n,
 * FP64).  Allocates 8 m |I| + 8 |I| n + 16 m l bytes.  spc_too = 0 drops
 * the H^T products from the pushes (the SPC finishers then return
 * LRS_EINVAL).
 *   lrs_spc_stream_cpwr_svd  the C-PWR basis from A_c and W alone: Q_np =
 *       QR(A_c); q times T = QR(W^T G), G = W T (G re-orthonormalised between
 *       iterations); Q_b = QR(G) by pivoted Householder QR (rtol) and one
 *       Cholesky-QR pass, written as Q_b = W M with M = T(:, piv) R_11^-1
 *       R_2^-1 (the same triangular solves that give Q_b from G); then
 *       B = M^T Z^T = Q_b^T A_f (r x n FP64) and the SVD of B as lrs_svd_k
 *       (U m x k, S, V n x k FP64, err_est).  *r_out = r (host).  1 <= q <= 16;
 *       LRS_ERANK when r < k (the first r columns written).
 *   lrs_spc_stream_cpwr_id   the row ID of the iterate without
 *       re-orthonormalisation, (W W^T)^q A_c (lrs_power_pass_from in FP64,
 *       then lrs_id_k): J, P, err_est as lrs_id_k.
 * The products run in FP64 whatever the stream's prec: B = M^T Z^T carries
 * Z^T's rounding amplified by ||M|| ||W||, up to the condition number of
 * W T (~1/rtol), and FP32-level products would leave the trailing
 * directions of B at the rounding level.  Synchronises.
 */
lrs_status lrs_spc_stream_cpwr(lrs_spc_stream* s, const lrs_grid* gram, int32_t spc_too);
lrs_status lrs_spc_stream_cpwr_svd(lrs_spc_stream* s, int32_t q, double rtol, int32_t k, double* U, int64_t ldu,
                                   double* S, double* V, int64_t ldv, double* err_est, int64_t* r_out);
lrs_status lrs_spc_stream_cpwr_id(lrs_spc_stream* s, int32_t q, double rtol, int32_t k, int32_t* J, double* P,
                                  int64_t ldp, double* err_est);

/*
 * lrs_gemm_tn -- the dense contraction every A-pass uses:
 *   C (M x N) = X^T A,   X: K x M,  A: K x N  (both row-major, K rows).
 * Exposed for tests and benchmarks of the A-pass kernel alone.
 *   x_dtype, a_dtype: lrs_dtype of X and A.  c_f64: C is FP64 (else FP32).
 *   c_trans: write C^T (N x M, row stride ldc) instead of C.
 */
lrs_status lrs_gemm_tn(lrs_ctx* ctx, int64_t M, int64_t N, int64_t K,
                       const void* X, int32_t x_dtype, int64_t ldx,
                       const void* A, int32_t a_dtype, int64_t lda,
                       void* C, int32_t c_f64, int32_t c_trans, int64_t ldc, int32_t prec);

/*
 * lrs_id_k_static -- lrs_id_k for callers that must not allocate device
 * memory while they run: a real-time loop whose time budget has no room for
 * cudaMalloc (it can synchronise the whole device and take milliseconds), or
 * a host framework that owns every device allocation and does not let a
 * library make its own.  The paper has no counterpart: it is a deployment
 * variant of the same row ID.
 *   Same arguments, results and statuses as lrs_id_k.  All scratch lives in
 *   one file-scope device array of LRS_ID_STATIC_SCRATCH_BYTES (32 MiB) that
 *   every GPU loading the library keeps until the process exits; the call
 *   makes no cudaMalloc/cudaFree and calls no allocating library routine.
 *   Scratch needed: about 8*m*l + 16*S*l + 16*k*m + 8*k*l bytes (S = SM
 *   count) when m >= 128 (the column-owner pivoted QR); for m < 128 the
 *   row-slab pivoted QR needs less unless a block's slab overflows shared
 *   memory.  A request above the array's size is rejected with LRS_EINVAL
 *   before any launch, and lrs_last_error then states the exact byte count.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture
 *   begins on that device.
 *   Every call shares the array and finds in it what the last call left:
 *   calls whose GPU work overlaps (two streams or two contexts at once) race.
 *   The call synchronises ctx's stream (it reads the rank and the error
 *   terms back), also when it fails after queueing work, so no work of a
 *   returned call is still using the array.
 */
#define LRS_ID_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
lrs_status lrs_id_k_static(lrs_ctx* ctx, const double* Ysk, int64_t m, int64_t l, int64_t ldy, int32_t k,
                           int32_t* J, double* P, int64_t ldp, double* err_est);

/* Number of kernel launches this context has issued (for launch accounting). */
int64_t lrs_launch_count(const lrs_ctx* ctx);

/* Kernel timing (measurement support; the paper has no counterpart).
 * lrs_set_kernel_timing(ctx, 1) makes every later call that runs a
 * tensor-core product kernel (the TMA A-pass -- the one full read of A_f
 * inside lrs_svd_k and lrs_gemm_tn, and the SPC lifting read -- or the
 * generic product of wide operands) bracket that kernel alone with two CUDA
 * events on ctx's stream; lrs_last_kernel_ms then returns its duration in
 * milliseconds for the most recent such call, or -1 when none was timed.
 * The events are created on the first call with on = 1 (LRS_ECUDA if that
 * fails) and released by lrs_destroy.  Timing costs one event record on
 * each side of the kernel; the calls synchronise ctx's stream anyway. */
lrs_status lrs_set_kernel_timing(lrs_ctx* ctx, int32_t on);
double lrs_last_kernel_ms(const lrs_ctx* ctx);

/* FP64 FMA throughput of ctx's device (measurement support: the roofline
 * denominator of the FP64 kernels).  One launch of 4 blocks per SM x 256
 * threads, each thread running 8 independent chains of `iters` dependent
 * FP64 FMAs, timed with CUDA events on ctx's stream; *tflops = 2 x FMAs /
 * time (best of 3 launches).  iters in [16, 1 << 20].  Synchronises. */
lrs_status lrs_fp64_peak(lrs_ctx* ctx, int32_t iters, double* tflops);

/* Failure injection for tests (the paper has no counterpart).
 * lrs_set_workspace_limit caps the device workspace later calls on ctx may
 * reserve at `bytes` (0 removes the cap): a call that needs more returns
 * LRS_ENOMEM before any launch, and ctx stays usable.
 * lrs_selftest_barrier_timeout launches, on ctx's stream, a two-block
 * cooperative kernel in which one block never arrives at the grid barrier that
 * the library's cooperative kernels use; the other block gives up after
 * spin_limit polls (1 .. the library's own limit) and the call returns
 * LRS_ETIMEOUT.  Nothing faults or hangs; ctx stays usable.  Synchronises. */
lrs_status lrs_set_workspace_limit(lrs_ctx* ctx, size_t bytes);
lrs_status lrs_selftest_barrier_timeout(lrs_ctx* ctx, int64_t spin_limit);

/* ------------------------------------------------------------------------
 * Batching form: many independent decompositions of different sizes.
 *
 * The paper treats one snapshot matrix at a time; this runs a list of them
 * (each its own A_f, grid, k, q, precision) through the same path as
 * lrs_power_pass + lrs_range_find + lrs_svd_k (SVD, Algs. 7 and 2) and
 * lrs_power_pass + lrs_id_k (row ID, Alg. 4), with re-orthonormalisation on
 * for the SVD and off for the ID, exactly as the single-matrix calls.
 *
 * Item (all pointers device pointers on `device`, caller-owned; U/S/V may be
 * NULL when do_svd = 0, J/P when do_id = 0):
 *   A, dtype, m, lda      the m x n matrix, n = sketch.N product
 *   sketch, gram          the sketch grid; the C-PWR subsample grid (q > 0)
 *   q, k, prec, rtol      as in lrs_power_pass / lrs_svd_k
 *   U (m x k, ldu), S (k), V (n x k, ldv; FP64 for LRS_PREC_FP64 else FP32)
 *   J (k), P (m x k, ldp)
 * Written by the call: r (SVD basis rank), err_svd, err_id, status (an
 * lrs_status; LRS_ERANK means fewer than k directions, outputs at rank r),
 * launches (kernels launched for this item).
 *
 * lrs_batch_run: n_streams worker threads, each with its own context and
 * CUDA stream, take items largest-first from a shared queue, so the
 * latency-bound steps of different matrices overlap on the GPU.  Results are
 * bit-identical to running the items one by one.  Returns LRS_OK when every
 * item ended LRS_OK or LRS_ERANK, else the first other status (the items'
 * own statuses tell which).  Blocks until all items are done.
 *
 * lrs_batch_autotune: times lrs_batch_run on a sample of the items (every
 * 4th when there are 32 or more) for each candidate stream count and returns the fastest
 * in *best (its time per sampled item in *ms_per_item).
 *
 * The worker contexts, streams and buffers are kept per device across calls
 * (the first runs size them; later runs allocate nothing); calls for one
 * device are serialised.  lrs_batch_release frees them.
 * ---------------------------------------------------------------------- */
typedef struct lrs_batch_item {
  const void* A;
  int32_t dtype;
  int64_t m, lda;
  lrs_grid sketch;
  lrs_grid gram;
  int32_t q, k, prec;
  double rtol;
  int32_t do_svd, do_id;
  double* U;
  int64_t ldu;
  double* S;
  void* V;
  int64_t ldv;
  int32_t* J;
  double* P;
  int64_t ldp;
  int64_t r;
  double err_svd, err_id;
  int32_t status;
  int64_t launches;   /* kernels this item launched */
  char error[120];    /* lrs_last_error text when status is not OK/ERANK */
} lrs_batch_item;

lrs_status lrs_batch_run(int device, lrs_batch_item* items, int64_t n_items, int32_t n_streams);
lrs_status lrs_batch_autotune(int device, lrs_batch_item* items, int64_t n_items, const int32_t* candidates,
                              int32_t n_candidates, int32_t* best, double* ms_per_item);
lrs_status lrs_batch_release(int device);

/*
 * The batch as one CUDA graph (batching form; the paper has one matrix at a
 * time).  The calls above read a few values back to the host as they run
 * (ranks that size the next launches, breakdown checks, the bounded waits'
 * error flags), and a stream capture cannot contain a read-back.
 *   lrs_batch_graph_create  runs the items once as lrs_batch_run does (their
 *       outputs, r, err and status are written: the batch's results), on
 *       `branches` contexts and streams (largest first onto the least loaded),
 *       each context recording every value it reads back, in call order.
 *       Then it captures the same call sequence from all branches into one
 *       CUDA graph: each read-back becomes the recorded value plus a
 *       one-thread guard kernel that compares the device's value with it
 *       when the graph runs, and the error estimates are computed on the
 *       device.  Items must have q = 0 (LRS_EINVAL otherwise).  An item whose
 *       recorded run failed stays out of the graph and runs eagerly at every
 *       launch.
 *   lrs_batch_graph_launch  one launch of the graph (the whole batch), then
 *       the items' r, err and status; an item whose guard saw another value
 *       (its data, changed in place since the capture, now takes another
 *       rank or route) is run again eagerly with the single-matrix path, so
 *       the outputs are always lrs_batch_run's.  *reruns (may be NULL) counts
 *       those items.  `items` must describe the captured batch (the same
 *       pointers, sizes and parameters; LRS_EINVAL otherwise): new data goes
 *       into the same buffers.  Blocks until the batch is done.
 *   lrs_batch_graph_destroy frees the graph, its contexts and buffers.
 * Each branch keeps its own workspace, sized by the recorded run.
 */
typedef struct lrs_batch_graph lrs_batch_graph;
lrs_status lrs_batch_graph_create(int device, lrs_batch_item* items, int64_t n_items, int32_t branches,
                                  lrs_batch_graph** out);
lrs_status lrs_batch_graph_launch(lrs_batch_graph* g, lrs_batch_item* items, int64_t n_items, int64_t* reruns);
void lrs_batch_graph_destroy(lrs_batch_graph* g);

/* ------------------------------------------------------------------------
 * Range error: how much of A_f a basis Q captures.
 *   *err = ||A_f - Q Q^T A_f||_F / ||A_f||_F = sqrt(1 - ||Q^T A_f||_F^2 / ||A_f||_F^2)
 * for Q (m x r, row-major ldq) with orthonormal columns.  The products run in
 * FP64 (the difference of two squared norms must resolve tolerances near
 * 1e-3, i.e. 1e-6 in the squares).  err is a host pointer.  Synchronises.
 * ---------------------------------------------------------------------- */
lrs_status lrs_range_error(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                           const double* Q, int64_t ldq, int64_t r, double* err);

/* ------------------------------------------------------------------------
 * Learned sketch proposal (an addition to the paper's method): a 3-layer MLP
 * that maps the leading LRS_MLP_NSIGMA diagonal entries of the pivoted R of
 * the cheapest configuration's sketch (the first thing the adaptive
 * enlargement computes) plus the sizes to one of LRS_MLP_OUT sketch
 * configurations (coarsening factor, C-PWR passes).
 * Width LRS_MLP_HID, ReLU, softmax cross-entropy; BF16 weights, FP32
 * accumulation; trained by Adam in these kernels.
 *
 * Parameters: one FP32 buffer of lrs_mlp_param_count() values, laid out
 *   W1 [HID x IN] | b1 [HID] | W2 [HID x HID] | b2 [HID] | W3 [OUT x HID] | b3 [OUT]
 * (row-major), the master copy; wbf16 (uint16, same layout) holds the BF16
 * rounding (RNE) of the weight slots, which the products read.  All device
 * pointers.
 *   lrs_mlp_init_bf16  wbf16 <- round(params) on the weight slots
 *   lrs_mlp_features   x (IN floats) of one matrix from d = |R_ii| (device,
 *                      non-increasing, ns of them) written by
 *                      lrs_range_find_diag for the cheapest configuration's
 *                      sketch Y (m x l) at rtol 1e-6, rank r, grid N:
 *                      clip(log10(d_i / d_0), -6, 0) / 6 (missing -1),
 *                      log2(N) / 8, log2(m) / 11, r / min(m, l)
 *   lrs_mlp_forward    logits (B x OUT) for X (B x IN)
 *   lrs_mlp_loss_grad  mean cross-entropy over labels y (B, int32) into *loss
 *                      (device) and its gradient w.r.t. the BF16 weights and
 *                      the biases into grad (param layout)
 *   lrs_mlp_adam       one Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected
 *                      by `step` >= 1) on params, refreshing wbf16
 * ---------------------------------------------------------------------- */
#define LRS_MLP_NSIGMA 64
#define LRS_MLP_IN 67
#define LRS_MLP_HID 128
#define LRS_MLP_OUT 6
int64_t lrs_mlp_param_count(void);
lrs_status lrs_mlp_init_bf16(lrs_ctx* ctx, const float* params, uint16_t* wbf16);
lrs_status lrs_mlp_features(lrs_ctx* ctx, const double* rdiag, int64_t ns, int64_t r, int64_t l, int64_t N, int64_t m,
                            float* x);
lrs_status lrs_mlp_forward(lrs_ctx* ctx, const float* params, const uint16_t* wbf16, const float* X, int64_t B,
                           float* logits);
lrs_status lrs_mlp_loss_grad(lrs_ctx* ctx, const float* params, const uint16_t* wbf16, const float* X,
                             const int32_t* y, int64_t B, float* grad, float* loss);
lrs_status lrs_mlp_adam(lrs_ctx* ctx, float* params, uint16_t* wbf16, const float* grad, float* m1, float* m2,
                        int64_t step, float lr);


#ifdef __cplusplus
}
#endif
#endif /* LRS_H_ */
