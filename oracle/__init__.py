"""FP64 CPU oracle for the deterministic-sketch low-rank path (Dunton & Doostan,
"Deterministic matrix sketches for low-rank compression of high-dimensional
simulation data", arXiv 2105.01271).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path; the two meet only in the seeded generators of ``synth``.

Every routine is a plain, slow restatement of the paper in float64 with
numpy/scipy (LAPACK) as the only library steps:

  sketch.py       Sec. 2 (injection, nearest-neighbour and global sketch
                  definitions, Table 1): the sketch matrix D formed
                  explicitly (scipy.sparse), A_c = A_f D; the C-PWR column
                  subsample A_f(:, I).
  cpqr.py         Sec. 4: Householder QR with column pivoting (own code).
  rangefinder.py  Algs. 2/3/7 "QR(.)": rank-revealing orthonormal basis.
  cpwr.py         Sec. 5, Alg. 7: coarse-grid power iteration; its single-read
                  form (the final basis as W M, B = M^T (W^T A_f)).
  svd.py          Sec. 3.1, Alg. 2: TPC-SVD projection B = Q^T A_f and SVD(B).
  interp.py       Sec. 4, Alg. 4: TPC-ID (row ID of the sketch by CPQR of A_c^T).
  spc.py          Sec. 4, Algs. 5/6: SPC-ID lifting operator T_r, the
                  single-pass error estimate eps_hat(tau) and the SPC-ID
                  error bound.
  learned.py      the learned sketch proposal (not in the paper): features,
                  labels, the MLP and Adam in float64.
  metrics.py      Sec. 6: relative Frobenius error, Eckart-Young, MREO.

Pins (tests/test_oracle_*.py) tie each routine to something other than itself:
Eckart-Young for Omega = I, exact recovery of exact-rank inputs, the DST-I
closed form of the heat field, sigma^(2q+1) of standard power iteration,
LAPACK dgeqp3 pivots, P(J,:) = I, Theorems 3.1/3.2 and the ID existence bound,
and brute force on tiny grids.
"""
from .sketch import restriction_1d, sketch_operator, sketch, subsample_index, subsample  # noqa
from .cpqr import cpqr  # noqa
from .rangefinder import range_find  # noqa
from .cpwr import cpwr  # noqa
from .svd import tpc_svd, svd_of_projection, sign_fix  # noqa
from .interp import row_id, tpc_id  # noqa
from .metrics import rel_fro_error, id_rel_error, eckart_young, mreo, singular_values  # noqa
from .pipeline import svd_path, id_path  # noqa
