// Tensor-core (tcgen05) forms of C = X^T A.
#include "common.cuh"
#include "internal.h"

namespace lrs {

lrs_status launch_gemm_tc(lrs_ctx* ctx, const GemmArgs& a, int prec) {
  (void)a;
  return lrs_fail(ctx, LRS_EINVAL, "gemm: precision mode %d is not available in this build", prec);
}

}  // namespace lrs
