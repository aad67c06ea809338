// Reduced-precision sigma build (TF32 / split BF16 alpha-beta GEMM on the
// tensor cores, FP32 same-spin terms).
#include "forte_internal.h"

namespace forte {

int sigma_mixed(forte_ctx *ctx, const double *C, double *S, int nvec, int mode) {
  (void)ctx; (void)C; (void)S; (void)nvec;
  set_error("precision mode %d is not available in this build", mode);
  return FORTE_ERR_ARG;
}

}  // namespace forte
