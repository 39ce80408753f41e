// Tensor-core GEMM on tcgen05 (placeholder until the kernel lands).
#include "common.h"

namespace ccpnk {

void gemm_tc(const Exec& ex, cc_precision prec, const GemmArgs& g) {
  (void)ex; (void)prec; (void)g;
  fail(CC_ERR_INVALID, "tensor-core contractions are not available in this build");
}

}  // namespace ccpnk
