// Tensor-core fused apply (3xTF32 complex GEMM); filled in by the tcgen05 kernel.
#include "internal.h"

namespace qsim {

bool fused_tc_supported(const StateDev &, int) { return false; }

size_t tc_operand_floats(int k) { return (size_t)2 * (2 << k) * (2 << k); }

void build_tc_operands(int, const cd *, float *, float *) {}

qsim_status launch_fused_tc(const StateDev &, int, const void *, int, int, int64_t *) {
  set_error("tensor-core fused apply is not built");
  return QSIM_EUNSUPPORTED;
}

}  // namespace qsim
