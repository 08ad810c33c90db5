// Step (a) on the tensor cores (BF16 operands, FP32 accumulation).
#include "tachiom_internal.cuh"

namespace tachiom {

int topc_tc_supported() { return 0; }

tachiom_status launch_topc_tc(const Index &, const __nv_bfloat16 *, int, int, int, int, float, uint64_t *,
                              int32_t *, uint32_t *, cudaStream_t) {
  return fail(TACHIOM_ERR_INVALID, "tensor-core step (a) not built");
}

}  // namespace tachiom
