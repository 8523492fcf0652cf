// 16-bit population storage (FP16 and BF16) with FP32 arithmetic.
#include "sweep.cuh"

namespace btrirt {
BTRIRT_INSTANTIATE(float, __half)
BTRIRT_INSTANTIATE(float, __nv_bfloat16)
}  // namespace btrirt
