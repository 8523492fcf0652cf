// FP32 storage and arithmetic instantiation of the fused sweep.
#include "sweep.cuh"

namespace btrirt {
BTRIRT_INSTANTIATE(float, float)
}  // namespace btrirt
