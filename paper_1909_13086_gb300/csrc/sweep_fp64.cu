// FP64 storage and arithmetic instantiation of the fused sweep (parity path).
#include "sweep.cuh"

namespace btrirt {
BTRIRT_INSTANTIATE(double, double)
}  // namespace btrirt
