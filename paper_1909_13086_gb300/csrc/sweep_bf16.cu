// BF16 population storage with FP32 arithmetic (round to nearest / stochastic).
#include "sweep.cuh"

namespace btrirt {
BTRIRT_INSTANTIATE(float, BF16<false>)
BTRIRT_INSTANTIATE(float, BF16<true>)
}  // namespace btrirt
