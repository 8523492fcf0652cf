// FP32 storage and arithmetic instantiation of the fused sweep.
#include "sweep.cuh"

namespace btrirt {
template cudaError_t launch_lattice<float>(const SweepArgs<float> &, int, bool, int, dim3, dim3,
                                           cudaStream_t);
template cudaError_t launch_init<float>(const SweepArgs<float> &, double, uint64_t, dim3, dim3,
                                        cudaStream_t);
template cudaError_t launch_fields0<float>(const SweepArgs<float> &, bool, dim3, dim3,
                                           cudaStream_t);
template cudaError_t launch_repack<float>(float *, float *, double *, int, int, bool, cudaStream_t);
}  // namespace btrirt
