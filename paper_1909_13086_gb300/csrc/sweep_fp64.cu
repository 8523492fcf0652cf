// FP64 storage and arithmetic instantiation of the fused sweep (parity path).
#include "sweep.cuh"

namespace btrirt {
template cudaError_t launch_lattice<double>(const SweepArgs<double> &, int, bool, int, dim3,
                                            dim3, cudaStream_t);
template cudaError_t launch_init<double>(const SweepArgs<double> &, double, uint64_t, dim3,
                                         dim3, cudaStream_t);
template cudaError_t launch_fields0<double>(const SweepArgs<double> &, bool, dim3, dim3,
                                            cudaStream_t);
template cudaError_t launch_repack<double>(double *, double *, double *, int, int, bool, cudaStream_t);
}  // namespace btrirt
