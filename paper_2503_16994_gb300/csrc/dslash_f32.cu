// FP32-storage instantiations of the hopping kernel.
#include "dslash_inst.cuh"

namespace lqcd {
template void launch_hop<F32, F32, F32>(const HopArgs<F32, F32, F32> &, int, bool, bool, cudaStream_t);
}  // namespace lqcd
