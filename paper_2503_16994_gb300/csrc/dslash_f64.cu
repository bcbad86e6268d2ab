// FP64-storage instantiations of the hopping kernel.
#include "dslash_inst.cuh"

namespace lqcd {
template void launch_hop<F64, F64, F64>(const HopArgs<F64, F64, F64> &, int, bool, bool, cudaStream_t);
}  // namespace lqcd
