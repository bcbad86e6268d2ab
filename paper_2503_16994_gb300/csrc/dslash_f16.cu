// FP16-storage instantiations of the hopping kernel.
#include "dslash_inst.cuh"

namespace lqcd {
template void launch_hop<F16, F16, F16>(const HopArgs<F16, F16, F16> &, int, bool, bool, cudaStream_t);
}  // namespace lqcd
