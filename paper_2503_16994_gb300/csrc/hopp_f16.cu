// 16-bit-storage instantiations of the paired hopping kernel.
#include "hopp_inst.cuh"

namespace lqcd {
template void hopp_dispatch<F16>(const FastHop<F16> &, int, bool, bool, cudaStream_t);
}  // namespace lqcd
