// 32-bit-storage instantiations of the paired hopping kernel.
#include "hopp_inst.cuh"

namespace lqcd {
template void hopp_dispatch<F32>(const FastHop<F32> &, int, bool, bool, cudaStream_t);
}  // namespace lqcd
