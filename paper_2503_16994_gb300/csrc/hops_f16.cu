// Instantiations of the staged paired hopping kernel (FP16 storage).
#include <mutex>
#include <set>

#include "hops.cuh"
#include "lqcd_impl.h"

namespace lqcd {

template <int MODE, bool DAG, bool NORM, int MINB, int PD>
static void hops_launch(const FastHop<F16> &f, unsigned grid, cudaStream_t st)
{
    constexpr int smem = stage_bytes(PD);
    // the stage plus the kernel's static shared memory (reductions) exceeds
    // the 48 KB a block gets without opting in; the opt-in is a per-device
    // attribute, set the first time the kernel runs on each device (the
    // autotuner's eager launches, before any stream capture)
    static std::mutex mu;
    static std::set<int> opted;
    int dev = 0;
    LQCD_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(mu);
        if (opted.insert(dev).second) {
            const cudaError_t e = cudaFuncSetAttribute(hops_kernel<MODE, DAG, NORM, MINB, PD>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) {
                opted.erase(dev);
                LQCD_CUDA(e);
            }
        }
    }
    hops_kernel<MODE, DAG, NORM, MINB, PD><<<grid, kBlock, smem, st>>>(f);
}

template <int MODE, bool DAG, bool NORM>
static void hops_go(const FastHop<F16> &f, int pd, cudaStream_t st)
{
    const int ngr = (f.nrhs + 1) / 2;
    const unsigned grid = unsigned(padded_tiles(f) * ((ngr + f.gpb - 1) / f.gpb));
    if (pd >= 3) hops_launch<MODE, DAG, NORM, 3, 3>(f, grid, st);  // 64 KB: 3 blocks per SM
    else if (f.minb >= 4) hops_launch<MODE, DAG, NORM, 4, 2>(f, grid, st);
    else hops_launch<MODE, DAG, NORM, 3, 2>(f, grid, st);
}

void hops_dispatch(const FastHop<F16> &f, int pd, int mode, bool dag, bool norm, cudaStream_t st)
{
    if (mode == HOP_CLOV) {
        if (dag) norm ? hops_go<HOP_CLOV, true, true>(f, pd, st) : hops_go<HOP_CLOV, true, false>(f, pd, st);
        else norm ? hops_go<HOP_CLOV, false, true>(f, pd, st) : hops_go<HOP_CLOV, false, false>(f, pd, st);
    } else {
        if (dag) norm ? hops_go<SELF_CLOV, true, true>(f, pd, st) : hops_go<SELF_CLOV, true, false>(f, pd, st);
        else norm ? hops_go<SELF_CLOV, false, true>(f, pd, st) : hops_go<SELF_CLOV, false, false>(f, pd, st);
    }
}

}  // namespace lqcd
