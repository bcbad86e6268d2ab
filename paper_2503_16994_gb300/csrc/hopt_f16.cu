// Instantiations of the tile hopping kernel (FP16 storage).
#include <mutex>
#include <set>

#include "hopt.cuh"
#include "lqcd_impl.h"

namespace lqcd {

template <int MODE, bool DAG, bool NORM, int MINB, bool PF>
static void hopt_launch(const FastHop<F16> &f, int npw, cudaStream_t st)
{
    constexpr int smem = tile_smem_bytes();
    // more than the 48 KB a block gets without opting in: the opt-in is a
    // per-device attribute, set the first time the kernel runs on each device
    // (the autotuner's eager launches, before any stream capture)
    static std::mutex mu;
    static std::set<int> opted;
    int dev = 0;
    LQCD_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(mu);
        if (opted.insert(dev).second) {
            const cudaError_t e = cudaFuncSetAttribute(hopt_kernel<MODE, DAG, NORM, MINB, PF>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) {
                opted.erase(dev);
                LQCD_CUDA(e);
            }
        }
    }
    const int npairs = (f.nrhs + 1) / 2;
    const int nbt = (npairs + npw - 1) / npw;
    const unsigned grid = unsigned(4L * f.ntiles * nbt);
    hopt_kernel<MODE, DAG, NORM, MINB, PF><<<grid, unsigned(kTileSites * npw), smem, st>>>(f);
}

template <int MODE, bool DAG, bool NORM>
static void hopt_go(const FastHop<F16> &f, bool pf, cudaStream_t st)
{
    const int npw = std::max(1, std::min(f.gpb, kTileMaxPairs));
    if (pf) {
        if (f.minb >= 3) hopt_launch<MODE, DAG, NORM, 3, true>(f, npw, st);
        else hopt_launch<MODE, DAG, NORM, 2, true>(f, npw, st);
    } else {
        if (f.minb >= 3) hopt_launch<MODE, DAG, NORM, 3, false>(f, npw, st);
        else hopt_launch<MODE, DAG, NORM, 2, false>(f, npw, st);
    }
}

// gpb: pairs of right-hand sides (warps) per block, minb: resident blocks
// per SM the registers are capped for (2 or 3), pf: prefetch one direction
void hopt_dispatch(const FastHop<F16> &f, bool pf, int mode, bool dag, bool norm, cudaStream_t st)
{
    if (mode == HOP_CLOV) {
        if (dag) norm ? hopt_go<HOP_CLOV, true, true>(f, pf, st) : hopt_go<HOP_CLOV, true, false>(f, pf, st);
        else norm ? hopt_go<HOP_CLOV, false, true>(f, pf, st) : hopt_go<HOP_CLOV, false, false>(f, pf, st);
    } else {
        if (dag) norm ? hopt_go<SELF_CLOV, true, true>(f, pf, st) : hopt_go<SELF_CLOV, true, false>(f, pf, st);
        else norm ? hopt_go<SELF_CLOV, false, true>(f, pf, st) : hopt_go<SELF_CLOV, false, false>(f, pf, st);
    }
}

}  // namespace lqcd
