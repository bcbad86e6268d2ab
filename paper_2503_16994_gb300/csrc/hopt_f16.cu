// Instantiations of the tile hopping kernel (FP16 storage).
#include <mutex>
#include <set>

#include "hopt.cuh"
#include "lqcd_impl.h"

namespace lqcd {

template <int MODE, bool DAG, bool NORM, int MINB, int PD>
static void hopt_launch(const FastHop<F16> &f, int npw, cudaStream_t st)
{
    constexpr int smem_max = tile_smem_bytes(kTileSites * kTileMaxPairs, PD);
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
            const cudaError_t e = cudaFuncSetAttribute(hopt_kernel<MODE, DAG, NORM, MINB, PD>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
            if (e != cudaSuccess) {
                opted.erase(dev);
                LQCD_CUDA(e);
            }
        }
    }
    const int npairs = (f.nrhs + 1) / 2;
    const int nbt = (npairs + npw - 1) / npw;
    const unsigned grid = unsigned(4L * f.ntiles * nbt);
    hopt_kernel<MODE, DAG, NORM, MINB, PD>
        <<<grid, unsigned(kTileSites * npw), tile_smem_bytes(kTileSites * npw, PD), st>>>(f);
}

template <int MODE, bool DAG, bool NORM>
static void hopt_go(const FastHop<F16> &f, bool pf, cudaStream_t st)
{
    const int npw = std::max(1, std::min(f.gpb, kTileMaxPairs));
    if (pf) hopt_launch<MODE, DAG, NORM, 2, 2>(f, npw, st);
    else hopt_launch<MODE, DAG, NORM, 2, 1>(f, npw, st);
}

// gpb: pairs of right-hand sides (warps) per block; pf: spinor words staged
// two directions ahead instead of one (registers capped for 2 blocks per SM)
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
