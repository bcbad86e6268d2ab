// Launcher of the paired (two right-hand sides per thread, packed FP32x2)
// hopping kernel; included by one translation unit per storage precision.
#pragma once
#include "hopfast.cuh"
#include "lqcd_impl.h"

namespace lqcd {

template <class S, int MODE, bool DAG, bool NORM>
static void hopp_go(const FastHop<S> &f, cudaStream_t st)
{
    const int ngr = (f.nrhs + 1) / 2;
    const unsigned grid = unsigned(padded_tiles(f) * ((ngr + f.gpb - 1) / f.gpb));
    if (f.minb >= 4)
        hopp_kernel<S, MODE, DAG, NORM, 4><<<grid, kBlock, 0, st>>>(f);
    else if (f.minb == 3)
        hopp_kernel<S, MODE, DAG, NORM, 3><<<grid, kBlock, 0, st>>>(f);
    else
        hopp_kernel<S, MODE, DAG, NORM, 1><<<grid, kBlock, 0, st>>>(f);
}

template <class S>
void hopp_dispatch(const FastHop<S> &f, int mode, bool dag, bool norm, cudaStream_t st)
{
    if (mode == HOP_CLOV) {
        if (dag) norm ? hopp_go<S, HOP_CLOV, true, true>(f, st) : hopp_go<S, HOP_CLOV, true, false>(f, st);
        else norm ? hopp_go<S, HOP_CLOV, false, true>(f, st) : hopp_go<S, HOP_CLOV, false, false>(f, st);
    } else {
        if (dag) norm ? hopp_go<S, SELF_CLOV, true, true>(f, st) : hopp_go<S, SELF_CLOV, true, false>(f, st);
        else norm ? hopp_go<S, SELF_CLOV, false, true>(f, st) : hopp_go<S, SELF_CLOV, false, false>(f, st);
    }
}

}  // namespace lqcd
