// Launcher for the hopping kernel; included once per storage precision so
// the instantiations compile in parallel translation units.
#pragma once
#include "lqcd_impl.h"

namespace lqcd {

template <class S, class L, class C, int MODE, bool DAG, bool NORM>
static void hop_go(const HopArgs<S, L, C> &a, cudaStream_t st)
{
    using R = typename std::conditional<std::is_same<S, F64>::value, double, float>::type;
    hop_kernel<S, L, C, R, MODE, DAG, NORM><<<unsigned(a.ntiles * a.nrhs), kBlock, 0, st>>>(a);
}

template <class S, class L, class C, int MODE>
static bool hop_mode(const HopArgs<S, L, C> &a, int mode, bool dag, bool norm, cudaStream_t st)
{
    if (mode != MODE) return false;
    if (dag) {
        if (norm) hop_go<S, L, C, MODE, true, true>(a, st);
        else hop_go<S, L, C, MODE, true, false>(a, st);
    } else {
        if (norm) hop_go<S, L, C, MODE, false, true>(a, st);
        else hop_go<S, L, C, MODE, false, false>(a, st);
    }
    return true;
}

static const char *const kHopNames[3][5] = {
    {"hop_f64_hopclov", "hop_f64_selfclov", "hop_f64_self", "hop_f64_clovsum", "hop_f64_resid"},
    {"hop_f32_hopclov", "hop_f32_selfclov", "hop_f32_self", "hop_f32_clovsum", "hop_f32_resid"},
    {"hop_f16_hopclov", "hop_f16_selfclov", "hop_f16_self", "hop_f16_clovsum", "hop_f16_resid"}};

template <class S, class L, class C>
void launch_hop(const HopArgs<S, L, C> &a, int mode, bool dag, bool norm, cudaStream_t st)
{
    // algorithmic bytes: input spinor (read once), output, self / b where used,
    // 8 links per output site, the clover blocks where used
    const double sb = spinor_bytes<S>();
    double per_rhs = sb + (mode == RESID ? 0.0 : sb) + (mode == HOP_CLOV ? 0.0 : sb) + (mode == RESID ? sb : 0.0);
    double shared = 8.0 * link_bytes<L>() + (mode == SELF_PLAIN ? 0.0 : clover_bytes<C>());
    const int pi = S::W == 2 ? 0 : (S::W == 4 ? 1 : 2);
    ProfScope prof(kHopNames[pi][mode], double(a.g.vh) * (a.nrhs * per_rhs + shared), st);
    bool ok = hop_mode<S, L, C, HOP_CLOV>(a, mode, dag, norm, st) || hop_mode<S, L, C, SELF_CLOV>(a, mode, dag, norm, st);
    if constexpr (std::is_same<S, F64>::value) {
        ok = ok || hop_mode<S, L, C, SELF_PLAIN>(a, mode, dag, norm, st) ||
             hop_mode<S, L, C, CLOV_SUM>(a, mode, dag, norm, st);
        if (!ok && mode == RESID) {
            if (dag) hop_go<S, L, C, RESID, true, true>(a, st);
            else hop_go<S, L, C, RESID, false, true>(a, st);
            ok = true;
        }
    }
    if (!ok) throw Error{LQCD_EINVAL, "hopping kernel: mode not built for this precision"};
    LQCD_CHECK_LAUNCH();
}

}  // namespace lqcd
