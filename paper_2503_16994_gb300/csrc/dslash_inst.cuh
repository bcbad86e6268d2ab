// Launcher for the hopping kernel; included once per storage precision so
// the instantiations compile in parallel translation units.
#pragma once
#include <cstdlib>

#include "hopfast.cuh"
#include "hopt.cuh"
#include "lqcd_impl.h"

namespace lqcd {

template <class S, int NR, int MODE, bool DAG, bool NORM>
static void hopf_go(const FastHop<S> &f, cudaStream_t st)
{
    const int ngr = (f.nrhs + NR - 1) / NR;
    const unsigned grid = unsigned(padded_tiles(f) * ((ngr + f.gpb - 1) / f.gpb));
    // minimum resident blocks per SM (register cap) as chosen by the autotuner
    if (NR == 1 && f.minb >= 6)
        hopf_kernel<S, NR, MODE, DAG, NORM, 6><<<grid, kBlock, 0, st>>>(f);
    else
        hopf_kernel<S, NR, MODE, DAG, NORM, 1><<<grid, kBlock, 0, st>>>(f);
}

template <class S, int NR>
static void hopf_dispatch(const FastHop<S> &f, int mode, bool dag, bool norm, cudaStream_t st)
{
    if constexpr (std::is_same<S, F64>::value) {
        // the FP64 set-up and final modes of the solver (no dagger)
        if (mode == SELF_PLAIN) {
            norm ? hopf_go<S, NR, SELF_PLAIN, false, true>(f, st) : hopf_go<S, NR, SELF_PLAIN, false, false>(f, st);
            return;
        }
        if (mode == CLOV_SUM) {
            norm ? hopf_go<S, NR, CLOV_SUM, false, true>(f, st) : hopf_go<S, NR, CLOV_SUM, false, false>(f, st);
            return;
        }
        if (mode == RESID) {
            norm ? hopf_go<S, NR, RESID, false, true>(f, st) : hopf_go<S, NR, RESID, false, false>(f, st);
            return;
        }
    }
    if (mode == HOP_CLOV) {
        if (dag) norm ? hopf_go<S, NR, HOP_CLOV, true, true>(f, st) : hopf_go<S, NR, HOP_CLOV, true, false>(f, st);
        else norm ? hopf_go<S, NR, HOP_CLOV, false, true>(f, st) : hopf_go<S, NR, HOP_CLOV, false, false>(f, st);
    } else {
        if (dag) norm ? hopf_go<S, NR, SELF_CLOV, true, true>(f, st) : hopf_go<S, NR, SELF_CLOV, true, false>(f, st);
        else norm ? hopf_go<S, NR, SELF_CLOV, false, true>(f, st) : hopf_go<S, NR, SELF_CLOV, false, false>(f, st);
    }
}

// paired kernels: instantiated in hopp_f16.cu / hopp_f32.cu (own translation
// units, so they compile in parallel with the rest)
template <class S>
void hopp_dispatch(const FastHop<S> &f, int mode, bool dag, bool norm, cudaStream_t st);
// staged paired kernel (hops_f16.cu): pd directions of cp.async copies ahead
void hops_dispatch(const FastHop<F16> &f, int pd, int mode, bool dag, bool norm, cudaStream_t st);
// tile kernel (hopt_f16.cu): links, clover and neighbours prepared once per
// 32-site tile in shared memory; pf: one direction of loads ahead
void hopt_dispatch(const FastHop<F16> &f, bool pf, int mode, bool dag, bool norm, cudaStream_t st);

template <class S, int MODE, bool DAG, bool NORM>
static void hopq_go(const FastHop<S> &f, int pf, cudaStream_t st)
{
    const unsigned grid = unsigned(padded_tiles(f) * ((f.nrhs + f.gpb - 1) / f.gpb));
    if (pf == 8) hopq_kernel<S, MODE, DAG, NORM, 8><<<grid, kBlock, 0, st>>>(f);
    else if (pf == 4) hopq_kernel<S, MODE, DAG, NORM, 4><<<grid, kBlock, 0, st>>>(f);
    else hopq_kernel<S, MODE, DAG, NORM, 2><<<grid, kBlock, 0, st>>>(f);
}

template <class S>
static void hopq_dispatch(const FastHop<S> &f, int pf, int mode, bool dag, bool norm, cudaStream_t st)
{
    if (mode == HOP_CLOV) {
        if (dag) norm ? hopq_go<S, HOP_CLOV, true, true>(f, pf, st) : hopq_go<S, HOP_CLOV, true, false>(f, pf, st);
        else norm ? hopq_go<S, HOP_CLOV, false, true>(f, pf, st) : hopq_go<S, HOP_CLOV, false, false>(f, pf, st);
    } else {
        if (dag) norm ? hopq_go<S, SELF_CLOV, true, true>(f, pf, st) : hopq_go<S, SELF_CLOV, true, false>(f, pf, st);
        else norm ? hopq_go<S, SELF_CLOV, false, true>(f, pf, st) : hopq_go<S, SELF_CLOV, false, false>(f, pf, st);
    }
}

// nr in 1..3: NR right-hand sides per thread in scalar FP32/FP64 arithmetic;
// nr == 0: two right-hand sides per thread in the lanes of packed FP32x2;
// nr == -2, -4, -8: one right-hand side per thread, loads of 2, 4 or 8
// directions issued before their arithmetic (FP16/FP32 only);
// nr == 12, 13: as nr == 0 with the words of 2 or 3 directions ahead staged
// in shared memory by cp.async (FP16 only);
// nr == 20, 21: the tile kernel, gpb = pairs (warps) per block, spinor words
// staged one (20) or two (21) directions ahead (FP16 only)
constexpr bool is_tile_shape(int nr) { return nr == 20 || nr == 21; }

template <class S>
static void hopf_launch(const FastHop<S> &f, int nr, int mode, bool dag, bool norm, cudaStream_t st)
{
    if constexpr (std::is_same<S, F16>::value) {
        if (is_tile_shape(nr)) {
            hopt_dispatch(f, nr == 21, mode, dag, norm, st);
            return;
        }
        if (nr >= 12) {
            hops_dispatch(f, nr - 10, mode, dag, norm, st);
            return;
        }
    }
    if constexpr (!std::is_same<S, F64>::value) {
        if (nr == 0) {
            hopp_dispatch<S>(f, mode, dag, norm, st);
            return;
        }
        if (nr < 0) {
            hopq_dispatch<S>(f, -nr, mode, dag, norm, st);
            return;
        }
    }
    if constexpr (std::is_same<S, F64>::value) {
        hopf_dispatch<S, 1>(f, mode, dag, norm, st);
    } else {
        switch (nr) {
        case 1: hopf_dispatch<S, 1>(f, mode, dag, norm, st); break;
        case 2: hopf_dispatch<S, 2>(f, mode, dag, norm, st); break;
        default: hopf_dispatch<S, 3>(f, mode, dag, norm, st); break;
        }
    }
}

// Autotuned shape: right-hand sides per thread (NR) and groups of NR per
// block (GPB), keyed by (sites, nrhs, format, mode).  The first launch of a
// key times the candidates (no reductions, same stream and buffers: every
// candidate writes the output the real launch then overwrites) and keeps
// the fastest.  LQCD_HOP_NR / LQCD_HOP_GPB force a value.
struct HopShape {
    int nr, gpb, minb, swz;
};

template <class S>
static HopShape hopf_tuned(FastHop<S> f, int mode, cudaStream_t st)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, HopShape> table;
    const char *env_nr = std::getenv("LQCD_HOP_NR");
    const char *env_gpb = std::getenv("LQCD_HOP_GPB");
    if (env_nr || env_gpb) {
        int nr = env_nr ? std::atoi(env_nr) : 1, gpb = env_gpb ? std::atoi(env_gpb) : 1;
        const bool staged = std::is_same<S, F16>::value && (nr == 12 || nr == 13 || is_tile_shape(nr));
        if (std::is_same<S, F64>::value || (!staged && nr != -2 && nr != -4 && nr != -8 && (nr < 0 || nr > 3)))
            nr = 1;
        if (is_tile_shape(nr) && !env_gpb) gpb = std::min(kTileMaxPairs, (f.nrhs + 1) / 2);
        const char *env_mb = std::getenv("LQCD_HOP_MINB");
        const char *env_sw = std::getenv("LQCD_HOP_SWZ");
        return HopShape{nr, std::max(gpb, 1), env_mb ? std::atoi(env_mb) : 1, env_sw ? std::max(1, std::atoi(env_sw)) : 1};
    }
    auto key = std::make_tuple(f.vh, f.nrhs, S::W, mode);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = table.find(key);
        if (it != table.end()) return it->second;
    }
    {
        // a shape imported from an earlier process (lqcd_tune_import) is used as is
        int sh[4];
        if (tune_imported(prec_name<S>(), mode, f.vh, f.nrhs, sh)) {
            const HopShape h{sh[0], sh[1], sh[2], sh[3]};
            std::lock_guard<std::mutex> lk(mu);
            if (table.emplace(key, h).second)
                tune_record(prec_name<S>(), mode, f.vh, f.nrhs, h.nr, h.gpb, h.minb, h.swz, -1.f);
            return table[key];
        }
    }
    // one tuning at a time in the process (server slots may ask concurrently);
    // whoever waited finds the result in the table
    static std::mutex tuning;
    std::lock_guard<std::mutex> tl(tuning);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = table.find(key);
        if (it != table.end()) return it->second;
    }
    std::vector<HopShape> cand;
    const int maxnr = std::is_same<S, F64>::value ? 1 : 3;
    for (int nr = (std::is_same<S, F64>::value || f.nrhs < 2) ? 1 : 0; nr <= maxnr && nr <= f.nrhs; ++nr) {
        const int per = nr == 0 ? 2 : nr;
        const int ngr = (f.nrhs + per - 1) / per;
        for (int gpb : {1, 2, 3, 4, 6, 12})
            if (gpb <= ngr && (gpb == 1 || ngr % gpb == 0)) {
                // FP64 is bound by the FP64 units: only the grouping is worth timing
                if (std::is_same<S, F64>::value) {
                    if (gpb <= 2) cand.push_back(HopShape{nr, gpb, 1, 1});
                    continue;
                }
                for (int swz : {1, 8, 32}) {
                    if (swz > 1 && ngr / gpb < 2) continue;  // one block per tile: order is irrelevant
                    cand.push_back(HopShape{nr, gpb, 1, swz});
                }
                if (!std::is_same<S, F64>::value && nr == 1) cand.push_back(HopShape{nr, gpb, 6, 1});
                if (nr == 0) {
                    cand.push_back(HopShape{nr, gpb, 3, 1});
                    cand.push_back(HopShape{nr, gpb, 4, 1});
                }
            }
    }
    if (std::is_same<S, F16>::value && f.nrhs >= 2) {
        const int ngr = (f.nrhs + 1) / 2;
        for (int gpb : {1, 2, 3, 6})
            if (gpb <= ngr && (gpb == 1 || ngr % gpb == 0)) {
                cand.push_back(HopShape{12, gpb, 3, 1});
                cand.push_back(HopShape{12, gpb, 4, 1});
                cand.push_back(HopShape{13, gpb, 3, 1});
            }
    }
    if (!std::is_same<S, F64>::value)
        for (int pf : {2, 4, 8})
            for (int gpb : {1, 2, 3})
                if (gpb <= f.nrhs && (gpb == 1 || f.nrhs % gpb == 0)) cand.push_back(HopShape{-pf, gpb, 1, 1});
    HopShape best{1, 1, 1, 1};
    float best_ms = 1e30f;
    // candidates are timed on every RHS (the caller's gate may be partial;
    // the outputs of the fast kernels are scratch fields the launch that
    // follows overwrites)
    f.gate_st = nullptr;
    cudaEvent_t e0, e1;
    LQCD_CUDA(cudaEventCreate(&e0));
    LQCD_CUDA(cudaEventCreate(&e1));
    for (const HopShape &c : cand) {
        f.gpb = c.gpb;
        f.minb = c.minb;
        f.swz = c.swz;
        hopf_launch<S>(f, c.nr, mode, false, false, st);  // warm-up
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            LQCD_CUDA(cudaEventRecord(e0, st));
            hopf_launch<S>(f, c.nr, mode, false, false, st);
            LQCD_CUDA(cudaEventRecord(e1, st));
            LQCD_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            LQCD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LQCD_CHECK_LAUNCH();
    std::lock_guard<std::mutex> lk(mu);
    table[key] = best;
    tune_record(prec_name<S>(), mode, f.vh, f.nrhs, best.nr, best.gpb, best.minb, best.swz, best_ms);
    return best;
}

template <class S>
static FastHop<S> make_fast(const HopArgs<S, S, S> &a)
{
    FastHop<S> f{};
    for (int m = 0; m < 4; ++m) {
        f.L[m] = a.g.L[m];
        f.th_re[m] = a.th_re[m];
        f.th_im[m] = a.th_im[m];
        if (a.th_re[m] != 1.0 || a.th_im[m] != 0.0) f.theta_mask |= 1 << m;
    }
    f.Lxh = a.g.Lxh;
    f.vh = a.g.vh;
    f.nrhs = a.nrhs;
    f.ntiles = a.ntiles;
    f.parity = a.parity;
    f.dx = make_fastdiv(unsigned(a.g.Lxh));
    f.dy = make_fastdiv(unsigned(a.g.L[1]));
    f.dz = make_fastdiv(unsigned(a.g.L[2]));
    f.oy = a.g.Lxh;
    f.oz = a.g.Lxh * a.g.L[1];
    f.ot = a.g.Lxh * a.g.L[1] * a.g.L[2];
    f.coef = a.coef;
    f.gpb = 1;
    f.minb = 1;
    f.swz = 1;
    f.in = a.in;
    f.self = a.self;
    f.out = a.out;
    f.b = a.b;
    f.U = a.U;
    f.clov = a.clov;
    f.gate_st = a.gate_st;
    f.gate = a.gate;
    f.red = a.red;
    return f;
}

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
    const int nact = a.nactive >= 0 ? std::min(a.nactive, a.nrhs) : a.nrhs;  // RHS that pass the gate
    double per_rhs = sb + (mode == RESID ? 0.0 : sb) + (mode == HOP_CLOV ? 0.0 : sb) + (mode == RESID ? sb : 0.0);
    // the twisted inverse reads two Hermitian block pairs (B and C)
    const bool twinv = a.tau != 0.0 && (mode == HOP_CLOV || mode == CLOV_SUM);
    double shared = 8.0 * link_bytes<L>() + (mode == SELF_PLAIN ? 0.0 : (twinv ? 2.0 : 1.0) * clover_bytes<C>());
    const int pi = S::W == 2 ? 0 : (S::W == 4 ? 1 : 2);
    // twisted mass runs on the generic kernel (hop_kernel) in every storage
    // format; the set-up and final modes have the fast kernel in FP64, without dagger
    const bool extra = std::is_same<S, F64>::value && !dag && (mode == SELF_PLAIN || mode == CLOV_SUM || mode == RESID);
    if ((mode == HOP_CLOV || mode == SELF_CLOV || extra) && (a.tau == 0.0 || mode == SELF_PLAIN)) {
        FastHop<S> f = make_fast(a);
        const HopShape sh = a.fixed_shape ? HopShape{1, 1, 1, 1} : hopf_tuned<S>(f, mode, st);
        f.gpb = sh.gpb;
        f.minb = sh.minb;
        f.swz = sh.swz;
        const bool quad = is_tile_shape(sh.nr);
        if (quad && norm && !a.red.partial_f) throw Error{LQCD_EINVAL, "tile hopping kernel: no FP32 partials"};
        {
            ProfScope prof(kHopNames[pi][mode], double(a.g.vh) * (nact * per_rhs + (nact ? shared : 0.0)), st);
            hopf_launch<S>(f, sh.nr, mode, dag, norm, st);
            LQCD_CHECK_LAUNCH();
        }
        if (norm) launch_partial_finish(a.red, a.ntiles, a.nrhs, a.gate_st, a.gate, st, quad);
        return;
    }
    ProfScope prof(kHopNames[pi][mode], double(a.g.vh) * (nact * per_rhs + (nact ? shared : 0.0)), st);
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
