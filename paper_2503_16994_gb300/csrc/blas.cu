// Launchers of the CG vector kernels (explicit instantiations).
#include "lqcd_impl.h"

namespace lqcd {

// |x|^2 of an FP64 field -> red.op
__global__ void __launch_bounds__(128) norm2_f64(VecArgs v, SpinorField<F64> x)
{
    const int j = blockIdx.x % v.nrhs, tile = blockIdx.x / v.nrhs;
    if (v.gate_st && v.gate_st[j].status != v.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    double n2 = 0.0;
    if (i < v.vh) n2 = norm2_sp(load_spinor<F64, double>(x, j, i));
    reduce_finish(v.red, j, tile, v.ntiles, n2);
}

// Partial of 128-site tile k of RHS j.  QUAD: the FP32 sums of its four
// 32-site quarters, combined as the 128-thread block of reduce_partial2
// combines its four warps ((q0 + q2) + (q1 + q3), in FP32), so both give the
// same value.
template <bool QUAD>
__device__ __forceinline__ double tile_partial(const Reduce &r, int j, int ntiles, int k)
{
    if constexpr (QUAD) {
        const float *q = r.partial_f + ((long)j * ntiles + k) * 4;
        return double((q[0] + q[2]) + (q[1] + q[3]));
    } else {
        return r.partial[(long)j * ntiles + k];
    }
}

// Sum of the per-tile partials of each gated-in RHS (one block of 512
// threads per RHS, four independent accumulators per thread, fixed order:
// deterministic) and its operation.
constexpr int kFinishThreads = 512;
template <bool QUAD>
__global__ void __launch_bounds__(kFinishThreads) partial_finish_kernel(Reduce r, int ntiles, const RhsState *gate_st,
                                                                       int gate)
{
    __shared__ double sh[32];
    const int j = blockIdx.x;
    if (gate_st && gate_st[j].status != gate) return;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    int k = threadIdx.x;
    for (; k + 3 * kFinishThreads < ntiles; k += 4 * kFinishThreads) {
        t0 += tile_partial<QUAD>(r, j, ntiles, k);
        t1 += tile_partial<QUAD>(r, j, ntiles, k + kFinishThreads);
        t2 += tile_partial<QUAD>(r, j, ntiles, k + 2 * kFinishThreads);
        t3 += tile_partial<QUAD>(r, j, ntiles, k + 3 * kFinishThreads);
    }
    for (; k < ntiles; k += kFinishThreads) t0 += tile_partial<QUAD>(r, j, ntiles, k);
    double t = block_sum((t0 + t1) + (t2 + t3), sh);
    if (threadIdx.x == 0) apply_op(r, j, t);
}

void launch_partial_finish(const Reduce &r, int ntiles, int nrhs, const RhsState *gate_st, int gate, cudaStream_t st,
                           bool quad)
{
    ProfScope prof("norm_finish", double(nrhs) * ntiles * (quad ? 16.0 : 8.0), st);
    if (quad)
        partial_finish_kernel<true><<<unsigned(nrhs), kFinishThreads, 0, st>>>(r, ntiles, gate_st, gate);
    else
        partial_finish_kernel<false><<<unsigned(nrhs), kFinishThreads, 0, st>>>(r, ntiles, gate_st, gate);
    LQCD_CHECK_LAUNCH();
}

static unsigned grid_of(const VecArgs &v) { return unsigned(v.ntiles * v.nrhs); }
// right-hand sides a launch is expected to work on (accounting only)
static double nact(const VecArgs &v) { return v.nactive >= 0 ? std::min(v.nactive, v.nrhs) : v.nrhs; }

template <class W, class E>
void launch_er_update(const VecArgs &v, SpinorField<W> p, SpinorField<W> w, SpinorField<W> r, SpinorField<E> e,
                      cudaStream_t st)
{
    ProfScope prof(prec_name<W>() == std::string("f64") ? "cg_er_update_f64" : (prec_name<W>() == std::string("f32") ? "cg_er_update_f32" : "cg_er_update_f16"),
                   double(v.vh) * nact(v) * (4.0 * spinor_bytes<W>() + 2.0 * spinor_bytes<E>()), st);
    cg_er_update<W, E><<<grid_of(v), kBlock, 0, st>>>(v, p, w, r, e);
    LQCD_CHECK_LAUNCH();
}

template <class W>
void launch_p_update(const VecArgs &v, const RhsState *s, SpinorField<W> z, SpinorField<W> p, cudaStream_t st)
{
    ProfScope prof("cg_p_update", double(v.vh) * nact(v) * 3.0 * spinor_bytes<W>(), st);
    cg_p_update<W><<<grid_of(v), kBlock, 0, st>>>(v, s, z, p);
    LQCD_CHECK_LAUNCH();
}

template <class E>
void launch_x_update(const VecArgs &v, const RhsState *s, SpinorField<E> e, SpinorField<F64> x, cudaStream_t st)
{
    ProfScope prof("cg_x_update", double(v.vh) * nact(v) * (2.0 * spinor_bytes<E>() + 2.0 * 192.0), st);
    cg_x_update<E><<<grid_of(v), kBlock, 0, st>>>(v, s, e, x);
    LQCD_CHECK_LAUNCH();
}

template <class W, class WI>
void launch_r_replace(const VecArgs &v, SpinorField<F64> src, SpinorField<WI> w, SpinorField<W> r,
                      SpinorField<F64> save, bool w_scaled, cudaStream_t st)
{
    ProfScope prof("cg_r_replace",
                   double(v.vh) * nact(v) * (192.0 + spinor_bytes<WI>() + spinor_bytes<W>() + (save.p ? 192.0 : 0.0)),
                   st);
    cg_r_replace<W, WI><<<grid_of(v), kBlock, 0, st>>>(v, src, w, r, save, w_scaled);
    LQCD_CHECK_LAUNCH();
}

void launch_norm2_f64(const VecArgs &v, SpinorField<F64> x, cudaStream_t st)
{
    ProfScope prof("norm2_f64", double(v.vh) * v.nrhs * 192.0, st);
    norm2_f64<<<grid_of(v), kBlock, 0, st>>>(v, x);
    LQCD_CHECK_LAUNCH();
}

template <class S, class C>
void launch_clover_apply(long vh, int nrhs, int parity, CloverField<C> cl, SpinorField<S> in, SpinorField<S> out,
                         cudaStream_t st, double tau, CloverField<C> cl2)
{
    ProfScope prof("clover_apply",
                   double(vh) * (nrhs * 2.0 * spinor_bytes<S>() + (tau != 0.0 ? 2.0 : 1.0) * clover_bytes<C>()), st);
    clover_apply_kernel<S, C>
        <<<unsigned(ntiles_of(vh) * nrhs), kBlock, 0, st>>>(int(vh), nrhs, parity, cl, in, out, tau, cl2);
    LQCD_CHECK_LAUNCH();
}

template <class SI, class SO>
void launch_convert(long vh, int nrhs, SpinorField<SI> in, SpinorField<SO> out, cudaStream_t st)
{
    ProfScope prof("convert", double(vh) * nrhs * (spinor_bytes<SI>() + spinor_bytes<SO>()), st);
    convert_kernel<SI, SO><<<unsigned(ntiles_of(vh) * nrhs), kBlock, 0, st>>>(int(vh), nrhs, in, out);
    LQCD_CHECK_LAUNCH();
}

template void launch_convert<F64, F64>(long, int, SpinorField<F64>, SpinorField<F64>, cudaStream_t);
template void launch_convert<F64, F32>(long, int, SpinorField<F64>, SpinorField<F32>, cudaStream_t);
template void launch_convert<F64, F16>(long, int, SpinorField<F64>, SpinorField<F16>, cudaStream_t);
template void launch_convert<F32, F64>(long, int, SpinorField<F32>, SpinorField<F64>, cudaStream_t);
template void launch_convert<F16, F64>(long, int, SpinorField<F16>, SpinorField<F64>, cudaStream_t);
template void launch_er_update<F64, F64>(const VecArgs &, SpinorField<F64>, SpinorField<F64>, SpinorField<F64>,
                                         SpinorField<F64>, cudaStream_t);
template void launch_er_update<F32, F32>(const VecArgs &, SpinorField<F32>, SpinorField<F32>, SpinorField<F32>,
                                         SpinorField<F32>, cudaStream_t);
template void launch_er_update<F16, F32>(const VecArgs &, SpinorField<F16>, SpinorField<F16>, SpinorField<F16>,
                                         SpinorField<F32>, cudaStream_t);
template void launch_p_update<F64>(const VecArgs &, const RhsState *, SpinorField<F64>, SpinorField<F64>, cudaStream_t);
template void launch_p_update<F32>(const VecArgs &, const RhsState *, SpinorField<F32>, SpinorField<F32>, cudaStream_t);
template void launch_p_update<F16>(const VecArgs &, const RhsState *, SpinorField<F16>, SpinorField<F16>, cudaStream_t);
template void launch_x_update<F64>(const VecArgs &, const RhsState *, SpinorField<F64>, SpinorField<F64>, cudaStream_t);
template void launch_x_update<F32>(const VecArgs &, const RhsState *, SpinorField<F32>, SpinorField<F64>, cudaStream_t);
template void launch_r_replace<F64, F64>(const VecArgs &, SpinorField<F64>, SpinorField<F64>, SpinorField<F64>,
                                         SpinorField<F64>, bool, cudaStream_t);
template void launch_r_replace<F32, F64>(const VecArgs &, SpinorField<F64>, SpinorField<F64>, SpinorField<F32>,
                                         SpinorField<F64>, bool, cudaStream_t);
template void launch_r_replace<F16, F64>(const VecArgs &, SpinorField<F64>, SpinorField<F64>, SpinorField<F16>,
                                         SpinorField<F64>, bool, cudaStream_t);
template void launch_r_replace<F32, F32>(const VecArgs &, SpinorField<F64>, SpinorField<F32>, SpinorField<F32>,
                                         SpinorField<F64>, bool, cudaStream_t);
template void launch_r_replace<F16, F32>(const VecArgs &, SpinorField<F64>, SpinorField<F32>, SpinorField<F16>,
                                         SpinorField<F64>, bool, cudaStream_t);
template void launch_clover_apply<F64, F64>(long, int, int, CloverField<F64>, SpinorField<F64>, SpinorField<F64>,
                                            cudaStream_t, double, CloverField<F64>);

}  // namespace lqcd
