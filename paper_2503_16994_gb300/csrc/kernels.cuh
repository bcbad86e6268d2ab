// Kernel templates of the Wilson-clover path.  Included by the translation
// units that instantiate them (one per storage precision, plus field_ops.cu).
#pragma once
#include <type_traits>

#include "lqcd_dev.cuh"

namespace lqcd {

// ---------------------------------------------------------------------------
// per right-hand-side solver state (device resident, one struct per RHS)
// ---------------------------------------------------------------------------
// ST_RESUME: just updated in FP64 while the others went on (batched
// solves); runs the second half of its iteration, then becomes ST_ACTIVE.
enum RhsStatus : int { ST_DONE = 0, ST_ACTIVE = 1, ST_UPDATE = 2, ST_MAXITER = 3, ST_IDLE = 4, ST_RESUME = 5 };

struct RhsState {
    double gamma;    // |z|^2, z = Dhat^dag r (CGLS)
    double alpha, beta;
    double rr;       // |r|^2 of the low-precision residual
    double rr_ref;   // |r|^2 right after the last FP64 residual recomputation
    double scale;    // FP64 residual = scale * r, correction = scale * e
    double bnorm2;   // |b|^2 of the full system
    double target2;  // stop when the FP64 residual norm^2 <= target2
    double delta2;   // reliable-update factor squared
    double acc;      // accumulator for norms (true residual, |b|^2)
    double anchor2;  // |rhat|^2 of the last FP64 residual (the anchor of the incremental updates)
    int status;
    int iter;
    int updates;
    int maxiter;
    int resume;      // status after an FP64 residual that did not finish: ST_ACTIVE or ST_RESUME
};

// What the last block does with a finished per-RHS sum.
enum RedOp : int {
    RED_STORE = 0,   // acc = sum
    RED_ADD = 1,     // acc += sum
    RED_ALPHA = 2,   // alpha = gamma / sum
    RED_BETA = 3,    // beta = sum / gamma (0 on the first pass); gamma = sum
    RED_RUPDATE = 4, // rr = sum; iter++; request an FP64 residual when due
    RED_RHAT = 5,    // sum = |FP64 residual|^2: finish, or resume the inner iteration
    RED_RHAT_COARSE = 6  // sum = |residual|^2 updated with an FP32 operator: resume (never finishes)
};

struct Reduce {
    double *partial;     // [nrhs][ntiles]
    unsigned *counter;   // [nrhs], zero between uses
    RhsState *st;        // [nrhs]
    int op;
    float *partial_f;    // [nrhs][4 ntiles]: FP32 sums per 32 sites (tile hopping kernel), or null
};

__device__ __forceinline__ void apply_op(const Reduce &r, int j, double sum)
{
    RhsState &s = r.st[j];
    switch (r.op) {
    case RED_STORE: s.acc = sum; break;
    case RED_ADD: s.acc += sum; break;
    case RED_ALPHA: s.alpha = sum > 0.0 ? s.gamma / sum : 0.0; break;
    case RED_BETA:
        s.beta = s.gamma > 0.0 ? sum / s.gamma : 0.0;
        s.gamma = sum;
        break;
    case RED_RUPDATE:
        s.rr = sum;
        s.iter += 1;
        if (sum <= s.delta2 * s.rr_ref || s.scale * s.scale * sum <= s.target2 || s.iter >= s.maxiter ||
            !(sum == sum))
            s.status = ST_UPDATE;
        break;
    case RED_RHAT:
        s.updates += 1;
        s.rr = sum / (s.scale * s.scale);
        s.rr_ref = s.rr;
        s.anchor2 = sum;
        if (sum <= s.target2)
            s.status = ST_DONE;
        else if (s.iter >= s.maxiter || !(sum == sum))
            s.status = ST_MAXITER;
        else
            s.status = s.resume;
        break;
    case RED_RHAT_COARSE:
        s.rr = sum / (s.scale * s.scale);
        s.rr_ref = s.rr;
        s.status = (sum == sum) ? s.resume : ST_UPDATE;  // a NaN goes to the FP64 update
        break;
    }
}

// Block-wide sum of v, written as this block's partial; the last block of
// RHS j to arrive sums all partials in a fixed order (deterministic) and
// applies the operation.  Must be called by every thread of the block.
__device__ __forceinline__ void reduce_finish(const Reduce &r, int j, int tile, int ntiles, double v)
{
    __shared__ double sh[32];
    __shared__ int last;
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) {
        r.partial[(long)j * ntiles + tile] = s;
        __threadfence();
        unsigned prev = atomicAdd(&r.counter[j], 1u);
        last = (prev == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0.0;
        for (int k = threadIdx.x; k < ntiles; k += blockDim.x) t += __ldcg(r.partial + (long)j * ntiles + k);
        t = block_sum(t, sh);
        if (threadIdx.x == 0) {
            r.counter[j] = 0;
            apply_op(r, j, t);
        }
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of v written as this block's partial of RHS j, nothing
// else: no fence, no atomic, so the block does not wait for its own stores.
// The partials are summed in FP64 by partial_finish_kernel (launched after
// the producing kernel).  T is the type the block sums in: float for the
// FP16/FP32 kernels, whose per-thread values are FP32 sums already (FP64 adds
// are scarce on this GPU), double for the FP64 kernels.  Must be called by
// every thread of the block.
template <typename T>
__device__ __forceinline__ void reduce_partial(const Reduce &r, int j, int tile, int ntiles, T v)
{
    __shared__ T sh[32];
    v = warp_sum_t(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = warp_sum_t(lane < nw ? sh[lane] : T(0));
        if (lane == 0) r.partial[(long)j * ntiles + tile] = double(v);
    }
}
// the same for two right-hand sides at once (one pair of barriers), in FP32
__device__ __forceinline__ void reduce_partial2(const Reduce &r, int ja, bool on_a, int jb, bool on_b, int tile,
                                                int ntiles, float va, float vb)
{
    __shared__ float sh[2][32];
    va = warp_sum_t(va);
    vb = warp_sum_t(vb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[0][wid] = va;
        sh[1][wid] = vb;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        va = warp_sum_t(lane < nw ? sh[0][lane] : 0.f);
        vb = warp_sum_t(lane < nw ? sh[1][lane] : 0.f);
        if (lane == 0) {
            if (on_a) r.partial[(long)ja * ntiles + tile] = double(va);
            if (on_b) r.partial[(long)jb * ntiles + tile] = double(vb);
        }
    }
}

// ---------------------------------------------------------------------------
// hopping term with fused epilogues
//
// H psi (x) = sum_mu [ (1 - s g_mu) U~_mu(x) psi(x+mu) + (1 + s g_mu) U~_mu(x-mu)^dag psi(x-mu) ]
// with s = +1 (D) or s = -1 (D^dag = g5 D g5, which swaps the projectors).
// Output sites have parity `parity`; psi lives on the other parity.
// ---------------------------------------------------------------------------
enum HopMode : int {
    HOP_CLOV = 0,   // out = coef * C (H in)
    SELF_CLOV = 1,  // out = C self + coef * H in
    SELF_PLAIN = 2, // out = self + coef * H in
    CLOV_SUM = 3,   // out = C (self + coef * H in)
    RESID = 4       // |b - (C self + coef * H in)|^2 only, nothing stored
};

template <class S, class L, class C>
struct HopArgs {
    Geom g;
    int parity;
    int nrhs;
    int ntiles;
    SpinorField<S> in, self, out, b;
    LinkField<L> U;
    CloverField<C> clov;   // clover blocks used by the epilogue (output parity taken from `parity`)
    CloverField<C> clov2;  // twisted mass: the C blocks of the inverse (clov then holds B), else unused
    double tau;            // twisted mass 2 kappa mu of the site term (0: none); the dagger uses -tau
    double coef;
    double th_re[4], th_im[4];
    const RhsState *gate_st;  // nullptr: every RHS runs
    int gate;                 // RHS j runs only if gate_st[j].status == gate
    Reduce red;
    int nactive = -1;         // launch accounting only: right-hand sides expected to pass the gate (-1: all)
    bool fixed_shape = false; // true: the scalar one-RHS-per-thread shape, neither tuned nor forced by
                              // the environment (its bits do not depend on the tuner's choice)
};

template <class S, class L, class C, typename R, int MU, int SGN>
__device__ __forceinline__ void hop_dir(const HopArgs<S, L, C> &a, int j, int i, const int x[4], spinor<R> &acc)
{
    constexpr int SF = -SGN;  // forward projector (1 - s g)
    constexpr int SB = SGN;   // backward projector (1 + s g)
    {
        int y = cb_neighbour(a.g, x, MU, +1);
        su3<R> U = load_link<L, R>(a.U, a.parity, MU, i);
        spinor<R> p = load_spinor<S, R>(a.in, j, y);
        hspinor<R> h = mul(U, project<R, MU, SF>(p));
        if (x[MU] == a.g.L[MU] - 1) scale_h(h, cx<R>{R(a.th_re[MU]), R(a.th_im[MU])});
        accumulate<R, MU, SF>(acc, h);
    }
    {
        int y = cb_neighbour(a.g, x, MU, -1);
        su3<R> U = load_link<L, R>(a.U, a.parity ^ 1, MU, y);
        spinor<R> p = load_spinor<S, R>(a.in, j, y);
        hspinor<R> h = mul_dag(U, project<R, MU, SB>(p));
        if (x[MU] == 0) scale_h(h, cx<R>{R(a.th_re[MU]), R(-a.th_im[MU])});
        accumulate<R, MU, SB>(acc, h);
    }
}

template <typename R> __device__ __forceinline__ spinor<R> axpy_sp(R c, const spinor<R> &x, const spinor<R> &y)
{
    spinor<R> r;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k) r.s[s][k] = c * x.s[s][k] + y.s[s][k];
    return r;
}

// out += i t g5 v: in the chiral basis g5 = +1 on spins 0, 1 and -1 on spins
// 2, 3, so the twisted-mass site term i tau g5 is a diagonal phase
template <typename R> __device__ __forceinline__ void add_twist(spinor<R> &out, R t, const spinor<R> &v)
{
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const R ts = s < 2 ? t : -t;
#pragma unroll
        for (int k = 0; k < 3; ++k) out.s[s][k] = out.s[s][k] + ts * mul_i(v.s[s][k]);
    }
}

// (A + i t g5)^-1 v = (B - i t g5 C) v for the Hermitian blocks B = A C and
// C = (A^2 + t^2)^-1 of each chirality (A Hermitian)
template <typename R>
__device__ __forceinline__ spinor<R> twisted_inverse(const clover_block<R> B[2], const clover_block<R> C[2], R t,
                                                     const spinor<R> &v)
{
    spinor<R> r = clover_apply(B, v);
    add_twist(r, -t, clover_apply(C, v));
    return r;
}

template <typename R> __device__ __forceinline__ double norm2_sp(const spinor<R> &x)
{
    R acc = R(0);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += norm2(x.s[s][k]);
    return double(acc);
}

template <class S, class L, class C, typename R, int MODE, bool DAG, bool NORM>
__global__ void __launch_bounds__(128) hop_kernel(const HopArgs<S, L, C> a)
{
    const int j = blockIdx.x % a.nrhs;
    const int tile = blockIdx.x / a.nrhs;
    if (a.gate_st && a.gate_st[j].status != a.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    double n2 = 0.0;
    if (i < a.g.vh) {
        int x[4];
        cb_coords(a.g, a.parity, i, x);
        spinor<R> acc;
        zero(acc);
        constexpr int SG = DAG ? -1 : 1;
        hop_dir<S, L, C, R, 0, SG>(a, j, i, x, acc);
        hop_dir<S, L, C, R, 1, SG>(a, j, i, x, acc);
        hop_dir<S, L, C, R, 2, SG>(a, j, i, x, acc);
        hop_dir<S, L, C, R, 3, SG>(a, j, i, x, acc);
        const R coef = R(a.coef);
        // twisted mass: the site term is A + i tau g5, its adjoint takes -tau
        const R tau = R(DAG ? -a.tau : a.tau);
        spinor<R> res;
        if constexpr (MODE == HOP_CLOV) {
            clover_block<R> blk[2];
            load_clover<C, R>(a.clov, a.parity, i, blk);
            if (tau != R(0)) {
                clover_block<R> blk2[2];
                load_clover<C, R>(a.clov2, a.parity, i, blk2);
                res = twisted_inverse(blk, blk2, tau, acc);
            } else {
                res = clover_apply(blk, acc);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int k = 0; k < 3; ++k) res.s[s][k] = coef * res.s[s][k];
        } else if constexpr (MODE == SELF_PLAIN) {
            res = axpy_sp(coef, acc, load_spinor<S, R>(a.self, j, i));
        } else if constexpr (MODE == CLOV_SUM) {
            clover_block<R> blk[2];
            load_clover<C, R>(a.clov, a.parity, i, blk);
            const spinor<R> v = axpy_sp(coef, acc, load_spinor<S, R>(a.self, j, i));
            if (tau != R(0)) {
                clover_block<R> blk2[2];
                load_clover<C, R>(a.clov2, a.parity, i, blk2);
                res = twisted_inverse(blk, blk2, tau, v);
            } else {
                res = clover_apply(blk, v);
            }
        } else {  // SELF_CLOV, RESID
            clover_block<R> blk[2];
            load_clover<C, R>(a.clov, a.parity, i, blk);
            const spinor<R> sv = load_spinor<S, R>(a.self, j, i);
            spinor<R> site = clover_apply(blk, sv);
            if (tau != R(0)) add_twist(site, tau, sv);
            res = axpy_sp(coef, acc, site);
        }
        if constexpr (MODE == RESID) {
            res = axpy_sp(R(-1), res, load_spinor<S, R>(a.b, j, i));
            n2 = norm2_sp(res);
        } else {
            double s2 = store_spinor<S, R>(a.out, j, i, res);
            if (NORM) n2 = s2;
        }
    }
    if (NORM) reduce_finish(a.red, j, tile, a.ntiles, n2);
}

// ---------------------------------------------------------------------------
// CG vector kernels (one parity, nrhs right-hand sides)
// ---------------------------------------------------------------------------
struct VecArgs {
    int vh, nrhs, ntiles;
    const RhsState *gate_st;
    int gate;
    Reduce red;
    int nactive = -1;  // launch accounting only: right-hand sides expected to pass the gate (-1: all)
};

// e += alpha p ; r -= alpha w ; |r|^2 -> RED_RUPDATE
template <class W, class E>
__global__ void __launch_bounds__(128) cg_er_update(VecArgs v, SpinorField<W> p, SpinorField<W> w, SpinorField<W> r,
                                                    SpinorField<E> e)
{
    const int j = blockIdx.x % v.nrhs, tile = blockIdx.x / v.nrhs;
    if (v.gate_st && v.gate_st[j].status != v.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    double n2 = 0.0;
    if (i < v.vh) {
        const double al = v.red.st[j].alpha;
        using R = typename std::conditional<std::is_same<E, F64>::value, double, float>::type;
        spinor<R> pv = load_spinor<W, R>(p, j, i);
        spinor<R> ev = load_spinor<E, R>(e, j, i);
        store_spinor<E, R>(e, j, i, axpy_sp(R(al), pv, ev));
        spinor<R> wv = load_spinor<W, R>(w, j, i);
        spinor<R> rv = load_spinor<W, R>(r, j, i);
        n2 = store_spinor<W, R>(r, j, i, axpy_sp(R(-al), wv, rv));
    }
    reduce_finish(v.red, j, tile, v.ntiles, n2);
}

// p = z + beta p
template <class W>
__global__ void __launch_bounds__(128) cg_p_update(VecArgs v, const RhsState *st, SpinorField<W> z, SpinorField<W> p)
{
    const int j = blockIdx.x % v.nrhs, tile = blockIdx.x / v.nrhs;
    if (v.gate_st && v.gate_st[j].status != v.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= v.vh) return;
    using R = typename std::conditional<std::is_same<W, F64>::value, double, float>::type;
    const double be = st[j].beta;
    store_spinor<W, R>(p, j, i, axpy_sp(R(be), load_spinor<W, R>(p, j, i), load_spinor<W, R>(z, j, i)));
}

// x += scale e ; e = 0   (FP64 x)
template <class E>
__global__ void __launch_bounds__(128) cg_x_update(VecArgs v, const RhsState *st, SpinorField<E> e, SpinorField<F64> x)
{
    const int j = blockIdx.x % v.nrhs, tile = blockIdx.x / v.nrhs;
    if (v.gate_st && v.gate_st[j].status != v.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= v.vh) return;
    spinor<double> ev = load_spinor<E, double>(e, j, i);
    spinor<double> xv = load_spinor<F64, double>(x, j, i);
    store_spinor<F64, double>(x, j, i, axpy_sp(st[j].scale, ev, xv));
    spinor<double> z;
    zero(z);
    store_spinor<E, double>(e, j, i, z);
}

// an FP64 spinor through the coherent path (a field the same launch also writes)
__device__ __forceinline__ spinor<double> load_spinor_f64_rw(const SpinorField<F64> &f, int j, int i)
{
    spinor<double> a;
    double *v = reinterpret_cast<double *>(&a);
    const double2 *b = f.p + (long)j * 12 * f.stride + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 w = b[k * f.stride];
        v[2 * k] = w.x;
        v[2 * k + 1] = w.y;
    }
    return a;
}

// rhat = src - c w (FP64 arithmetic): the FP64 update has src = bhat, w =
// Dhat x in FP64 and c = 1; the incremental update has src = the previous
// rhat, w = Dhat e in FP32 and c = scale (w_scaled).  r = rhat / scale (low
// precision); |rhat|^2 -> RED_RHAT(_COARSE); save (if set, may be src): rhat
// kept in FP64 for the next incremental update
template <class W, class WI>
__global__ void __launch_bounds__(128) cg_r_replace(VecArgs v, SpinorField<F64> src, SpinorField<WI> w,
                                                    SpinorField<W> r, SpinorField<F64> save, bool w_scaled)
{
    const int j = blockIdx.x % v.nrhs, tile = blockIdx.x / v.nrhs;
    if (v.gate_st && v.gate_st[j].status != v.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    double n2 = 0.0;
    if (i < v.vh) {
        const double c = w_scaled ? v.red.st[j].scale : 1.0;
        spinor<double> rh = axpy_sp(-c, load_spinor<WI, double>(w, j, i), load_spinor_f64_rw(src, j, i));
        if (save.p) store_spinor<F64, double>(save, j, i, rh);
        n2 = norm2_sp(rh);
        const double inv = 1.0 / v.red.st[j].scale;
        using R = typename std::conditional<std::is_same<W, F64>::value, double, float>::type;
        spinor<R> rl;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int k = 0; k < 3; ++k) rl.s[s][k] = cx<R>{R(rh.s[s][k].re * inv), R(rh.s[s][k].im * inv)};
        store_spinor<W, R>(r, j, i, rl);
    }
    reduce_finish(v.red, j, tile, v.ntiles, n2);
}

// out = in, converted between storage formats
template <class SI, class SO>
__global__ void __launch_bounds__(128) convert_kernel(int vh, int nrhs, SpinorField<SI> in, SpinorField<SO> out)
{
    const int j = blockIdx.x % nrhs, tile = blockIdx.x / nrhs;
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    store_spinor<SO, double>(out, j, i, load_spinor<SI, double>(in, j, i));
}

// out = C in (clover blocks of parity `parity`); with tau != 0 the twisted
// inverse (B - i tau g5 C2) in, cl holding B and cl2 C
template <class S, class C>
__global__ void __launch_bounds__(128) clover_apply_kernel(int vh, int nrhs, int parity, CloverField<C> cl,
                                                           SpinorField<S> in, SpinorField<S> out, double tau,
                                                           CloverField<C> cl2)
{
    const int j = blockIdx.x % nrhs, tile = blockIdx.x / nrhs;
    const int i = tile * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    using R = typename std::conditional<std::is_same<S, F64>::value, double, float>::type;
    clover_block<R> blk[2];
    load_clover<C, R>(cl, parity, i, blk);
    const spinor<R> v = load_spinor<S, R>(in, j, i);
    if (tau != 0.0) {
        clover_block<R> blk2[2];
        load_clover<C, R>(cl2, parity, i, blk2);
        store_spinor<S, R>(out, j, i, twisted_inverse(blk, blk2, R(tau), v));
    } else {
        store_spinor<S, R>(out, j, i, clover_apply(blk, v));
    }
}

}  // namespace lqcd
