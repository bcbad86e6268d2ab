// Even-odd preconditioned CG (CGLS form) with FP64 reliable updates.
//
// System: D x = b with D = [[A_ee, -k H_eo], [-k H_oe, A_oo]] (A = clover site
// term, H = hopping term, k = kappa).  Schur complement on the even sites:
//   Dhat = A_ee - k^2 H_eo A_oo^-1 H_oe,  bhat = b_e + k H_eo A_oo^-1 b_o,
//   x_o  = A_oo^-1 (b_o + k H_oe x_e),
// and the full residual equals bhat - Dhat x_e on the even sites (zero on the
// odd ones), so |b - D x| = |bhat - Dhat x_e| up to rounding.
//
// Dhat is solved by CG on the normal equations in CGLS form (the recursion
// tracks r = rhat - Dhat e, the residual of the system itself):
//   z = Dhat^dag r, p = z, gamma = |z|^2
//   repeat: w = Dhat p; alpha = gamma/|w|^2; e += alpha p; r -= alpha w;
//           z = Dhat^dag r; beta = |z|^2/gamma; gamma = |z|^2; p = z + beta p
// with Dhat^dag = g5 Dhat g5 (the hopping projectors swap, the clover term
// commutes with g5).  The inner vectors are FP64, FP32 or FP16; every time the
// inner residual has dropped by delta (or looks converged, or the iteration
// cap is hit) the correction is added to the FP64 solution and the residual
// is recomputed in FP64 (reliable update), keeping p.  Mixed solvers whose
// residual is still far from tol and from the last FP64 one instead move
// the FP64 residual by the FP32 image of the correction (incremental update,
// below).  Per-RHS scalars and the state machine live on the device; the host
// only polls the states every few iterations.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "lqcd_impl.h"

namespace lqcd {

template <class S> static size_t field_bytes(long stride, int nrhs)
{
    return sizeof(typename S::word) * spinor_planes<S>::n * (size_t)stride * nrhs;
}

template <class S> static SpinorField<S> fld(DevBuf &b, DevBuf *sc, long stride)
{
    return {b.as<typename S::word>(), sc ? sc->as<float>() : nullptr, stride};
}

Workspace::~Workspace()
{
    if (host_state) {
        if (host_pageable)
            std::free(host_state);
        else
            cudaFreeHost(host_state);
    }
}

// partial sums: the solver's reductions need nrhs * ntiles doubles followed
// by the 4 nrhs ntiles FP32 partials of the tile hopping kernel (the room of
// 2 nrhs ntiles doubles), the contraction T * ceil(V3/2 / 128) <= ntiles + T;
// counters: max(nrhs, T)
static size_t partial_count(const lqcd_lattice_s *lat, int nrhs)
{
    return std::max(3 * (size_t)nrhs * ntiles_of(lat->vh), (size_t)ntiles_of(lat->vh) + lat->dims[3]);
}

template <class W, class E>
static size_t workspace_bytes_t(const lqcd_lattice_s *lat, int nrhs)
{
    const long S = lat->stride;
    size_t b = 7 * field_bytes<F64>(S, nrhs) + 5 * field_bytes<W>(S, nrhs) + field_bytes<E>(S, nrhs);
    if (std::is_same<W, F16>::value) b += 5 * sizeof(float) * S * nrhs;
    b += sizeof(RhsState) * nrhs + sizeof(double) * partial_count(lat, nrhs) +
         sizeof(unsigned) * std::max(nrhs, lat->dims[3]);
    return b;
}

size_t workspace_bytes(const lqcd_lattice_s *lat, int nrhs, int prec)
{
    switch (prec) {
    case LQCD_PREC_FP64: return workspace_bytes_t<F64, F64>(lat, nrhs);
    case LQCD_PREC_MIXED_FP32: return workspace_bytes_t<F32, F32>(lat, nrhs);
    default: return workspace_bytes_t<F16, F32>(lat, nrhs);
    }
}

template <class W, class E>
static std::unique_ptr<Workspace> workspace_build_t(lqcd_lattice_s *lat, int nrhs, int prec, cudaStream_t st,
                                                    bool async)
{
    auto w = std::make_unique<Workspace>();
    w->nrhs = nrhs;
    w->prec = prec;
    if (async)
        for (DevBuf *b : {&w->b_e, &w->b_o, &w->bhat, &w->x_e, &w->x_o, &w->t64, &w->w64, &w->p, &w->t, &w->w, &w->r,
                          &w->z, &w->p_sc, &w->t_sc, &w->w_sc, &w->r_sc, &w->z_sc, &w->e, &w->state, &w->partial,
                          &w->counter})
            b->set_async(st);
    const long S = lat->stride;
    for (DevBuf *b : {&w->b_e, &w->b_o, &w->bhat, &w->x_e, &w->x_o, &w->t64, &w->w64}) b->ensure(field_bytes<F64>(S, nrhs));
    for (DevBuf *b : {&w->p, &w->t, &w->w, &w->r, &w->z}) b->ensure(field_bytes<W>(S, nrhs));
    if (std::is_same<W, F16>::value)
        for (DevBuf *b : {&w->p_sc, &w->t_sc, &w->w_sc, &w->r_sc, &w->z_sc}) b->ensure(sizeof(float) * S * nrhs);
    w->e.ensure(field_bytes<E>(S, nrhs));
    w->state.ensure(sizeof(RhsState) * nrhs);
    w->partial.ensure(sizeof(double) * partial_count(lat, nrhs));
    w->counter.ensure(sizeof(unsigned) * std::max(nrhs, lat->dims[3]));
    LQCD_CUDA(cudaMemsetAsync(w->counter.p, 0, w->counter.bytes, st));
    if (async) {
        w->host_pageable = true;
        w->host_state = static_cast<RhsState *>(std::malloc(sizeof(RhsState) * nrhs));
        if (!w->host_state) throw Error{LQCD_ENOMEM, "host allocation failed"};
    } else {
        LQCD_CUDA(cudaMallocHost(&w->host_state, sizeof(RhsState) * nrhs));
    }
    return w;
}

std::unique_ptr<Workspace> workspace_build(lqcd_lattice_s *lat, int nrhs, int prec, cudaStream_t st, bool async)
{
    switch (prec) {
    case LQCD_PREC_FP64: return workspace_build_t<F64, F64>(lat, nrhs, prec, st, async);
    case LQCD_PREC_MIXED_FP32: return workspace_build_t<F32, F32>(lat, nrhs, prec, st, async);
    default: return workspace_build_t<F16, F32>(lat, nrhs, prec, st, async);
    }
}

template <class W, class E>
static Workspace &workspace(lqcd_lattice_s *lat, int nrhs, int prec, cudaStream_t st)
{
    auto key = std::make_pair(nrhs, prec);
    auto it = lat->ws.find(key);
    if (it != lat->ws.end()) return *it->second;
    auto w = workspace_build_t<W, E>(lat, nrhs, prec, st, false);
    Workspace &ref = *w;
    lat->ws.emplace(key, std::move(w));
    return ref;
}

__global__ void init_state_kernel(RhsState *s, int nrhs, double tol2, double delta2, int maxiter, int resume)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nrhs) return;
    RhsState q = s[j];
    q.bnorm2 = q.acc;
    q.scale = q.bnorm2 > 0.0 ? sqrt(q.bnorm2) : 1.0;
    q.target2 = tol2 * q.bnorm2;
    q.delta2 = delta2;
    q.maxiter = maxiter;
    q.status = q.bnorm2 > 0.0 ? ST_UPDATE : ST_DONE;
    q.gamma = q.alpha = q.beta = 0.0;
    q.rr = q.rr_ref = q.anchor2 = 0.0;
    q.iter = 0;
    q.updates = -1;  // the first FP64 residual (of the zero start) is not an update
    q.resume = resume;
    s[j] = q;
}

__global__ void set_resume_kernel(RhsState *s, int nrhs, int v)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nrhs) s[j].resume = v;
}

__global__ void status_change_kernel(RhsState *s, int nrhs, int from, int to)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nrhs && s[j].status == from) s[j].status = to;
}

template <class W, class E>
struct Solver {
    lqcd_lattice_s *lat;
    Workspace &ws;
    int nrhs;
    double kappa;
    cudaStream_t st;
    HopArgs<F64, F64, F64> h64;
    HopArgs<W, W, W> hw;
    HopArgs<F32, F32, F32> h32;  // FP32 operator of the incremental residual updates (mixed solvers)
    CloverField<F64> a64, ai64, ci64;  // ci64: the C blocks of a twisted inverse
    CloverField<W> aw, aiw;
    SpinorField<F64> b_e, b_o, bhat, x_e, x_o, t64, w64;
    SpinorField<W> p, t, w, r, z;
    SpinorField<E> e;
    RhsState *S;
    VecArgs v;

    Solver(lqcd_lattice_s *l, Workspace &w_, GaugeSet &g, CloverSet &cl, const lqcd_dirac_params &dp, int n,
           cudaStream_t s)
        : lat(l), ws(w_), nrhs(n), kappa(dp.kappa), st(s)
    {
        const long Sd = lat->stride;
        b_e = fld<F64>(ws.b_e, nullptr, Sd);
        b_o = fld<F64>(ws.b_o, nullptr, Sd);
        bhat = fld<F64>(ws.bhat, nullptr, Sd);
        x_e = fld<F64>(ws.x_e, nullptr, Sd);
        x_o = fld<F64>(ws.x_o, nullptr, Sd);
        t64 = fld<F64>(ws.t64, nullptr, Sd);
        w64 = fld<F64>(ws.w64, nullptr, Sd);
        const bool h = std::is_same<W, F16>::value;
        p = fld<W>(ws.p, h ? &ws.p_sc : nullptr, Sd);
        t = fld<W>(ws.t, h ? &ws.t_sc : nullptr, Sd);
        w = fld<W>(ws.w, h ? &ws.w_sc : nullptr, Sd);
        r = fld<W>(ws.r, h ? &ws.r_sc : nullptr, Sd);
        z = fld<W>(ws.z, h ? &ws.z_sc : nullptr, Sd);
        e = fld<E>(ws.e, nullptr, Sd);
        S = ws.state.as<RhsState>();
        a64 = clover_field<F64>(cl, false, Sd);
        ai64 = clover_field<F64>(cl, true, Sd);
        ci64 = clover_field_c<F64>(cl, Sd);
        aw = clover_field<W>(cl, false, Sd);
        aiw = clover_field<W>(cl, true, Sd);
        const int nt = ntiles_of(lat->vh);
        Reduce red{ws.partial.as<double>(), ws.counter.as<unsigned>(), S, RED_STORE,
                   reinterpret_cast<float *>(ws.partial.as<double>() + (size_t)nrhs * nt)};
        v = VecArgs{int(lat->vh), nrhs, nt, nullptr, 0, red};
        h64 = HopArgs<F64, F64, F64>{};
        h64.g = lat->geom;
        h64.nrhs = nrhs;
        h64.ntiles = nt;
        h64.U = hop_links<F64>(g, Sd, dp.bc);
        hop_theta(dp, h64.th_re, h64.th_im);
        h64.red = red;
        h64.tau = cl.tau;
        h64.clov2 = ci64;
        hw = HopArgs<W, W, W>{};
        hw.g = lat->geom;
        hw.nrhs = nrhs;
        hw.ntiles = nt;
        hw.U = hop_links<W>(g, Sd, dp.bc);
        hop_theta(dp, hw.th_re, hw.th_im);
        hw.red = red;
        hw.tau = cl.tau;
        hw.clov2 = clover_field_c<W>(cl, Sd);
        h32 = HopArgs<F32, F32, F32>{};
        h32.g = lat->geom;
        h32.nrhs = nrhs;
        h32.ntiles = nt;
        h32.U = hop_links<F32>(g, Sd, dp.bc);
        hop_theta(dp, h32.th_re, h32.th_im);
        h32.red = red;
        h32.tau = cl.tau;
        a32 = clover_field<F32>(cl, false, Sd);
        ai32 = clover_field<F32>(cl, true, Sd);
        h32.clov2 = clover_field_c<F32>(cl, Sd);
    }
    CloverField<F32> a32, ai32;

    // right-hand sides expected to pass each gate, from the last host poll
    // (launch accounting only; -1 when unknown)
    int hint_active = -1, hint_update = -1;
    int hint(int gate) const { return gate == ST_UPDATE ? hint_update : hint_active; }

    VecArgs gated(int gate, int op) const
    {
        VecArgs q = v;
        q.gate_st = S;
        q.gate = gate;
        q.red.op = op;
        q.nactive = hint(gate);
        return q;
    }

    // |b|^2, bhat = b_e + k H_eo A_oo^-1 b_o, state initialisation, x = e = p = 0
    int resume = ST_ACTIVE;  // ST_RESUME for batched solves (the update happens between graph chunks)

    // guess: x_e already holds the even part of an initial guess (kept)
    void prepare(double tol_eff, double delta, int maxiter, bool guess)
    {
        VecArgs q = v;
        q.red.op = RED_STORE;
        launch_norm2_f64(q, b_e, st);
        q.red.op = RED_ADD;
        launch_norm2_f64(q, b_o, st);
        launch_clover_apply<F64, F64>(lat->vh, nrhs, 1, ai64, b_o, t64, st, h64.tau, ci64);
        HopArgs<F64, F64, F64> a = h64;
        a.parity = 0;
        a.in = t64;
        a.self = b_e;
        a.out = bhat;
        a.coef = kappa;
        launch_hop(a, SELF_PLAIN, false, false, st);
        init_state_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(S, nrhs, tol_eff * tol_eff, delta * delta, maxiter,
                                                           resume);
        LQCD_CHECK_LAUNCH();
        if (!guess) LQCD_CUDA(cudaMemsetAsync(ws.x_e.p, 0, ws.x_e.bytes, st));
        LQCD_CUDA(cudaMemsetAsync(ws.e.p, 0, ws.e.bytes, st));
        LQCD_CUDA(cudaMemsetAsync(ws.p.p, 0, ws.p.bytes, st));
        if (ws.p_sc.p) LQCD_CUDA(cudaMemsetAsync(ws.p_sc.p, 0, ws.p_sc.bytes, st));
    }

    // x += scale e; rhat = bhat - Dhat x (FP64); r = rhat / scale   [gate UPDATE]
    void reliable_update()
    {
        launch_x_update<E>(gated(ST_UPDATE, RED_STORE), S, e, x_e, st);
        HopArgs<F64, F64, F64> a = h64;
        a.gate_st = S;
        a.gate = ST_UPDATE;
        a.nactive = hint_update;
        a.parity = 1;
        a.in = x_e;
        a.out = t64;
        a.clov = ai64;
        a.coef = kappa;
        launch_hop(a, HOP_CLOV, false, false, st);
        a.parity = 0;
        a.in = t64;
        a.self = x_e;
        a.out = w64;
        a.clov = a64;
        a.coef = -kappa;
        launch_hop(a, SELF_CLOV, false, false, st);
        launch_r_replace<W, F64>(gated(ST_UPDATE, RED_RHAT), bhat, w64, r, x_o, false, st);
    }

    // Incremental update (mixed solvers): the residual moves from the last
    // recomputed rhat (FP64, kept in x_o, which holds nothing else until the
    // odd solution is rebuilt at the end) by the correction gathered since:
    //   rhat <- rhat - scale Dhat e,   x += scale e,   r = rhat / scale,
    // with Dhat e evaluated by the FP32 kernel in its scalar shape (untuned, so the
    // bits of a solve do not depend on the tuner) straight from e (FP32).
    // Each step adds an error of order 1e-7 |Dhat| |scale e|, i.e. a small
    // multiple of 1e-7 of the residual it starts from, so the error since the
    // last FP64 residual (the anchor) stays of order 1e-7 |anchor|.  It is
    // used while every RHS asking for an update has |rhat| >= kTau |anchor|
    // and >= kTolFactor tol |b|, and never declares convergence
    // (RED_RHAT_COARSE); the updates that can finish and the final true
    // residual are FP64.  t64 and w64 hold the FP32 intermediate and Dhat e.
    static constexpr double kTau = 1e-4;
    static constexpr double kTolFactor = 3.0;
    void reliable_update_incremental()
    {
        if constexpr (std::is_same<E, F32>::value) {
            const long Sd = lat->stride;
            SpinorField<F32> t32{ws.t64.as<float4>(), nullptr, Sd};
            SpinorField<F32> w32{ws.w64.as<float4>(), nullptr, Sd};
            HopArgs<F32, F32, F32> a = h32;
            a.gate_st = S;
            a.gate = ST_UPDATE;
            a.nactive = hint_update;
            a.fixed_shape = true;  // the solve's bits must not depend on the tuner's FP32 choice
            a.parity = 1;
            a.in = e;
            a.out = t32;
            a.clov = ai32;
            a.coef = kappa;
            launch_hop(a, HOP_CLOV, false, false, st);
            a.parity = 0;
            a.in = t32;
            a.self = e;
            a.out = w32;
            a.clov = a32;
            a.coef = -kappa;
            launch_hop(a, SELF_CLOV, false, false, st);
            launch_x_update<E>(gated(ST_UPDATE, RED_STORE), S, e, x_e, st);
            launch_r_replace<W, F32>(gated(ST_UPDATE, RED_RHAT_COARSE), x_o, w32, r, x_o, true, st);
        } else {
            reliable_update();
        }
    }

    // every RHS asking for an update allows the incremental one (host view after a poll)
    bool incremental_ok() const
    {
        if (!std::is_same<E, F32>::value) return false;
        const double lim2 = kTolFactor * kTolFactor * tol_ * tol_;
        for (int j = 0; j < nrhs; ++j) {
            const RhsState &q = ws.host_state[j];
            if (q.status != ST_UPDATE) continue;
            if (q.iter >= q.maxiter || !(q.rr == q.rr)) return false;
            const double r2 = q.rr * q.scale * q.scale;
            if (r2 < kTau * kTau * q.anchor2 || r2 < lim2 * q.bnorm2) return false;
        }
        return true;
    }

    // the cheapest residual recomputation every RHS asking for one allows
    // (host view after a poll)
    void update_best()
    {
        if (incremental_ok())
            reliable_update_incremental();
        else
            reliable_update();
    }

    // w = Dhat p (|w|^2 -> alpha); e += alpha p; r -= alpha w   [gate ACTIVE]
    void half1()
    {
        HopArgs<W, W, W> a = hw;
        a.gate_st = S;
        a.gate = ST_ACTIVE;
        a.nactive = hint_active;
        a.parity = 1;
        a.in = p;
        a.out = t;
        a.clov = aiw;
        a.coef = kappa;
        launch_hop(a, HOP_CLOV, false, false, st);
        a.parity = 0;
        a.in = t;
        a.self = p;
        a.out = w;
        a.clov = aw;
        a.coef = -kappa;
        a.red.op = RED_ALPHA;
        launch_hop(a, SELF_CLOV, false, true, st);
        launch_er_update<W, E>(gated(ST_ACTIVE, RED_RUPDATE), p, w, r, e, st);
    }

    // z = Dhat^dag r (|z|^2 -> beta, gamma); p = z + beta p   [gate ACTIVE or RESUME]
    void half2(int gate = ST_ACTIVE)
    {
        HopArgs<W, W, W> a = hw;
        a.gate_st = S;
        a.gate = gate;
        a.nactive = hint(gate);
        a.parity = 1;
        a.in = r;
        a.out = t;
        a.clov = aiw;
        a.coef = kappa;
        launch_hop(a, HOP_CLOV, true, false, st);
        a.parity = 0;
        a.in = t;
        a.self = r;
        a.out = z;
        a.clov = aw;
        a.coef = -kappa;
        a.red.op = RED_BETA;
        launch_hop(a, SELF_CLOV, true, true, st);
        launch_p_update<W>(gated(gate, RED_STORE), S, z, p, st);
    }

    void set_resume(int v)
    {
        set_resume_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(S, nrhs, v);
        LQCD_CHECK_LAUNCH();
    }

    // right-hand sides just updated in FP64 finish their iteration, then rejoin
    void resumed_to_active()
    {
        half2(ST_RESUME);
        status_change_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(S, nrhs, ST_RESUME, ST_ACTIVE);
        LQCD_CHECK_LAUNCH();
    }

    // x_o = A_oo^-1 (b_o + k H_oe x_e); acc = |b - D x|^2 over both parities
    void finish()
    {
        HopArgs<F64, F64, F64> a = h64;
        a.parity = 1;
        a.in = x_e;
        a.self = b_o;
        a.out = x_o;
        a.clov = ai64;
        a.coef = kappa;
        launch_hop(a, CLOV_SUM, false, false, st);
        a.parity = 0;
        a.in = x_o;
        a.self = x_e;
        a.b = b_e;
        a.clov = a64;
        a.coef = -kappa;
        a.red.op = RED_STORE;
        launch_hop(a, RESID, false, true, st);
        a.parity = 1;
        a.in = x_e;
        a.self = x_o;
        a.b = b_o;
        a.red.op = RED_ADD;
        launch_hop(a, RESID, false, true, st);
    }

    // w = Dhat p (or Dhat^dag p), no reductions, every RHS
    void apply_schur(bool dag)
    {
        HopArgs<W, W, W> a = hw;
        a.parity = 1;
        a.in = p;
        a.out = t;
        a.clov = aiw;
        a.coef = kappa;
        launch_hop(a, HOP_CLOV, dag, false, st);
        a.parity = 0;
        a.in = t;
        a.self = p;
        a.out = w;
        a.clov = aw;
        a.coef = -kappa;
        launch_hop(a, SELF_CLOV, dag, false, st);
    }

    void pull_states()
    {
        LQCD_CUDA(cudaMemcpyAsync(ws.host_state, S, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost, st));
        LQCD_CUDA(cudaStreamSynchronize(st));
        // an RHS updated in FP64 next resumes the inner iteration (or is done)
        int act = 0, upd = 0;
        for (int j = 0; j < nrhs; ++j) {
            act += ws.host_state[j].status == ST_ACTIVE || ws.host_state[j].status == ST_UPDATE;
            upd += ws.host_state[j].status == ST_UPDATE;
        }
        hint_active = act;
        hint_update = upd;
    }

    void push_states()
    {
        LQCD_CUDA(cudaMemcpyAsync(S, ws.host_state, sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, st));
    }

    bool any_status(int st_) const
    {
        for (int j = 0; j < nrhs; ++j)
            if (ws.host_state[j].status == st_) return true;
        return false;
    }

    bool all_finished() const
    {
        for (int j = 0; j < nrhs; ++j) {
            int s = ws.host_state[j].status;
            if (s == ST_ACTIVE || s == ST_UPDATE) return false;
        }
        return true;
    }

    const volatile bool *cancel = nullptr;  // set by the server: stop at the next poll

    double tol_ = 0, delta_ = 0;

    // |b|, bhat, the FP64 residual of the start (zero, or the guess already
    // in x_e) and the first z, p
    void start(const lqcd_solver_params &sp, bool guess = false)
    {
        // default reliable-update factor per inner format (measured at
        // 32^3 x 64): FP16 residuals drift, so they are refreshed every
        // decade; FP32 ones hold until 5e-3
        const double delta_default = std::is_same<W, F16>::value ? 0.1 : 0.005;
        delta_ = std::is_same<W, F64>::value ? 1e-30 : (sp.inner_tol > 0 ? sp.inner_tol : delta_default);
        tol_ = sp.tol;
        prepare(0.5 * tol_, delta_, sp.maxiter, guess);
        if (guess)
            reliable_update();
        else  // from x = 0 the first residual is bhat itself (x_e holds zeros)
            launch_r_replace<W, F64>(gated(ST_UPDATE, RED_RHAT), bhat, x_e, r, x_o, false, st);
        half2();
    }

    // Iterates until every RHS is done or capped.  Large batches: read the
    // states after every half-iteration and launch the FP64 update only when
    // some RHS asked for it (a gated-off launch of the FP64 kernels still
    // schedules every block; the host round trip costs ~15 us against
    // milliseconds of work).  Small batches: gated launches are cheap, so
    // poll every few iterations only.
    static constexpr int kGraphChunk = 8;  // iterations per poll of small batches
    void iterate(const lqcd_solver_params &sp)
    {
        const bool small = long(lat->vh) * nrhs < (1L << 20);
        if (small && !cancel) {
            iterate_graph(sp);
            return;
        }
        long guard = (long)sp.maxiter + 64;
        if (small) {
            // the serving loop's slots (cancel set) share the device with other
            // host threads and do not capture graphs: chunks of 8 eager
            // iterations, the (gated) FP64 update after every half 1, one poll
            // per chunk
            bool finished = false;
            for (long it = 0; it < guard && !finished && !(cancel && *cancel); it += kGraphChunk) {
                hint_active = hint_update = -1;  // statuses change unseen inside a chunk
                for (int k = 0; k < kGraphChunk; ++k) {
                    half1();
                    reliable_update();
                    half2();
                }
                pull_states();
                finished = all_finished();
            }
            return;
        }
        for (long it = 0; it < guard && !(cancel && *cancel); ++it) {
            half1();
            pull_states();
            if (all_finished()) break;
            if (any_status(ST_UPDATE)) update_best();
            half2();
        }
    }

    // Small batches, where launch latency dominates: chunks of kGraphChunk
    // iterations replayed from one CUDA graph.  Inside a chunk an RHS that
    // asks for a residual update pauses (its kernels are gated off); after the
    // chunk the host runs the update and the paused RHS finish their
    // iteration (ST_RESUME) before the next replay.  One eager iteration
    // first, so every kernel shape is autotuned outside the capture.
    void iterate_graph(const lqcd_solver_params &sp)
    {
        // the legacy default stream cannot be captured: run on a stream of our
        // own, ordered after and before the caller's by events
        if (st == nullptr || st == cudaStreamLegacy) {
            cudaStream_t orig = st, own = nullptr;
            cudaEvent_t ev = nullptr;
            LQCD_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
            auto restore = [&]() {
                st = orig;
                if (ev) cudaEventDestroy(ev);
                if (own) cudaStreamDestroy(own);
            };
            try {
                LQCD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
                LQCD_CUDA(cudaEventRecord(ev, orig));
                LQCD_CUDA(cudaStreamWaitEvent(own, ev, 0));
                st = own;
                iterate_graph(sp);
                LQCD_CUDA(cudaEventRecord(ev, own));
                LQCD_CUDA(cudaStreamWaitEvent(orig, ev, 0));
            } catch (...) {
                cudaStreamSynchronize(own);
                restore();
                throw;
            }
            restore();
            return;
        }
        half1();
        pull_states();
        if (!all_finished()) {
            if (any_status(ST_UPDATE)) update_best();
            half2();
        }
        set_resume(ST_RESUME);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        auto cleanup = [&]() {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            exec = nullptr;
            graph = nullptr;
        };
        try {
            pull_states();
            const long max_chunks = (long(sp.maxiter) + 64) / kGraphChunk + 2;
            for (long c = 0; c < max_chunks && !all_finished() && !(cancel && *cancel); ++c) {
                if (any_status(ST_UPDATE)) {
                    update_best();
                    resumed_to_active();
                }
                if (!exec) {
                    LQCD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                    try {
                        hint_active = hint_update = -1;  // statuses change unseen inside a chunk
                        for (int k = 0; k < kGraphChunk; ++k) {
                            half1();
                            half2();
                        }
                    } catch (...) {
                        cudaGraph_t g = nullptr;
                        cudaStreamEndCapture(st, &g);
                        if (g) cudaGraphDestroy(g);
                        throw;
                    }
                    LQCD_CUDA(cudaStreamEndCapture(st, &graph));
                    LQCD_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                }
                LQCD_CUDA(cudaGraphLaunch(exec, st));
                pull_states();
            }
            // a last update of RHS that paused in the final chunk
            if (any_status(ST_UPDATE) && !(cancel && *cancel)) {
                update_best();
                resumed_to_active();
                pull_states();
            }
        } catch (...) {
            cleanup();
            throw;
        }
        cleanup();
        set_resume(ST_ACTIVE);
    }

    // x_o, true residuals; RHS whose full-lattice residual misses tol (it
    // can, by rounding, after the reduced system converged) continue with a
    // tighter target.  Returns the number of RHS that did not reach tol.
    int finish_report(const lqcd_solver_params &sp, lqcd_solve_info *info)
    {
        const double tol = tol_;
        for (int attempt = 0; attempt < 4; ++attempt) {
            finish();
            pull_states();
            bool retry = false;
            for (int j = 0; j < nrhs; ++j) {
                RhsState &q = ws.host_state[j];
                double tr = q.bnorm2 > 0 ? std::sqrt(q.acc / q.bnorm2) : 0.0;
                if (q.status == ST_DONE && tr > tol && q.iter < q.maxiter) {
                    q.target2 *= 0.25 * std::min(1.0, tol * tol * q.bnorm2 / std::max(q.acc, 1e-300));
                    q.status = ST_UPDATE;
                    retry = true;
                }
            }
            if (!retry || (cancel && *cancel) || attempt == 3) break;
            push_states();
            reliable_update();
            half2();
            iterate(sp);
        }
        int failed = 0;
        for (int j = 0; j < nrhs; ++j) {
            const RhsState &q = ws.host_state[j];
            double tr = q.bnorm2 > 0 ? std::sqrt(q.acc / q.bnorm2) : 0.0;
            bool ok = (q.status == ST_DONE) && tr <= tol;
            if (!ok) ++failed;
            if (info) {
                info[j].iters_inner = q.iter;
                info[j].iters_outer = std::max(q.updates, 0);
                info[j].true_resid = tr;
                info[j].status = ok ? LQCD_OK : LQCD_ENOCONV;
            }
        }
        return failed;
    }

    // returns the number of RHS that did not reach tol
    int run(const lqcd_solver_params &sp, lqcd_solve_info *info, bool guess)
    {
        start(sp, guess);
        iterate(sp);
        return finish_report(sp, info);
    }
};

template <class W, class E>
static int solve_on_t(lqcd_lattice_s *lat, GaugeSet &g, CloverSet &cl, Workspace &ws, const lqcd_dirac_params &dp,
                      const lqcd_solver_params &sp, const double *b_dev, double *x_dev, const int *src, int nrhs,
                      lqcd_solve_info *info, double *corr_dev, cudaStream_t st, const volatile bool *cancel,
                      bool guess)
{
    Solver<W, E> s(lat, ws, g, cl, dp, nrhs, st);
    s.cancel = cancel;
    if (src)
        point_sources(lat, src, s.b_e, s.b_o, st);
    else
        spinor_to_soa(lat, b_dev, nrhs, s.b_e, s.b_o, st);
    guess = guess && x_dev;
    if (guess) spinor_to_soa(lat, x_dev, nrhs, s.x_e, s.x_o, st);  // only the even part is used
    int failed = s.run(sp, info, guess);
    if (cancel && *cancel) failed = nrhs;
    if (x_dev) spinor_from_soa(lat, x_dev, nrhs, s.x_e, s.x_o, st);
    if (corr_dev)
        pion_contract_soa(lat, s.x_e, s.x_o, src[3], corr_dev, ws.partial.as<double>(), ws.counter.as<unsigned>(), st);
    LQCD_CUDA(cudaStreamSynchronize(st));
    return failed;
}

int solve_on(lqcd_lattice_s *lat, GaugeSet &g, CloverSet &cl, Workspace &ws, const lqcd_dirac_params &dp,
             const lqcd_solver_params &sp, const double *b_dev, double *x_dev, const int *src, int nrhs,
             lqcd_solve_info *info, double *corr_dev, cudaStream_t st, const volatile bool *cancel, bool guess)
{
    switch (sp.precision) {
    case LQCD_PREC_FP64:
        return solve_on_t<F64, F64>(lat, g, cl, ws, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, cancel,
                                    guess);
    case LQCD_PREC_MIXED_FP32:
        return solve_on_t<F32, F32>(lat, g, cl, ws, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, cancel,
                                    guess);
    case LQCD_PREC_MIXED_FP16:
        return solve_on_t<F16, F32>(lat, g, cl, ws, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, cancel,
                                    guess);
    default: throw Error{LQCD_EINVAL, "unknown precision"};
    }
}

template <class W, class E>
static int solve_prec(lqcd_lattice_s *lat, GaugeSet &g, CloverSet &cl, const lqcd_dirac_params &dp,
                      const lqcd_solver_params &sp, const double *b_dev, double *x_dev, const int *src, int nrhs,
                      lqcd_solve_info *info, double *corr_dev, cudaStream_t st, bool guess)
{
    Workspace &ws = workspace<W, E>(lat, nrhs, sp.precision, st);
    return solve_on_t<W, E>(lat, g, cl, ws, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, nullptr, guess);
}

void dirac_apply_dev(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, const double *in, double *out,
                     bool dag, cudaStream_t st)
{
    CloverSet &cl = clover_get(lat, g, dp, st);
    Workspace &ws = workspace<F64, F64>(lat, 1, LQCD_PREC_FP64, st);
    const long Sd = lat->stride;
    SpinorField<F64> ie = fld<F64>(ws.b_e, nullptr, Sd), io = fld<F64>(ws.b_o, nullptr, Sd);
    SpinorField<F64> oe = fld<F64>(ws.x_e, nullptr, Sd), oo = fld<F64>(ws.x_o, nullptr, Sd);
    spinor_to_soa(lat, in, 1, ie, io, st);
    HopArgs<F64, F64, F64> a{};
    a.g = lat->geom;
    a.nrhs = 1;
    a.ntiles = ntiles_of(lat->vh);
    a.U = hop_links<F64>(g, Sd, dp.bc);
    hop_theta(dp, a.th_re, a.th_im);
    a.clov = clover_field<F64>(cl, false, Sd);
    a.tau = cl.tau;
    a.coef = -dp.kappa;
    // (D psi)_p = A_p psi_p - kappa H_{p,1-p} psi_{1-p} on both parities
    a.parity = 0;
    a.in = io;
    a.self = ie;
    a.out = oe;
    launch_hop(a, SELF_CLOV, dag, false, st);
    a.parity = 1;
    a.in = ie;
    a.self = io;
    a.out = oo;
    launch_hop(a, SELF_CLOV, dag, false, st);
    spinor_from_soa(lat, out, 1, oe, oo, st);
}

template <class W, class E>
static void schur_apply_prec(lqcd_lattice_s *lat, GaugeSet &g, CloverSet &cl, const lqcd_dirac_params &dp, int prec,
                             const double *in, double *out, int nrhs, int repeat, bool dag, cudaStream_t st)
{
    Workspace &ws = workspace<W, E>(lat, nrhs, prec, st);
    Solver<W, E> s(lat, ws, g, cl, dp, nrhs, st);
    spinor_to_soa(lat, in, nrhs, s.b_e, s.b_o, st);
    launch_convert<F64, W>(lat->vh, nrhs, s.b_e, s.p, st);
    for (int k = 0; k < repeat; ++k) s.apply_schur(dag);
    launch_convert<W, F64>(lat->vh, nrhs, s.w, s.x_e, st);
    LQCD_CUDA(cudaMemsetAsync(ws.x_o.p, 0, ws.x_o.bytes, st));
    spinor_from_soa(lat, out, nrhs, s.x_e, s.x_o, st);
}

void schur_apply_dev(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, int precision, const double *in,
                     double *out, int nrhs, int repeat, bool dag, cudaStream_t st)
{
    CloverSet &cl = clover_get(lat, g, dp, st);
    switch (precision) {
    case LQCD_PREC_FP64: schur_apply_prec<F64, F64>(lat, g, cl, dp, precision, in, out, nrhs, repeat, dag, st); break;
    case LQCD_PREC_MIXED_FP32:
        schur_apply_prec<F32, F32>(lat, g, cl, dp, precision, in, out, nrhs, repeat, dag, st);
        break;
    case LQCD_PREC_MIXED_FP16:
        schur_apply_prec<F16, F32>(lat, g, cl, dp, precision, in, out, nrhs, repeat, dag, st);
        break;
    default: throw Error{LQCD_EINVAL, "unknown precision"};
    }
}

int solve(lqcd_lattice_s *lat, int gauge_id, const lqcd_dirac_params &dp, const lqcd_solver_params &sp,
          const double *b_dev, double *x_dev, const int *src, int nrhs, lqcd_solve_info *info, double *corr_dev,
          cudaStream_t st, bool guess)
{
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) throw Error{LQCD_EINVAL, "unknown gauge id"};
    GaugeSet &g = *it->second;
    CloverSet &cl = clover_get(lat, g, dp, st);
    switch (sp.precision) {
    case LQCD_PREC_FP64:
        return solve_prec<F64, F64>(lat, g, cl, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, guess);
    case LQCD_PREC_MIXED_FP32:
        return solve_prec<F32, F32>(lat, g, cl, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, guess);
    case LQCD_PREC_MIXED_FP16:
        return solve_prec<F16, F32>(lat, g, cl, dp, sp, b_dev, x_dev, src, nrhs, info, corr_dev, st, guess);
    default: throw Error{LQCD_EINVAL, "unknown precision"};
    }
}

// ---------------------------------------------------------------------------
// Batched propagators on uneven lattices: every job is a 12-column point
// source solve on its own lattice, gauge field and kappa.  After one eager
// iteration (which also autotunes the kernels of every lattice size), the
// iterations of all unfinished jobs are captured into one CUDA graph, one
// branch per job and `chunk` iterations per branch, and that graph is
// launched until every job has finished.  Inside the graph a right-hand side
// that asks for an FP64 residual pauses; between launches the host runs the
// FP64 updates of the jobs that asked and the updated right-hand sides
// finish their iteration (ST_RESUME).  The graph is captured again whenever
// the set of unfinished jobs shrinks.
// ---------------------------------------------------------------------------
template <class W, class E>
struct BatchJob {
    lqcd_pion_job *job = nullptr;
    lqcd_lattice_s *lat = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t join = nullptr;
    std::unique_ptr<Workspace> ws;
    std::unique_ptr<Solver<W, E>> s;
    bool active = true;
    ~BatchJob()
    {
        s.reset();
        ws.reset();
        if (join) cudaEventDestroy(join);
        if (st) cudaStreamDestroy(st);
    }
};

template <class W, class E>
static int batch_t(lqcd_pion_job *jobs, int n, const lqcd_solver_params &sp, int chunk, cudaStream_t origin)
{
    std::vector<std::unique_ptr<BatchJob<W, E>>> J;
    for (int k = 0; k < n; ++k) {
        auto b = std::make_unique<BatchJob<W, E>>();
        b->job = &jobs[k];
        b->lat = jobs[k].lat;
        LQCD_CUDA(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
        LQCD_CUDA(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
        auto it = b->lat->gauges.find(jobs[k].gauge_id);
        if (it == b->lat->gauges.end()) throw Error{LQCD_EINVAL, "unknown gauge id in batch job " + std::to_string(k)};
        GaugeSet &g = *it->second;
        CloverSet &cl = clover_get(b->lat, g, jobs[k].dp, b->st);
        b->ws = workspace_build(b->lat, 12, sp.precision, b->st, false);
        b->s = std::make_unique<Solver<W, E>>(b->lat, *b->ws, g, cl, jobs[k].dp, 12, b->st);
        point_sources(b->lat, jobs[k].src, b->s->b_e, b->s->b_o, b->st);
        b->s->start(sp);
        J.push_back(std::move(b));
    }
    // one eager iteration per job (autotunes the kernels outside any capture)
    for (auto &b : J) {
        b->s->half1();
        b->s->pull_states();
        if (b->s->any_status(ST_UPDATE)) b->s->update_best();
        b->s->half2();
    }
    for (auto &b : J) {
        b->s->set_resume(ST_RESUME);
        LQCD_CUDA(cudaStreamSynchronize(b->st));
    }
    cudaEvent_t fork;
    LQCD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto capture = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        LQCD_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
        LQCD_CUDA(cudaEventRecord(fork, origin));
        for (auto &b : J) {
            if (!b->active) continue;
            b->s->hint_active = b->s->hint_update = -1;  // the graph is replayed as statuses change
            LQCD_CUDA(cudaStreamWaitEvent(b->st, fork, 0));
            for (int k = 0; k < chunk; ++k) {
                b->s->half1();
                b->s->half2();
            }
            LQCD_CUDA(cudaEventRecord(b->join, b->st));
            LQCD_CUDA(cudaStreamWaitEvent(origin, b->join, 0));
        }
        LQCD_CUDA(cudaStreamEndCapture(origin, &graph));
        LQCD_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    };
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaEventDestroy(fork);
    };
    try {
        int nactive = 0;
        for (auto &b : J) {
            b->active = !b->s->all_finished();
            nactive += b->active;
        }
        int captured_for = -1;
        const long max_chunks = (long(sp.maxiter) + 64) / chunk + 2;
        for (long c = 0; c < max_chunks && nactive > 0; ++c) {
            if (captured_for != nactive) {
                capture();
                captured_for = nactive;
            }
            LQCD_CUDA(cudaGraphLaunch(exec, origin));
            LQCD_CUDA(cudaStreamSynchronize(origin));
            for (auto &b : J) {
                if (!b->active) continue;
                b->s->pull_states();
                if (b->s->any_status(ST_UPDATE)) {
                    b->s->update_best();
                    b->s->resumed_to_active();
                }
            }
            nactive = 0;
            for (auto &b : J) {
                if (!b->active) continue;
                b->s->pull_states();
                b->active = !b->s->all_finished();
                nactive += b->active;
            }
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    int failed_jobs = 0;
    for (auto &b : J) {
        b->s->set_resume(ST_ACTIVE);
        const int T = b->lat->dims[3];
        lqcd_pion_job &jb = *b->job;
        int failed = b->s->finish_report(sp, jb.info);
        Workspace &ws = *b->ws;  // w64 is free after the solve: it receives C(t)
        pion_contract_soa(b->lat, b->s->x_e, b->s->x_o, jb.src[3], ws.w64.as<double>(), ws.partial.as<double>(),
                          ws.counter.as<unsigned>(), b->st);
        LQCD_CUDA(cudaMemcpyAsync(jb.corr, ws.w64.p, sizeof(double) * T, cudaMemcpyDeviceToHost, b->st));
        LQCD_CUDA(cudaStreamSynchronize(b->st));
        jb.status = failed ? LQCD_ENOCONV : LQCD_OK;
        failed_jobs += failed != 0;
    }
    return failed_jobs;
}

int pion_batch(lqcd_pion_job *jobs, int n, const lqcd_solver_params &sp, int chunk, cudaStream_t origin)
{
    switch (sp.precision) {
    case LQCD_PREC_FP64: return batch_t<F64, F64>(jobs, n, sp, chunk, origin);
    case LQCD_PREC_MIXED_FP32: return batch_t<F32, F32>(jobs, n, sp, chunk, origin);
    case LQCD_PREC_MIXED_FP16: return batch_t<F16, F32>(jobs, n, sp, chunk, origin);
    default: throw Error{LQCD_EINVAL, "unknown precision"};
    }
}

}  // namespace lqcd
