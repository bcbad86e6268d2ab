// Gauge observables and the Wilson flow (Sec. 3.2) on the resident FP64
// links of a gauge field.  One thread per link (flow) or per site
// (observables); FP64 throughout.
//
// Flow generator (the force of the Wilson action summed over oriented
// plaquettes): Z_mu(x) = -(1/2)(Omega - Omega^dag) + (1/6) tr(Omega - Omega^dag)
// with Omega = U_mu(x) S_mu(x), S_mu(x) the sum of the six staples that close
// the plaquettes through the link.  Third-order Runge-Kutta (wfl_rk3) in
// low-storage form, X accumulating the stage combinations:
//   X = eps Z(W0) / 4;               W1 = exp(X) W0
//   X = 8 eps Z(W1) / 9 - 17 X / 9;  W2 = exp(X) W1
//   X = 3 eps Z(W2) / 4 - X;         W3 = exp(X) W2
// (the stage exponents 8 Z1/9 - 17 Z0/36 and 3 Z2/4 - 8 Z1/9 + 17 Z0/36).
#include "gauge_dev.cuh"
#include "lqcd_impl.h"

namespace lqcd {

__device__ __forceinline__ m3 load_m3(const double2 *base, long stride, long cb)
{
    m3 r;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 w = base[k * stride + cb];
        r.m[k / 3][k % 3] = cd{w.x, w.y};
    }
    return r;
}

__device__ __forceinline__ void store_m3(double2 *base, long stride, long cb, const m3 &m)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) base[k * stride + cb] = make_double2(m.m[k / 3][k % 3].re, m.m[k / 3][k % 3].im);
}

__device__ __forceinline__ m3 madd(const m3 &a, const m3 &b)
{
    m3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = a.m[i][j] + b.m[i][j];
    return r;
}

__device__ m3 flow_generator(const Geom &g, const LinkField<F64> &U, const int x[4], int mu)
{
    m3 S;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S.m[i][j] = cd{0.0, 0.0};
    int xpm[4];
    shift(g, x, mu, +1, xpm);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int xpn[4], xmn[4], xpm_mn[4];
        shift(g, x, nu, +1, xpn);
        shift(g, x, nu, -1, xmn);
        shift(g, xpm, nu, -1, xpm_mn);
        S = madd(S, mm(mm(link_xy(g, U, xpm, nu, false), md(link_xy(g, U, xpn, mu, false))),
                       md(link_xy(g, U, x, nu, false))));
        S = madd(S, mm(mm(md(link_xy(g, U, xpm_mn, nu, false)), md(link_xy(g, U, xmn, mu, false))),
                       link_xy(g, U, xmn, nu, false)));
    }
    const m3 om = mm(link_xy(g, U, x, mu, false), S);
    m3 Z;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Z.m[i][j] = -0.5 * (om.m[i][j] - conj(om.m[j][i]));
    const cd tr = (1.0 / 3.0) * (Z.m[0][0] + Z.m[1][1] + Z.m[2][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) Z.m[i][i] = Z.m[i][i] - tr;
    return Z;
}

// X_mu(x) = a Z_mu(x) + b X_mu(x) for every link (b = 0: X not read)
__global__ void __launch_bounds__(64) flow_force_kernel(Geom g, LinkField<F64> U, double2 *X, double a, double b)
{
    const long cb = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int p = blockIdx.y, mu = blockIdx.z;
    if (cb >= g.vh) return;
    int x[4];
    cb_coords(g, p, int(cb), x);
    const m3 Z = flow_generator(g, U, x, mu);
    double2 *xb = X + (long)(p * 4 + mu) * 9 * g.stride;
    m3 r;
    if (b != 0.0) {
        const m3 old = load_m3(xb, g.stride, cb);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) r.m[i][j] = a * Z.m[i][j] + b * old.m[i][j];
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) r.m[i][j] = a * Z.m[i][j];
    }
    store_m3(xb, g.stride, cb, r);
}

// exp(X) by scaling and squaring of a degree-16 Taylor polynomial (Horner
// form): X / 2^s has a row-sum norm <= 1/4, where the truncated terms are
// below 1e-25 of the sum
__device__ m3 expm3(const m3 &X)
{
    double n = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) r += sqrt(norm2(X.m[i][j]));
        n = fmax(n, r);
    }
    int s = 0;
    while (n > 0.25 && s < 60) {
        n *= 0.5;
        ++s;
    }
    const double sc = ldexp(1.0, -s);
    m3 Y, E;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Y.m[i][j] = sc * X.m[i][j];
            E.m[i][j] = cd{i == j ? 1.0 : 0.0, 0.0};
        }
    for (int k = 16; k >= 1; --k) {  // E = 1 + Y E / k
        const m3 YE = mm(Y, E);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) E.m[i][j] = cd{i == j ? 1.0 : 0.0, 0.0} + (1.0 / k) * YE.m[i][j];
    }
    for (int k = 0; k < s; ++k) E = mm(E, E);
    return E;
}

// U_mu(x) <- exp(s X_mu(x)) U_mu(x)
__global__ void __launch_bounds__(128) flow_update_kernel(Geom g, double2 *u64, const double2 *X, double s)
{
    const long cb = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int p = blockIdx.y, mu = blockIdx.z;
    if (cb >= g.vh) return;
    double2 *ub = u64 + (long)(p * 4 + mu) * 9 * g.stride;
    const double2 *xb = X + (long)(p * 4 + mu) * 9 * g.stride;
    m3 x = load_m3(xb, g.stride, cb);
    if (s != 1.0)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) x.m[i][j] = s * x.m[i][j];
    store_m3(ub, g.stride, cb, mm(expm3(x), load_m3(ub, g.stride, cb)));
}

// HMC momenta: P_mu(x) = sum_a pi_a i lambda_a / 2 from the caller's
// coordinates pi (host layout [site][mu][8], on the device)
__global__ void __launch_bounds__(128) momenta_kernel(Geom g, long V, const double *pi, double2 *P)
{
    const long s = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V) return;
    long r = s;
    int x[4];
    x[0] = int(r % g.L[0]);
    r /= g.L[0];
    x[1] = int(r % g.L[1]);
    r /= g.L[1];
    x[2] = int(r % g.L[2]);
    x[3] = int(r / g.L[2]);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const long cb = s >> 1;
    const double r3 = 0.57735026918962576451;  // 1 / sqrt 3
    for (int mu = 0; mu < 4; ++mu) {
        const double *a = pi + (s * 4 + mu) * 8;
        m3 M;
        // i lambda_1..8 / 2 weighted by a[0..7]
        M.m[0][0] = cd{0.0, 0.5 * (a[2] + r3 * a[7])};
        M.m[1][1] = cd{0.0, 0.5 * (-a[2] + r3 * a[7])};
        M.m[2][2] = cd{0.0, -r3 * a[7]};
        M.m[0][1] = cd{0.5 * a[1], 0.5 * a[0]};
        M.m[1][0] = cd{-0.5 * a[1], 0.5 * a[0]};
        M.m[0][2] = cd{0.5 * a[4], 0.5 * a[3]};
        M.m[2][0] = cd{-0.5 * a[4], 0.5 * a[3]};
        M.m[1][2] = cd{0.5 * a[6], 0.5 * a[5]};
        M.m[2][1] = cd{-0.5 * a[6], 0.5 * a[5]};
        store_m3(P + (long)(p * 4 + mu) * 9 * g.stride, g.stride, cb, M);
    }
}

// partial[block] = sum over the block's links of -tr P^2 (one thread per link)
__global__ void __launch_bounds__(128) kinetic_kernel(Geom g, const double2 *P, double *partial)
{
    __shared__ double sh[32];
    const long cb = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;  // parity * 4 + mu
    double v = 0.0;
    if (cb < g.vh) {
        const m3 M = load_m3(P + (long)q * 9 * g.stride, g.stride, cb);
        const m3 MM = mm(M, M);
        v = -(MM.m[0][0].re + MM.m[1][1].re + MM.m[2][2].re);
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) partial[(long)q * gridDim.x + blockIdx.x] = v;
}

// out[0] = sum of the n partials in a fixed order (one block)
__global__ void __launch_bounds__(512) sum_partials_kernel(const double *partial, long n, double *out)
{
    __shared__ double sh[32];
    double t = 0.0;
    for (long k = threadIdx.x; k < n; k += blockDim.x) t += partial[k];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) out[0] = t;
}

// FP32 / FP16 reconstruct-12 copies from the FP64 links (after the flow)
__global__ void __launch_bounds__(128) recon_copies_kernel(Geom g, const double2 *u64, float4 *u32, uint4 *u16,
                                                           uint2 *u16b)
{
    const long cb = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;  // parity * 4 + mu
    if (cb >= g.vh) return;
    double m[18];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 w = u64[((long)q * 9 + k) * g.stride + cb];
        m[2 * k] = w.x;
        m[2 * k + 1] = w.y;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        u32[((long)q * 3 + k) * g.stride + cb] =
            make_float4(float(m[4 * k]), float(m[4 * k + 1]), float(m[4 * k + 2]), float(m[4 * k + 3]));
    uint4 w;
    __half2 *h = reinterpret_cast<__half2 *>(&w);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(float(m[2 * k]), float(m[2 * k + 1]));
    u16[(long)q * g.stride + cb] = w;
    uint2 w2;
    __half2 *h2 = reinterpret_cast<__half2 *>(&w2);
#pragma unroll
    for (int k = 0; k < 2; ++k) h2[k] = __floats2half2_rn(float(m[8 + 2 * k]), float(m[9 + 2 * k]));
    u16b[(long)q * g.stride + cb] = w2;
}

// Gauge observables per time slice (Sec. 3.2; plaquette, Eoft_plaq,
// Eoft_clover, Qtop): thread = site of slice t (lexicographic within the
// slice), sums over the slice by slice_finish into
//   out[0 T + t]: sum Re tr U_p / 3 over the 6 planes,
//   out[1 T + t]: 2 sum_{mu<nu} Re tr (1 - U_p)            (plaquette action density),
//   out[2 T + t]: - sum_{mu<nu} tr F_{mu nu}^2              (clover action density),
//   out[3 T + t]: -(8 / 32 pi^2) [tr F_xy F_zt - tr F_xz F_yt + tr F_xt F_yz]  (clover charge density).
__global__ void __launch_bounds__(128) gauge_obs_kernel(Geom g, LinkField<F64> U, double *partial,
                                                        unsigned *counter, double *out)
{
    const int t = blockIdx.y, c = blockIdx.x, nchunk = gridDim.x;
    const int T = g.L[3];
    const long v3 = long(g.L[0]) * g.L[1] * g.L[2];
    const long k = long(c) * blockDim.x + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < v3) {
        int x[4];
        long r = k;
        x[0] = int(r % g.L[0]);
        r /= g.L[0];
        x[1] = int(r % g.L[1]);
        x[2] = int(r / g.L[1]);
        x[3] = t;
        const int planes[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
        m3 F[6];
        for (int q = 0; q < 6; ++q) {
            const int mu = planes[q][0], nu = planes[q][1];
            int xpm[4], xpn[4];
            shift(g, x, mu, +1, xpm);
            shift(g, x, nu, +1, xpn);
            const m3 P = mm(mm(link_xy(g, U, x, mu, false), link_xy(g, U, xpm, nu, false)),
                            mm(md(link_xy(g, U, xpn, mu, false)), md(link_xy(g, U, x, nu, false))));
            const double re = P.m[0][0].re + P.m[1][1].re + P.m[2][2].re;
            v[0] += re / 3.0;
            v[1] += 2.0 * (3.0 - re);
            F[q] = field_strength(g, U, x, mu, nu, false);
            const m3 FF = mm(F[q], F[q]);
            v[2] -= FF.m[0][0].re + FF.m[1][1].re + FF.m[2][2].re;
        }
        const m3 a = mm(F[0], F[5]), b = mm(F[1], F[4]), d = mm(F[2], F[3]);
        const double e = (a.m[0][0].re + a.m[1][1].re + a.m[2][2].re) - (b.m[0][0].re + b.m[1][1].re + b.m[2][2].re) +
                         (d.m[0][0].re + d.m[1][1].re + d.m[2][2].re);
        v[3] = -8.0 * e / (32.0 * 3.14159265358979323846 * 3.14159265358979323846);
    }
    for (int o = 0; o < 4; ++o)
        slice_finish(v[o], t, c, nchunk, T, 0, partial + (long)o * T * nchunk, counter + o * T, out + o * T);
}

// host layout U[site][mu][3][3] from the FP64 SoA links
__global__ void __launch_bounds__(128) gauge_unpack_kernel(Geom g, long V, const double2 *u64, double *U)
{
    const long s = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V) return;
    long r = s;
    int x[4];
    x[0] = int(r % g.L[0]);
    r /= g.L[0];
    x[1] = int(r % g.L[1]);
    r /= g.L[1];
    x[2] = int(r % g.L[2]);
    x[3] = int(r / g.L[2]);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const long cb = s >> 1;
    for (int mu = 0; mu < 4; ++mu) {
        double *m = U + (s * 4 + mu) * 18;
        for (int k = 0; k < 9; ++k) {
            const double2 w = u64[((long)(p * 4 + mu) * 9 + k) * g.stride + cb];
            m[2 * k] = w.x;
            m[2 * k + 1] = w.y;
        }
    }
}

// one stage of the low-storage RK3 step (W_stage -> W_stage+1) of the links
// u (FP64 planes), X the stage accumulator
static void flow_stage(lqcd_lattice_s *lat, double2 *u, double2 *X, int stage, double eps, cudaStream_t st)
{
    const long S = lat->stride;
    const dim3 gf(unsigned((lat->vh + 63) / 64), 2, 4), gu(unsigned((lat->vh + 127) / 128), 2, 4);
    // per link: 6 staples of 2 products and a product with the link (~13 3x3 complex products)
    const double fbytes = double(lat->V) * 4 * (7 * 144.0 + 144.0), ubytes = double(lat->V) * 4 * 3 * 144.0;
    const LinkField<F64> U{u, nullptr, S};
    const double a[3] = {0.25, 8.0 / 9.0, 0.75}, b[3] = {0.0, -17.0 / 9.0, -1.0};
    {
        ProfScope prof("flow_force", fbytes, st);
        flow_force_kernel<<<gf, 64, 0, st>>>(lat->geom, U, X, a[stage] * eps, b[stage]);
        LQCD_CHECK_LAUNCH();
    }
    ProfScope prof("flow_update", ubytes, st);
    flow_update_kernel<<<gu, 128, 0, st>>>(lat->geom, u, X, 1.0);
    LQCD_CHECK_LAUNCH();
}

// the FP32/FP16 copies of the flowed links; the clover fields of the old links are dropped
static void flow_finish(lqcd_lattice_s *lat, GaugeSet &g, cudaStream_t st)
{
    const dim3 gr(unsigned((lat->vh + 127) / 128), 8);
    recon_copies_kernel<<<gr, 128, 0, st>>>(lat->geom, g.u64.as<const double2>(), g.u32.as<float4>(),
                                            g.u16.as<uint4>(), g.u16b.as<uint2>());
    LQCD_CHECK_LAUNCH();
    LQCD_CUDA(cudaStreamSynchronize(st));  // scratch buffers are freed on return
    g.clover.clear();
    g.sf_ready = false;  // the SF hopping links belong to the old links
}

void gauge_flow(lqcd_lattice_s *lat, GaugeSet &g, double eps, int nsteps, cudaStream_t st)
{
    const long S = lat->stride;
    DevBuf X;
    X.ensure(sizeof(double2) * 2 * 4 * 9 * S);
    for (int k = 0; k < nsteps; ++k)
        for (int stage = 0; stage < 3; ++stage) flow_stage(lat, g.u64.as<double2>(), X.as<double2>(), stage, eps, st);
    flow_finish(lat, g, st);
}

// ---------------------------------------------------------------------------
// Fermion flow: d chi/dt = Delta chi with the covariant Laplacian
//   (Delta chi)(x) = sum_mu [U~_mu(x) chi(x+mu) + U~_mu(x-mu)^dag chi(x-mu) - 2 chi(x)]
// (colour only; U~ carries the boundary phases theta), the links flowed
// alongside.  Third-order scheme on the gauge stages W0, W1, W2 of a step:
//   lambda1 = chi + eps/4 Delta(W0) chi
//   lambda2 = chi + 8 eps/9 Delta(W1) lambda1 - 2 eps/9 Delta(W0) chi
//   chi'    = lambda1 + 3 eps/4 Delta(W2) lambda2
// With Delta(W0) chi = 4 (lambda1 - chi) / eps and H the hopping sum this is
//   lambda1 = eps/4 H chi + (1 - 2 eps) chi
//   lambda2 = 8 eps/9 H lambda1 - 8/9 (1 + 8 eps) lambda1 + 17/9 chi
//   chi'    = 3 eps/4 H lambda2 - 6 eps lambda2 + lambda1
// so each stage is one pass per parity of
//   out(x) = cH H in (x) + c0 in(x) + c1 a1(x).
// ---------------------------------------------------------------------------
struct Phases {
    double re[4], im[4];
};

__global__ void __launch_bounds__(128) laplace_kernel(Geom g, int p, LinkField<F64> U, Phases th,
                                                      SpinorField<F64> self, SpinorField<F64> other,
                                                      SpinorField<F64> a1, SpinorField<F64> a2, SpinorField<F64> out,
                                                      int nrhs, double cH, double c0, double c1, double c2)
{
    const int j = blockIdx.x % nrhs, tile = blockIdx.x / nrhs;
    const int cb = tile * blockDim.x + threadIdx.x;
    if (cb >= g.vh) return;
    int x[4];
    cb_coords(g, p, cb, x);
    spinor<double> acc;
    zero(acc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int y[4];
        shift(g, x, mu, +1, y);
        int ycb = cb_index(g, y);
        const su3<double> Uf = load_link<F64, double>(U, p, mu, cb);
        spinor<double> v = load_spinor<F64, double>(other, j, ycb);
        cx<double> ph = x[mu] == g.L[mu] - 1 ? cx<double>{th.re[mu], th.im[mu]} : cx<double>{1.0, 0.0};
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc.s[s][a] = acc.s[s][a] + ph * (Uf.m[a][0] * v.s[s][0] + Uf.m[a][1] * v.s[s][1] + Uf.m[a][2] * v.s[s][2]);
        shift(g, x, mu, -1, y);
        ycb = cb_index(g, y);
        const su3<double> Ub = load_link<F64, double>(U, p ^ 1, mu, ycb);
        v = load_spinor<F64, double>(other, j, ycb);
        ph = x[mu] == 0 ? cx<double>{th.re[mu], -th.im[mu]} : cx<double>{1.0, 0.0};
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc.s[s][a] = acc.s[s][a] + ph * (cmul(Ub.m[0][a], v.s[s][0]) + cmul(Ub.m[1][a], v.s[s][1]) +
                                                   cmul(Ub.m[2][a], v.s[s][2]));
    }
    const spinor<double> sv = load_spinor<F64, double>(self, j, cb);
    spinor<double> res;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) res.s[s][a] = cH * acc.s[s][a] + c0 * sv.s[s][a];
    if (a1.p) {
        const spinor<double> av = load_spinor<F64, double>(a1, j, cb);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) res.s[s][a] = res.s[s][a] + c1 * av.s[s][a];
    }
    if (a2.p) {
        const spinor<double> av = load_spinor<F64, double>(a2, j, cb);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) res.s[s][a] = res.s[s][a] + c2 * av.s[s][a];
    }
    store_spinor<F64, double>(out, j, cb, res);
}

// backflow combination: u = eta + z1; w = a u - c z2 (one parity, every RHS)
__global__ void __launch_bounds__(128) backflow_combine_kernel(long vh, int nrhs, SpinorField<F64> eta,
                                                               SpinorField<F64> z1, SpinorField<F64> z2,
                                                               SpinorField<F64> u, SpinorField<F64> w, double a,
                                                               double c)
{
    const int j = blockIdx.x % nrhs, tile = blockIdx.x / nrhs;
    const int cb = tile * blockDim.x + threadIdx.x;
    if (cb >= vh) return;
    const spinor<double> e = load_spinor<F64, double>(eta, j, cb), p1 = load_spinor<F64, double>(z1, j, cb),
                         p2 = load_spinor<F64, double>(z2, j, cb);
    spinor<double> uu, ww;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uu.s[s][k] = e.s[s][k] + p1.s[s][k];
            ww.s[s][k] = a * uu.s[s][k] - c * p2.s[s][k];
        }
    store_spinor<F64, double>(u, j, cb, uu);
    store_spinor<F64, double>(w, j, cb, ww);
}

namespace {
// a full-lattice FP64 field: even and odd halves of nrhs right-hand sides
struct Full {
    SpinorField<F64> e, o;
    const SpinorField<F64> &half(int p) const { return p ? o : e; }
};

Full full_of(DevBuf &b, long stride, int nrhs)
{
    double2 *p = b.as<double2>();
    const long half = (long)12 * stride * nrhs;
    return Full{SpinorField<F64>{p, nullptr, stride}, SpinorField<F64>{p + half, nullptr, stride}};
}
}  // namespace

// out = cH H in + c0 in + c1 a1 + c2 a2 on both parities (in != out; a1, a2 may be null)
static void laplace_stage(lqcd_lattice_s *lat, const LinkField<F64> &U, const Phases &th, const Full &in,
                          const Full *a1, const Full &out, int nrhs, double cH, double c0, double c1, cudaStream_t st,
                          const Full *a2 = nullptr, double c2 = 0.0)
{
    // per output site and RHS: the spinor at 8 neighbours and itself (+ a1, a2), the output; 8 links per site
    const double bytes = double(lat->vh) * (nrhs * 192.0 * (2.0 + (a1 ? 1.0 : 0.0) + (a2 ? 1.0 : 0.0)) + 8 * 144.0);
    for (int p = 0; p < 2; ++p) {
        ProfScope prof("fermion_flow_laplace", bytes, st);
        laplace_kernel<<<unsigned(ntiles_of(lat->vh) * nrhs), kBlock, 0, st>>>(
            lat->geom, p, U, th, in.half(p), in.half(p ^ 1), a1 ? a1->half(p) : SpinorField<F64>{},
            a2 ? a2->half(p) : SpinorField<F64>{}, out.half(p), nrhs, cH, c0, c1, c2);
        LQCD_CHECK_LAUNCH();
    }
}

void fermion_flow(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, double *psi_dev, int nrhs,
                  double eps, int nsteps, cudaStream_t st)
{
    const long S = lat->stride;
    const size_t fb = sizeof(double2) * 2 * 12 * (size_t)S * nrhs;
    DevBuf X, bchi, bl1, bl2;
    X.ensure(sizeof(double2) * 2 * 4 * 9 * S);
    bchi.ensure(fb);
    bl1.ensure(fb);
    bl2.ensure(fb);
    const Full chi = full_of(bchi, S, nrhs), l1 = full_of(bl1, S, nrhs), l2 = full_of(bl2, S, nrhs);
    Phases th;
    hop_theta(dp, th.re, th.im);
    const LinkField<F64> U{g.u64.as<const double2>(), nullptr, S};
    spinor_to_soa(lat, psi_dev, nrhs, chi.e, chi.o, st);
    for (int k = 0; k < nsteps; ++k) {
        laplace_stage(lat, U, th, chi, nullptr, l1, nrhs, 0.25 * eps, 1.0 - 2.0 * eps, 0.0, st);  // W0
        flow_stage(lat, g.u64.as<double2>(), X.as<double2>(), 0, eps, st);
        laplace_stage(lat, U, th, l1, &chi, l2, nrhs, 8.0 / 9.0 * eps, -8.0 / 9.0 * (1.0 + 8.0 * eps), 17.0 / 9.0,
                      st);  // W1
        flow_stage(lat, g.u64.as<double2>(), X.as<double2>(), 1, eps, st);
        laplace_stage(lat, U, th, l2, &l1, chi, nrhs, 0.75 * eps, -6.0 * eps, 1.0, st);  // W2
        flow_stage(lat, g.u64.as<double2>(), X.as<double2>(), 2, eps, st);
    }
    spinor_from_soa(lat, psi_dev, nrhs, chi.e, chi.o, st);
    flow_finish(lat, g, st);
}

// S = (beta / 6) sum_t Eplaq[t] from the observables kernel (host value)
static double wilson_action(lqcd_lattice_s *lat, GaugeSet &g, double beta, double *out_dev, cudaStream_t st)
{
    const int T = lat->dims[3];
    gauge_observables(lat, g, out_dev, st);
    std::vector<double> h(T);
    LQCD_CUDA(cudaMemcpyAsync(h.data(), out_dev + T, sizeof(double) * T, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += h[t];
    return beta / 6.0 * s;
}

static double kinetic_energy(lqcd_lattice_s *lat, const double2 *P, double *scratch, cudaStream_t st)
{
    const unsigned nb = unsigned((lat->vh + 127) / 128);
    kinetic_kernel<<<dim3(nb, 8), 128, 0, st>>>(lat->geom, P, scratch);
    LQCD_CHECK_LAUNCH();
    sum_partials_kernel<<<1, 512, 0, st>>>(scratch, long(nb) * 8, scratch + long(nb) * 8);
    LQCD_CHECK_LAUNCH();
    double k = 0.0;
    LQCD_CUDA(cudaMemcpyAsync(&k, scratch + long(nb) * 8, sizeof(double), cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return k;
}

int hmc_trajectory(lqcd_lattice_s *lat, GaugeSet &g, double beta, double eps, int nsteps, const double *mom_dev,
                   double u, double *dH, cudaStream_t st)
{
    const long S = lat->stride;
    const int T = lat->dims[3];
    const size_t ubytes = sizeof(double2) * 2 * 4 * 9 * S;
    DevBuf P, backup, scratch;
    P.ensure(ubytes);
    backup.ensure(ubytes);
    const unsigned nb = unsigned((lat->vh + 127) / 128);
    scratch.ensure(sizeof(double) * std::max<size_t>(4 * T, size_t(nb) * 8 + 1));
    double2 *u64 = g.u64.as<double2>();
    LQCD_CUDA(cudaMemcpyAsync(backup.p, u64, ubytes, cudaMemcpyDeviceToDevice, st));
    momenta_kernel<<<unsigned((lat->V + 127) / 128), 128, 0, st>>>(lat->geom, lat->V, mom_dev, P.as<double2>());
    LQCD_CHECK_LAUNCH();
    const double H0 = kinetic_energy(lat, P.as<const double2>(), scratch.as<double>(), st) +
                      wilson_action(lat, g, beta, scratch.as<double>(), st);
    const dim3 gf(unsigned((lat->vh + 63) / 64), 2, 4), gu(unsigned((lat->vh + 127) / 128), 2, 4);
    const LinkField<F64> U{u64, nullptr, S};
    const double fbytes = double(lat->V) * 4 * (8 * 144.0 + 144.0), lbytes = double(lat->V) * 4 * 3 * 144.0;
    for (int s = 0; s <= nsteps; ++s) {
        const double h = (s == 0 || s == nsteps) ? 0.5 * eps : eps;  // P += h F(U), F = (beta / 6) Z
        {
            ProfScope prof("hmc_force", fbytes, st);
            flow_force_kernel<<<gf, 64, 0, st>>>(lat->geom, U, P.as<double2>(), h * beta / 6.0, 1.0);
            LQCD_CHECK_LAUNCH();
        }
        if (s == nsteps) break;
        ProfScope prof("hmc_links", lbytes, st);  // U = exp(eps P) U
        flow_update_kernel<<<gu, 128, 0, st>>>(lat->geom, u64, P.as<const double2>(), eps);
        LQCD_CHECK_LAUNCH();
    }
    const double H1 = kinetic_energy(lat, P.as<const double2>(), scratch.as<double>(), st) +
                      wilson_action(lat, g, beta, scratch.as<double>(), st);
    *dH = H1 - H0;
    const bool acc = u < std::exp(-*dH);
    if (!acc) LQCD_CUDA(cudaMemcpyAsync(u64, backup.p, ubytes, cudaMemcpyDeviceToDevice, st));
    const dim3 gr(unsigned((lat->vh + 127) / 128), 8);
    recon_copies_kernel<<<gr, 128, 0, st>>>(lat->geom, g.u64.as<const double2>(), g.u32.as<float4>(),
                                            g.u16.as<uint4>(), g.u16b.as<uint2>());
    LQCD_CHECK_LAUNCH();
    LQCD_CUDA(cudaStreamSynchronize(st));
    g.clover.clear();
    g.sf_ready = false;  // the SF hopping links belong to the old links
    return acc ? 1 : 0;
}

void gauge_observables(lqcd_lattice_s *lat, GaugeSet &g, double *out_dev, cudaStream_t st)
{
    const int T = lat->dims[3];
    const long v3 = lat->V / T;
    const int nchunk = int((v3 + kBlock - 1) / kBlock);
    lat->red_partial.ensure(sizeof(double) * 4 * (size_t)T * nchunk);
    if (lat->red_counter.bytes < sizeof(unsigned) * (size_t)std::max(4 * T, 4096)) {
        lat->red_counter.ensure(sizeof(unsigned) * (size_t)std::max(4 * T, 4096));
        LQCD_CUDA(cudaMemsetAsync(lat->red_counter.p, 0, lat->red_counter.bytes, st));
    }
    ProfScope prof("gauge_obs", double(lat->V) * 4 * 144.0, st);
    gauge_obs_kernel<<<dim3(nchunk, T), kBlock, 0, st>>>(lat->geom, link_field<F64>(g, lat->stride),
                                                        lat->red_partial.as<double>(),
                                                        lat->red_counter.as<unsigned>(), out_dev);
    LQCD_CHECK_LAUNCH();
}

void gauge_download(lqcd_lattice_s *lat, GaugeSet &g, double *U_dev, cudaStream_t st)
{
    gauge_unpack_kernel<<<unsigned((lat->V + 127) / 128), 128, 0, st>>>(lat->geom, lat->V, g.u64.as<const double2>(),
                                                                        U_dev);
    LQCD_CHECK_LAUNCH();
}

}  // namespace lqcd

namespace lqcd {

// ---------------------------------------------------------------------------
// Fermion backflow: the exact adjoint of the forward steps above, run over the
// steps in reverse order.  One forward step is chi' = M chi with
//   M = (1 + a D0) + d D2 + d b D2 D1 (1 + a D0) - d c D2 D0,
// a = eps/4, b = 8 eps/9, c = 2 eps/9, d = 3 eps/4, Di = Delta(Wi) (Hermitian),
// so one backward step is
//   z2 = d D2 eta,  z1 = b D1 z2,  u = eta + z1,  w = a u - c z2,
//   eta <- u + z2 + D0 w.
// The gauge field at the start of every step is rebuilt from checkpoints:
// a forward pass keeps the field at the start of every m-th step (m =
// ceil(nsteps / nsave)); each segment of m steps is then flowed again from
// its checkpoint, keeping the start field of each of its steps, and walked
// backwards; the stages W1, W2 of a step are recomputed from its start field.
// The resident links are left at flow time 0.
// ---------------------------------------------------------------------------
void fermion_backflow(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, double *eta_dev, int nrhs,
                      double eps, int nsteps, int nsave, cudaStream_t st)
{
    const long S = lat->stride;
    const size_t ub = sizeof(double2) * 2 * 4 * 9 * (size_t)S;  // one gauge field
    const size_t fb = sizeof(double2) * 2 * 12 * (size_t)S * nrhs;
    const int m = nsteps > 0 ? (nsteps + nsave - 1) / nsave : 1;
    const int nck = nsteps > 0 ? (nsteps + m - 1) / m : 0;
    DevBuf X, ck, seg, w1, w2, be, bz1, bz2, bu, bw;
    X.ensure(ub);
    ck.ensure(ub * std::max(nck, 1));
    seg.ensure(ub * m);
    w1.ensure(ub);
    w2.ensure(ub);
    for (DevBuf *b : {&be, &bz1, &bz2, &bu, &bw}) b->ensure(fb);
    const Full eta = full_of(be, S, nrhs), z1 = full_of(bz1, S, nrhs), z2 = full_of(bz2, S, nrhs),
               u = full_of(bu, S, nrhs), w = full_of(bw, S, nrhs);
    const size_t nlink = ub / sizeof(double2);
    double2 *ckp = ck.as<double2>(), *segp = seg.as<double2>(), *W1 = w1.as<double2>(), *W2 = w2.as<double2>();
    Phases th;
    hop_theta(dp, th.re, th.im);
    spinor_to_soa(lat, eta_dev, nrhs, eta.e, eta.o, st);
    // forward pass: checkpoints at the start of steps 0, m, 2m, ... (w1 is the running field)
    LQCD_CUDA(cudaMemcpyAsync(W1, g.u64.p, ub, cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k < nsteps; ++k) {
        if (k % m == 0) LQCD_CUDA(cudaMemcpyAsync(ckp + (k / m) * nlink, W1, ub, cudaMemcpyDeviceToDevice, st));
        if (k + 1 < nsteps)  // the end field of the last step is not needed
            for (int stage = 0; stage < 3; ++stage) flow_stage(lat, W1, X.as<double2>(), stage, eps, st);
    }
    const double a = 0.25 * eps, b = 8.0 / 9.0 * eps, c = 2.0 / 9.0 * eps, d = 0.75 * eps;
    const unsigned gvec = unsigned(ntiles_of(lat->vh) * nrhs);
    for (int sgi = nck - 1; sgi >= 0; --sgi) {
        const int k0 = sgi * m, k1 = std::min(nsteps, k0 + m);
        // start fields of the steps k0 .. k1-1 of this segment
        LQCD_CUDA(cudaMemcpyAsync(segp, ckp + sgi * nlink, ub, cudaMemcpyDeviceToDevice, st));
        for (int k = k0 + 1; k < k1; ++k) {
            double2 *dst = segp + (k - k0) * nlink;
            LQCD_CUDA(cudaMemcpyAsync(dst, dst - nlink, ub, cudaMemcpyDeviceToDevice, st));
            for (int stage = 0; stage < 3; ++stage) flow_stage(lat, dst, X.as<double2>(), stage, eps, st);
        }
        for (int k = k1 - 1; k >= k0; --k) {
            double2 *W0 = segp + (k - k0) * nlink;
            LQCD_CUDA(cudaMemcpyAsync(W1, W0, ub, cudaMemcpyDeviceToDevice, st));
            flow_stage(lat, W1, X.as<double2>(), 0, eps, st);
            LQCD_CUDA(cudaMemcpyAsync(W2, W1, ub, cudaMemcpyDeviceToDevice, st));
            flow_stage(lat, W2, X.as<double2>(), 1, eps, st);
            const LinkField<F64> U0{W0, nullptr, S}, U1{W1, nullptr, S}, U2{W2, nullptr, S};
            laplace_stage(lat, U2, th, eta, nullptr, z2, nrhs, d, -8.0 * d, 0.0, st);  // z2 = d D2 eta
            laplace_stage(lat, U1, th, z2, nullptr, z1, nrhs, b, -8.0 * b, 0.0, st);   // z1 = b D1 z2
            for (int p = 0; p < 2; ++p) {
                ProfScope prof("fermion_backflow_combine", double(lat->vh) * nrhs * 5 * 192.0, st);
                backflow_combine_kernel<<<gvec, kBlock, 0, st>>>(lat->vh, nrhs, eta.half(p), z1.half(p), z2.half(p),
                                                                 u.half(p), w.half(p), a, c);
                LQCD_CHECK_LAUNCH();
            }
            laplace_stage(lat, U0, th, w, &u, eta, nrhs, 1.0, -8.0, 1.0, st, &z2, 1.0);  // eta = u + z2 + D0 w
        }
    }
    spinor_from_soa(lat, eta_dev, nrhs, eta.e, eta.o, st);
    LQCD_CUDA(cudaStreamSynchronize(st));  // scratch buffers are freed on return
}

}  // namespace lqcd
