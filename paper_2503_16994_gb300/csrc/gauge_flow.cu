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

void gauge_flow(lqcd_lattice_s *lat, GaugeSet &g, double eps, int nsteps, cudaStream_t st)
{
    const long S = lat->stride;
    DevBuf X;
    X.ensure(sizeof(double2) * 2 * 4 * 9 * S);
    const dim3 gf(unsigned((lat->vh + 63) / 64), 2, 4), gu(unsigned((lat->vh + 127) / 128), 2, 4);
    // per link: 6 staples of 2 products and a product with the link (~13 3x3 complex products)
    const double fbytes = double(lat->V) * 4 * (7 * 144.0 + 144.0), ubytes = double(lat->V) * 4 * 3 * 144.0;
    double2 *u = g.u64.as<double2>();
    const LinkField<F64> U{u, nullptr, S};
    const double a[3] = {0.25, 8.0 / 9.0, 0.75}, b[3] = {0.0, -17.0 / 9.0, -1.0};
    for (int k = 0; k < nsteps; ++k)
        for (int stage = 0; stage < 3; ++stage) {
            {
                ProfScope prof("flow_force", fbytes, st);
                flow_force_kernel<<<gf, 64, 0, st>>>(lat->geom, U, X.as<double2>(), a[stage] * eps, b[stage]);
                LQCD_CHECK_LAUNCH();
            }
            ProfScope prof("flow_update", ubytes, st);
            flow_update_kernel<<<gu, 128, 0, st>>>(lat->geom, u, X.as<const double2>(), 1.0);
            LQCD_CHECK_LAUNCH();
        }
    const dim3 gr(unsigned((lat->vh + 127) / 128), 8);
    recon_copies_kernel<<<gr, 128, 0, st>>>(lat->geom, g.u64.as<const double2>(), g.u32.as<float4>(),
                                            g.u16.as<uint4>(), g.u16b.as<uint2>());
    LQCD_CHECK_LAUNCH();
    LQCD_CUDA(cudaStreamSynchronize(st));  // X is freed on return
    g.clover.clear();                      // the clover fields belong to the old links
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
