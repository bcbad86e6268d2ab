// Gauge-field repacking, clover-field construction and inversion, spinor
// repacking between the host layout and the even-odd SoA layout, point
// sources and the pion contraction.
#include "lqcd_impl.h"

namespace lqcd {

// ---------------------------------------------------------------------------
// layout helpers
// ---------------------------------------------------------------------------
template <>
LinkField<F64> link_field<F64>(const GaugeSet &g, long stride)
{
    return {g.u64.as<const double2>(), nullptr, stride};
}
template <>
LinkField<F32> link_field<F32>(const GaugeSet &g, long stride)
{
    return {g.u32.as<const float4>(), nullptr, stride};
}
template <>
LinkField<F16> link_field<F16>(const GaugeSet &g, long stride)
{
    return {g.u16.as<const uint4>(), g.u16b.as<const uint2>(), stride};
}
template <>
CloverField<F64> clover_field<F64>(const CloverSet &c, bool inv, long stride)
{
    return {(inv ? c.ainv64 : c.a64).as<const double2>(), stride};
}
template <>
CloverField<F32> clover_field<F32>(const CloverSet &c, bool inv, long stride)
{
    return {(inv ? c.ainv32 : c.a32).as<const float4>(), stride};
}
template <>
CloverField<F16> clover_field<F16>(const CloverSet &c, bool inv, long stride)
{
    return {(inv ? c.ainv16 : c.a16).as<const uint4>(), stride};
}

__device__ __forceinline__ void lex_coords(const Geom &g, long s, int x[4])
{
    x[0] = int(s % g.L[0]);
    s /= g.L[0];
    x[1] = int(s % g.L[1]);
    s /= g.L[1];
    x[2] = int(s % g.L[2]);
    x[3] = int(s / g.L[2]);
}

// ---------------------------------------------------------------------------
// gauge field: host layout U[site][mu][3][3] (FP64, on the device) ->
// FP64 full, FP32 and FP16 reconstruct-12 SoA copies
// ---------------------------------------------------------------------------
__global__ void gauge_repack_kernel(Geom g, long V, const double *U, double2 *u64, float4 *u32, uint4 *u16,
                                    uint2 *u16b)
{
    long s = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int x[4];
    lex_coords(g, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const long cb = s >> 1;
    for (int mu = 0; mu < 4; ++mu) {
        const double *m = U + (s * 4 + mu) * 18;
        const long q = p * 4 + mu;
        for (int k = 0; k < 9; ++k) u64[(q * 9 + k) * g.stride + cb] = make_double2(m[2 * k], m[2 * k + 1]);
        for (int k = 0; k < 3; ++k)
            u32[(q * 3 + k) * g.stride + cb] =
                make_float4(float(m[4 * k]), float(m[4 * k + 1]), float(m[4 * k + 2]), float(m[4 * k + 3]));
        uint4 w;
        __half2 *h = reinterpret_cast<__half2 *>(&w);
        for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(float(m[2 * k]), float(m[2 * k + 1]));
        u16[q * g.stride + cb] = w;
        uint2 w2;
        __half2 *h2 = reinterpret_cast<__half2 *>(&w2);
        for (int k = 0; k < 2; ++k) h2[k] = __floats2half2_rn(float(m[8 + 2 * k]), float(m[9 + 2 * k]));
        u16b[q * g.stride + cb] = w2;
    }
}

void gauge_repack(lqcd_lattice_s *lat, GaugeSet &g, const double *U_dev, cudaStream_t st)
{
    const long S = lat->stride;
    g.u64.ensure(sizeof(double2) * 2 * 4 * 9 * S);
    g.u32.ensure(sizeof(float4) * 2 * 4 * 3 * S);
    g.u16.ensure(sizeof(uint4) * 2 * 4 * S);
    g.u16b.ensure(sizeof(uint2) * 2 * 4 * S);
    long nb = (lat->V + kBlock - 1) / kBlock;
    ProfScope prof("gauge_repack", double(lat->V) * (576.0 + 4 * (144.0 + 48.0 + 24.0)), st);
    gauge_repack_kernel<<<unsigned(nb), kBlock, 0, st>>>(lat->geom, lat->V, U_dev, g.u64.as<double2>(),
                                                         g.u32.as<float4>(), g.u16.as<uint4>(), g.u16b.as<uint2>());
    LQCD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// clover field (Csw! of Sec. 3.3)
// ---------------------------------------------------------------------------
using cd = cx<double>;
using m3 = su3<double>;

__device__ __forceinline__ m3 mm(const m3 &a, const m3 &b)
{
    m3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
    return r;
}

__device__ __forceinline__ m3 md(const m3 &a)  // a^dag
{
    m3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

__device__ __forceinline__ m3 link_xy(const Geom &g, const LinkField<F64> &U, const int y[4], int mu)
{
    int p = (y[0] + y[1] + y[2] + y[3]) & 1;
    return load_link<F64, double>(U, p, mu, cb_index(g, y));
}

__device__ __forceinline__ void shift(const Geom &g, const int x[4], int mu, int d, int y[4])
{
    for (int k = 0; k < 4; ++k) y[k] = x[k];
    y[mu] = (y[mu] + d + g.L[mu]) % g.L[mu];
}

// F_{mu nu}(x) = (Q - Q^dag)/8 made traceless, Q = sum of the four leaves
// around x, each leaf walked mu-direction first.
__device__ m3 field_strength(const Geom &g, const LinkField<F64> &U, const int x[4], int mu, int nu)
{
    int xpm[4], xpn[4], xmm[4], xmn[4], a[4], b[4], c[4];
    shift(g, x, mu, +1, xpm);
    shift(g, x, nu, +1, xpn);
    shift(g, x, mu, -1, xmm);
    shift(g, x, nu, -1, xmn);
    shift(g, xmm, nu, +1, a);  // x - mu + nu
    shift(g, xmm, nu, -1, b);  // x - mu - nu
    shift(g, xpm, nu, -1, c);  // x + mu - nu
    m3 Umx = link_xy(g, U, x, mu), Unx = link_xy(g, U, x, nu);
    m3 q = mm(mm(Umx, link_xy(g, U, xpm, nu)), mm(md(link_xy(g, U, xpn, mu)), md(Unx)));
    m3 t = mm(mm(Unx, md(link_xy(g, U, a, mu))), mm(md(link_xy(g, U, xmm, nu)), link_xy(g, U, xmm, mu)));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + t.m[i][j];
    t = mm(mm(md(link_xy(g, U, xmm, mu)), md(link_xy(g, U, b, nu))), mm(link_xy(g, U, b, mu), link_xy(g, U, xmn, nu)));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + t.m[i][j];
    t = mm(mm(md(link_xy(g, U, xmn, nu)), link_xy(g, U, xmn, mu)), mm(link_xy(g, U, c, nu), md(Umx)));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + t.m[i][j];
    m3 f;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f.m[i][j] = 0.125 * (q.m[i][j] - conj(q.m[j][i]));
    cd tr = (1.0 / 3.0) * (f.m[0][0] + f.m[1][1] + f.m[2][2]);
    for (int i = 0; i < 3; ++i) f.m[i][i] = f.m[i][i] - tr;
    return f;
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting.
__device__ void invert6(cd a[6][6], cd inv[6][6])
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) inv[i][j] = cd{i == j ? 1.0 : 0.0, 0.0};
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = norm2(a[c][c]);
        for (int r = c + 1; r < 6; ++r)
            if (norm2(a[r][c]) > best) {
                best = norm2(a[r][c]);
                piv = r;
            }
        if (piv != c)
            for (int j = 0; j < 6; ++j) {
                cd t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
                t = inv[c][j];
                inv[c][j] = inv[piv][j];
                inv[piv][j] = t;
            }
        double n = norm2(a[c][c]);
        cd d = cd{a[c][c].re / n, -a[c][c].im / n};  // 1 / a_cc
        for (int j = 0; j < 6; ++j) {
            a[c][j] = a[c][j] * d;
            inv[c][j] = inv[c][j] * d;
        }
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            cd f = a[r][c];
            for (int j = 0; j < 6; ++j) {
                a[r][j] = a[r][j] - f * a[c][j];
                inv[r][j] = inv[r][j] - f * inv[c][j];
            }
        }
    }
}

__device__ void store_block(double2 *base, long stride, long cb, int off, const cd m[6][6])
{
    // 36 reals: d[6] then the 15 upper entries; as double2 words: reals (2k, 2k+1)
    double v[36];
    for (int i = 0; i < 6; ++i) v[i] = m[i][i].re;
    int q = 6;
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            // Hermitian: average the two triangles to remove rounding asymmetry
            v[q++] = 0.5 * (m[i][j].re + m[j][i].re);
            v[q++] = 0.5 * (m[i][j].im - m[j][i].im);
        }
    for (int k = 0; k < 18; ++k) base[(long)(off + k) * stride + cb] = make_double2(v[2 * k], v[2 * k + 1]);
}

// A_+- = 1 - i kc sum_k s_k (x) (B_k +- E_k), B = (F_yz, F_zx, F_xy), E_k = F_kt:
// in 2x2 spin blocks of 3x3 colour matrices with M_k = B_k +- E_k,
//   A = [[1 - i kc M_z, -i kc (M_x - i M_y)], [-i kc (M_x + i M_y), 1 + i kc M_z]].
__global__ void __launch_bounds__(64) clover_build_kernel(Geom g, LinkField<F64> U, double kc, double2 *a64,
                                                          double2 *ainv64)
{
    const int p = blockIdx.y;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.vh) return;
    int x[4];
    cb_coords(g, p, cb, x);
    m3 Fxy = field_strength(g, U, x, 0, 1), Fxz = field_strength(g, U, x, 0, 2), Fxt = field_strength(g, U, x, 0, 3);
    m3 Fyz = field_strength(g, U, x, 1, 2), Fyt = field_strength(g, U, x, 1, 3), Fzt = field_strength(g, U, x, 2, 3);
    for (int blk = 0; blk < 2; ++blk) {
        const double sg = blk == 0 ? 1.0 : -1.0;
        cd A[6][6], Ai[6][6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                cd Mx = Fyz.m[i][j] + sg * Fxt.m[i][j];
                cd My = (-1.0) * Fxz.m[i][j] + sg * Fyt.m[i][j];
                cd Mz = Fxy.m[i][j] + sg * Fzt.m[i][j];
                cd id = cd{i == j ? 1.0 : 0.0, 0.0};
                A[i][j] = id - kc * mul_i(Mz);
                A[3 + i][3 + j] = id + kc * mul_i(Mz);
                A[i][3 + j] = (-kc) * mul_i(Mx - mul_i(My));
                A[3 + i][j] = (-kc) * mul_i(Mx + mul_i(My));
            }
        store_block(a64 + (long)p * 36 * g.stride, g.stride, cb, 18 * blk, A);
        invert6(A, Ai);
        store_block(ainv64 + (long)p * 36 * g.stride, g.stride, cb, 18 * blk, Ai);
    }
}

// FP64 clover planes -> FP32 / FP16 copies (all parities)
__global__ void clover_convert_kernel(long vh, long stride, const double2 *src, float4 *d32, uint4 *d16)
{
    long cb = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (cb >= vh) return;
    const double2 *s = src + (long)p * 36 * stride + cb;
    double v[72];
    for (int k = 0; k < 36; ++k) {
        double2 w = s[k * stride];
        v[2 * k] = w.x;
        v[2 * k + 1] = w.y;
    }
    for (int k = 0; k < 18; ++k)
        d32[((long)p * 18 + k) * stride + cb] =
            make_float4(float(v[4 * k]), float(v[4 * k + 1]), float(v[4 * k + 2]), float(v[4 * k + 3]));
    for (int k = 0; k < 9; ++k) {
        float f[8];
        for (int q = 0; q < 8; ++q) f[q] = float(v[8 * k + q]);
        d16[((long)p * 9 + k) * stride + cb] = pack_h8(f, 1.0f);
    }
}

size_t clover_bytes(const lqcd_lattice_s *lat)
{
    return 2 * 2 * (size_t)lat->stride * (36 * sizeof(double2) + 18 * sizeof(float4) + 9 * sizeof(uint4));
}

size_t gauge_bytes(const lqcd_lattice_s *lat)
{
    return 2 * 4 * (size_t)lat->stride * (9 * sizeof(double2) + 3 * sizeof(float4) + sizeof(uint4) + sizeof(uint2));
}

std::unique_ptr<CloverSet> clover_build(lqcd_lattice_s *lat, GaugeSet &g, double kappa, double csw, cudaStream_t st,
                                        bool async)
{
    const double kc = kappa * csw;
    auto c = std::make_unique<CloverSet>();
    if (async)
        for (DevBuf *b : {&c->a64, &c->ainv64, &c->a32, &c->ainv32, &c->a16, &c->ainv16}) b->set_async(st);
    const long S = lat->stride;
    c->a64.ensure(sizeof(double2) * 2 * 36 * S);
    c->ainv64.ensure(sizeof(double2) * 2 * 36 * S);
    c->a32.ensure(sizeof(float4) * 2 * 18 * S);
    c->ainv32.ensure(sizeof(float4) * 2 * 18 * S);
    c->a16.ensure(sizeof(uint4) * 2 * 9 * S);
    c->ainv16.ensure(sizeof(uint4) * 2 * 9 * S);
    dim3 grid(unsigned((lat->vh + 63) / 64), 2);
    ProfScope prof("clover_build", double(lat->V) * (4 * 144.0 + 2 * 576.0), st);
    clover_build_kernel<<<grid, 64, 0, st>>>(lat->geom, link_field<F64>(g, S), kc, c->a64.as<double2>(),
                                             c->ainv64.as<double2>());
    LQCD_CHECK_LAUNCH();
    dim3 g2(unsigned((lat->vh + kBlock - 1) / kBlock), 2);
    clover_convert_kernel<<<g2, kBlock, 0, st>>>(lat->vh, S, c->a64.as<const double2>(), c->a32.as<float4>(),
                                                 c->a16.as<uint4>());
    clover_convert_kernel<<<g2, kBlock, 0, st>>>(lat->vh, S, c->ainv64.as<const double2>(), c->ainv32.as<float4>(),
                                                 c->ainv16.as<uint4>());
    LQCD_CHECK_LAUNCH();
    return c;
}

CloverSet &clover_get(lqcd_lattice_s *lat, GaugeSet &g, double kappa, double csw, cudaStream_t st)
{
    const double kc = kappa * csw;
    auto it = g.clover.find(kc);
    if (it != g.clover.end()) return *it->second;
    auto c = clover_build(lat, g, kappa, csw, st, false);
    CloverSet &ref = *c;
    g.clover.emplace(kc, std::move(c));
    return ref;
}

// ---------------------------------------------------------------------------
// spinors: host layout psi[j][site][24] (device) <-> SoA FP64 even/odd
// ---------------------------------------------------------------------------
__global__ void spinor_to_soa_kernel(Geom g, long V, const double *aos, SpinorField<F64> ev, SpinorField<F64> od)
{
    long s = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (s >= V) return;
    int x[4];
    lex_coords(g, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    SpinorField<F64> f = p ? od : ev;
    const double2 *src = reinterpret_cast<const double2 *>(aos + ((long)j * V + s) * 24);
    double2 *dst = f.p + (long)j * 12 * f.stride + (s >> 1);
    for (int k = 0; k < 12; ++k) dst[k * f.stride] = src[k];
}

__global__ void spinor_from_soa_kernel(Geom g, long V, double *aos, SpinorField<F64> ev, SpinorField<F64> od)
{
    long s = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (s >= V) return;
    int x[4];
    lex_coords(g, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    SpinorField<F64> f = p ? od : ev;
    double2 *dst = reinterpret_cast<double2 *>(aos + ((long)j * V + s) * 24);
    const double2 *src = f.p + (long)j * 12 * f.stride + (s >> 1);
    for (int k = 0; k < 12; ++k) dst[k] = src[k * f.stride];
}

void spinor_to_soa(lqcd_lattice_s *lat, const double *aos, int nrhs, SpinorField<F64> even, SpinorField<F64> odd,
                   cudaStream_t st)
{
    dim3 grid(unsigned((lat->V + kBlock - 1) / kBlock), nrhs);
    ProfScope prof("spinor_to_soa", double(lat->V) * nrhs * 2 * 192.0, st);
    spinor_to_soa_kernel<<<grid, kBlock, 0, st>>>(lat->geom, lat->V, aos, even, odd);
    LQCD_CHECK_LAUNCH();
}

void spinor_from_soa(lqcd_lattice_s *lat, double *aos, int nrhs, SpinorField<F64> even, SpinorField<F64> odd,
                     cudaStream_t st)
{
    dim3 grid(unsigned((lat->V + kBlock - 1) / kBlock), nrhs);
    ProfScope prof("spinor_from_soa", double(lat->V) * nrhs * 2 * 192.0, st);
    spinor_from_soa_kernel<<<grid, kBlock, 0, st>>>(lat->geom, lat->V, aos, even, odd);
    LQCD_CHECK_LAUNCH();
}

// eta_j(x) = delta_{x,src} e_j, j = 0..11 (3 spin + colour); fields zeroed first
__global__ void point_source_kernel(SpinorField<F64> f, long cb)
{
    const int j = threadIdx.x;
    if (j < 12) f.p[((long)j * 12 + j) * f.stride + cb] = make_double2(1.0, 0.0);
}

void point_sources(lqcd_lattice_s *lat, const int src[4], SpinorField<F64> even, SpinorField<F64> odd,
                   cudaStream_t st)
{
    LQCD_CUDA(cudaMemsetAsync(even.p, 0, sizeof(double2) * 12 * 12 * even.stride, st));
    LQCD_CUDA(cudaMemsetAsync(odd.p, 0, sizeof(double2) * 12 * 12 * odd.stride, st));
    const int *L = lat->dims;
    long lex = src[0] + (long)L[0] * (src[1] + (long)L[1] * (src[2] + (long)L[2] * src[3]));
    const int p = (src[0] + src[1] + src[2] + src[3]) & 1;
    point_source_kernel<<<1, 32, 0, st>>>(p ? odd : even, lex >> 1);
    LQCD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// pion contraction: corr[(t - src_t) mod T] = sum over the time slice t of
// |S_j|^2 for the 12 columns, FP64.  Blocks (c, t) sum one chunk of slice t
// and the last block of the slice adds the chunks in a fixed order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void slice_finish(double v, int t, int c, int nchunk, int T, int src_t, double *partial,
                                             unsigned *counter, double *corr)
{
    __shared__ double sh[32];
    __shared__ int last;
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) {
        partial[(long)t * nchunk + c] = s;
        __threadfence();
        last = atomicAdd(&counter[t], 1u) == unsigned(nchunk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double a = 0.0;
        for (int k = threadIdx.x; k < nchunk; k += blockDim.x) a += __ldcg(partial + (long)t * nchunk + k);
        a = block_sum(a, sh);
        if (threadIdx.x == 0) {
            counter[t] = 0;
            corr[((t - src_t) % T + T) % T] = a;
        }
    }
}

// SoA columns: slice t of parity p is cb range [t V3h, (t+1) V3h)
__global__ void __launch_bounds__(128) contract_soa_kernel(long v3h, int T, int src_t, SpinorField<F64> ev,
                                                           SpinorField<F64> od, double *partial, unsigned *counter,
                                                           double *corr)
{
    const int t = blockIdx.y, c = blockIdx.x, nchunk = gridDim.x;
    long i = (long)c * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (i < v3h) {
        long cb = (long)t * v3h + i;
        for (int j = 0; j < 12; ++j)
            for (int k = 0; k < 12; ++k) {
                double2 a = ev.p[((long)j * 12 + k) * ev.stride + cb];
                double2 b = od.p[((long)j * 12 + k) * od.stride + cb];
                acc += a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
            }
    }
    slice_finish(acc, t, c, nchunk, T, src_t, partial, counter, corr);
}

// host-layout columns: slice t of column j is the contiguous range
// [(j V + t V3) 24, (j V + (t+1) V3) 24) of doubles
__global__ void __launch_bounds__(128) contract_aos_kernel(long V, long v3, int T, int src_t, const double *prop,
                                                           double *partial, unsigned *counter, double *corr)
{
    const int t = blockIdx.y, c = blockIdx.x, nchunk = gridDim.x;
    const long n2 = v3 * 12;  // double2 words per slice and column
    double acc = 0.0;
    for (int j = 0; j < 12; ++j) {
        const double2 *base = reinterpret_cast<const double2 *>(prop + ((long)j * V + (long)t * v3) * 24);
        for (long w = (long)c * blockDim.x * 4 + threadIdx.x; w < n2 && w < (long)(c + 1) * blockDim.x * 4;
             w += blockDim.x) {
            double2 a = base[w];
            acc += a.x * a.x + a.y * a.y;
        }
    }
    slice_finish(acc, t, c, nchunk, T, src_t, partial, counter, corr);
}

// partial: T * ceil(V3/2 / 128) doubles; counter: T zeroed counters (left zeroed)
void pion_contract_soa(lqcd_lattice_s *lat, SpinorField<F64> even, SpinorField<F64> odd, int src_t,
                       double *corr_dev, double *partial, unsigned *counter, cudaStream_t st)
{
    const int T = lat->dims[3];
    const long v3h = lat->vh / T;
    const int nchunk = int((v3h + kBlock - 1) / kBlock);
    ProfScope prof("pion_contract", double(lat->V) * 12 * 192.0, st);
    contract_soa_kernel<<<dim3(nchunk, T), kBlock, 0, st>>>(v3h, T, src_t, even, odd, partial, counter, corr_dev);
    LQCD_CHECK_LAUNCH();
}

void pion_contract_aos(lqcd_lattice_s *lat, const double *prop_dev, int src_t, double *corr_dev, double *partial,
                       unsigned *counter, cudaStream_t st)
{
    const int T = lat->dims[3];
    const long v3 = lat->V / T;
    const long n2 = v3 * 12;
    const int nchunk = int((n2 + kBlock * 4 - 1) / (kBlock * 4));
    ProfScope prof("pion_contract", double(lat->V) * 12 * 192.0, st);
    contract_aos_kernel<<<dim3(nchunk, T), kBlock, 0, st>>>(lat->V, v3, T, src_t, prop_dev, partial, counter, corr_dev);
    LQCD_CHECK_LAUNCH();
}

}  // namespace lqcd
