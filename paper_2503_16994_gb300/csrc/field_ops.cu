// Gauge-field repacking, clover-field construction and inversion, spinor
// repacking between the host layout and the even-odd SoA layout, point
// sources and the pion contraction.
#include "gauge_dev.cuh"
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
LinkField<F64> hop_links<F64>(const GaugeSet &g, long stride, int bc)
{
    if (bc == LQCD_BC_SF) return {g.u64sf.as<const double2>(), nullptr, stride};
    return link_field<F64>(g, stride);
}
template <>
LinkField<F32> hop_links<F32>(const GaugeSet &g, long stride, int bc)
{
    if (bc == LQCD_BC_SF) return {g.u32sf.as<const float4>(), nullptr, stride};
    return link_field<F32>(g, stride);
}
template <>
LinkField<F16> hop_links<F16>(const GaugeSet &g, long stride, int bc)
{
    if (bc == LQCD_BC_SF) return {g.u16sf.as<const uint4>(), g.u16bsf.as<const uint2>(), stride};
    return link_field<F16>(g, stride);
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
template <>
CloverField<F64> clover_field_c<F64>(const CloverSet &c, long stride)
{
    return {c.cinv64.as<const double2>(), stride};
}
template <>
CloverField<F32> clover_field_c<F32>(const CloverSet &c, long stride)
{
    return {c.cinv32.as<const float4>(), stride};
}
template <>
CloverField<F16> clover_field_c<F16>(const CloverSet &c, long stride)
{
    return {c.cinv16.as<const uint4>(), stride};
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

// Schroedinger-functional hopping links: every copy with the links U_mu(x) of
// the boundary slice x_t = 0 and U_t(x) of x_t = T - 1 (which ends on the
// boundary x_t = T, stored as slice 0) set to zero, so no hop reaches the
// boundary slice in either direction
__global__ void sf_links_kernel(Geom g, const double2 *u64, const float4 *u32, const uint4 *u16, const uint2 *u16b,
                                double2 *s64, float4 *s32, uint4 *s16, uint2 *s16b)
{
    const long cb = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const int p = blockIdx.y, mu = blockIdx.z;
    if (cb >= g.vh) return;
    int x[4];
    cb_coords(g, p, int(cb), x);
    const bool zero = x[3] == 0 || (mu == 3 && x[3] == g.L[3] - 1);
    const long q = p * 4 + mu;
    for (int k = 0; k < 9; ++k)
        s64[(q * 9 + k) * g.stride + cb] = zero ? make_double2(0.0, 0.0) : u64[(q * 9 + k) * g.stride + cb];
    for (int k = 0; k < 3; ++k)
        s32[(q * 3 + k) * g.stride + cb] = zero ? make_float4(0.f, 0.f, 0.f, 0.f) : u32[(q * 3 + k) * g.stride + cb];
    s16[q * g.stride + cb] = zero ? make_uint4(0u, 0u, 0u, 0u) : u16[q * g.stride + cb];
    s16b[q * g.stride + cb] = zero ? make_uint2(0u, 0u) : u16b[q * g.stride + cb];
}

static void sf_links(lqcd_lattice_s *lat, GaugeSet &g, cudaStream_t st)
{
    if (g.sf_ready) return;
    const long S = lat->stride;
    g.u64sf.ensure(sizeof(double2) * 2 * 4 * 9 * S);
    g.u32sf.ensure(sizeof(float4) * 2 * 4 * 3 * S);
    g.u16sf.ensure(sizeof(uint4) * 2 * 4 * S);
    g.u16bsf.ensure(sizeof(uint2) * 2 * 4 * S);
    ProfScope prof("sf_links", double(lat->V) * 4 * 2 * (144.0 + 48.0 + 24.0), st);
    sf_links_kernel<<<dim3(unsigned((lat->vh + kBlock - 1) / kBlock), 2, 4), kBlock, 0, st>>>(
        lat->geom, g.u64.as<const double2>(), g.u32.as<const float4>(), g.u16.as<const uint4>(),
        g.u16b.as<const uint2>(), g.u64sf.as<double2>(), g.u32sf.as<float4>(), g.u16sf.as<uint4>(),
        g.u16bsf.as<uint2>());
    LQCD_CHECK_LAUNCH();
    g.sf_ready = true;
}

void gauge_repack(lqcd_lattice_s *lat, GaugeSet &g, const double *U_dev, cudaStream_t st)
{
    g.sf_ready = false;
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
// bc: LQCD_BC_OPEN: open time boundary (absent links across it), cfterm =
// 2 kappa (cF - 1) added to the site term on the first and last time slice;
// LQCD_BC_SF: Schroedinger-functional boundary at x_t = 0 (identity site term
// there; clover leaves from every link), cfterm on the slices 1 and T - 1
__global__ void __launch_bounds__(64) clover_build_kernel(Geom g, LinkField<F64> U, double kc, double tau, int bc,
                                                          double cfterm, double2 *a64, double2 *ainv64,
                                                          double2 *cinv64)
{
    const int p = blockIdx.y;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.vh) return;
    int x[4];
    cb_coords(g, p, cb, x);
    const bool open = bc == LQCD_BC_OPEN, sf = bc == LQCD_BC_SF;
    m3 Fxy = field_strength(g, U, x, 0, 1, open), Fxz = field_strength(g, U, x, 0, 2, open);
    m3 Fxt = field_strength(g, U, x, 0, 3, open), Fyz = field_strength(g, U, x, 1, 2, open);
    m3 Fyt = field_strength(g, U, x, 1, 3, open), Fzt = field_strength(g, U, x, 2, 3, open);
    const bool improved = open ? (x[3] == 0 || x[3] == g.L[3] - 1) : (sf && (x[3] == 1 || x[3] == g.L[3] - 1));
    const double diag = improved ? 1.0 + cfterm : 1.0;
    if (sf && x[3] == 0) kc = 0.0;  // the boundary slice: identity site term
    for (int blk = 0; blk < 2; ++blk) {
        const double sg = blk == 0 ? 1.0 : -1.0;
        cd A[6][6], Ai[6][6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                cd Mx = Fyz.m[i][j] + sg * Fxt.m[i][j];
                cd My = (-1.0) * Fxz.m[i][j] + sg * Fyt.m[i][j];
                cd Mz = Fxy.m[i][j] + sg * Fzt.m[i][j];
                cd id = cd{i == j ? diag : 0.0, 0.0};
                A[i][j] = id - kc * mul_i(Mz);
                A[3 + i][3 + j] = id + kc * mul_i(Mz);
                A[i][3 + j] = (-kc) * mul_i(Mx - mul_i(My));
                A[3 + i][j] = (-kc) * mul_i(Mx + mul_i(My));
            }
        store_block(a64 + (long)p * 36 * g.stride, g.stride, cb, 18 * blk, A);
        if (tau == 0.0) {
            invert6(A, Ai);
            store_block(ainv64 + (long)p * 36 * g.stride, g.stride, cb, 18 * blk, Ai);
        } else {
            // twisted block A + i s tau (s = +1 upper, -1 lower): its inverse is
            // B - i s tau C with C = (A^2 + tau^2)^-1 and B = A C (A Hermitian)
            cd M[6][6], Ci[6][6], B[6][6];
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    cd acc = cd{i == j ? tau * tau : 0.0, 0.0};
                    for (int k = 0; k < 6; ++k) acc = acc + A[i][k] * A[k][j];
                    M[i][j] = acc;
                }
            invert6(M, Ci);
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    cd acc = cd{0.0, 0.0};
                    for (int k = 0; k < 6; ++k) acc = acc + A[i][k] * Ci[k][j];
                    B[i][j] = acc;
                }
            store_block(ainv64 + (long)p * 36 * g.stride, g.stride, cb, 18 * blk, B);
            store_block(cinv64 + (long)p * 36 * g.stride, g.stride, cb, 18 * blk, Ci);
        }
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

size_t clover_bytes(const lqcd_lattice_s *lat, bool twisted)
{
    return (twisted ? 3 : 2) * 2 * (size_t)lat->stride * (36 * sizeof(double2) + 18 * sizeof(float4) + 9 * sizeof(uint4));
}

size_t gauge_bytes(const lqcd_lattice_s *lat)
{
    return 2 * 4 * (size_t)lat->stride * (9 * sizeof(double2) + 3 * sizeof(float4) + sizeof(uint4) + sizeof(uint2));
}

std::unique_ptr<CloverSet> clover_build(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp,
                                        cudaStream_t st, bool async)
{
    const double kc = dp.kappa * dp.csw;
    const bool bnd = dp.bc == LQCD_BC_OPEN || dp.bc == LQCD_BC_SF;
    auto c = std::make_unique<CloverSet>();
    c->tau = 2.0 * dp.kappa * dp.mu;
    const bool tw = c->tau != 0.0;
    if (async)
        for (DevBuf *b : {&c->a64, &c->ainv64, &c->cinv64, &c->a32, &c->ainv32, &c->cinv32, &c->a16, &c->ainv16,
                          &c->cinv16})
            b->set_async(st);
    const long S = lat->stride;
    c->a64.ensure(sizeof(double2) * 2 * 36 * S);
    c->ainv64.ensure(sizeof(double2) * 2 * 36 * S);
    c->a32.ensure(sizeof(float4) * 2 * 18 * S);
    c->ainv32.ensure(sizeof(float4) * 2 * 18 * S);
    c->a16.ensure(sizeof(uint4) * 2 * 9 * S);
    c->ainv16.ensure(sizeof(uint4) * 2 * 9 * S);
    if (tw) {
        c->cinv64.ensure(sizeof(double2) * 2 * 36 * S);
        c->cinv32.ensure(sizeof(float4) * 2 * 18 * S);
        c->cinv16.ensure(sizeof(uint4) * 2 * 9 * S);
    }
    dim3 grid(unsigned((lat->vh + 63) / 64), 2);
    ProfScope prof("clover_build", double(lat->V) * (4 * 144.0 + (tw ? 3 : 2) * 576.0), st);
    clover_build_kernel<<<grid, 64, 0, st>>>(lat->geom, link_field<F64>(g, S), kc, c->tau, dp.bc,
                                             bnd ? 2.0 * dp.kappa * (dp.cF - 1.0) : 0.0, c->a64.as<double2>(),
                                             c->ainv64.as<double2>(), tw ? c->cinv64.as<double2>() : nullptr);
    LQCD_CHECK_LAUNCH();
    dim3 g2(unsigned((lat->vh + kBlock - 1) / kBlock), 2);
    clover_convert_kernel<<<g2, kBlock, 0, st>>>(lat->vh, S, c->a64.as<const double2>(), c->a32.as<float4>(),
                                                 c->a16.as<uint4>());
    clover_convert_kernel<<<g2, kBlock, 0, st>>>(lat->vh, S, c->ainv64.as<const double2>(), c->ainv32.as<float4>(),
                                                 c->ainv16.as<uint4>());
    if (tw)
        clover_convert_kernel<<<g2, kBlock, 0, st>>>(lat->vh, S, c->cinv64.as<const double2>(), c->cinv32.as<float4>(),
                                                     c->cinv16.as<uint4>());
    LQCD_CHECK_LAUNCH();
    return c;
}

void hop_theta(const lqcd_dirac_params &dp, double th_re[4], double th_im[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        th_re[mu] = dp.theta_re[mu];
        th_im[mu] = dp.theta_im[mu];
    }
    if (dp.bc == LQCD_BC_OPEN) th_re[3] = th_im[3] = 0.0;  // the hops across the time boundary vanish
}

CloverSet &clover_get(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, cudaStream_t st)
{
    if (dp.bc == LQCD_BC_SF) sf_links(lat, g, st);
    const bool bnd = dp.bc == LQCD_BC_OPEN || dp.bc == LQCD_BC_SF;
    const auto key = std::make_tuple(dp.kappa * dp.csw, dp.kappa * dp.mu, int(dp.bc),
                                     bnd ? dp.kappa * (dp.cF - 1.0) : 0.0);
    auto it = g.clover.find(key);
    if (it != g.clover.end()) return *it->second;
    auto c = clover_build(lat, g, dp, st, false);
    CloverSet &ref = *c;
    g.clover.emplace(key, std::move(c));
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
// and the last block of the slice adds the chunks in a fixed order
// (slice_finish, gauge_dev.cuh).
// ---------------------------------------------------------------------------

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

// ---------------------------------------------------------------------------
// boundary-to-bulk correlators (open boundary)
// ---------------------------------------------------------------------------
// column j (j = 3 s + c, s < 2) at every site of slice 0: (P+ e_j)_al = (delta_{al,s} + (g_t)_{al,s}) / 2,
// with g_t = [[0, -1], [-1, 0]] in 2x2 spin blocks: P+ e_s = (e_s - e_{s+2}) / 2
__global__ void wall_source_kernel(long V, long v3, double *aos)
{
    const long i = long(blockIdx.x) * blockDim.x + threadIdx.x;  // (j, site) over 6 V
    if (i >= 6 * V) return;
    const int j = int(i / V);
    const long x = i - long(j) * V;
    double *o = aos + i * 24;
    for (int k = 0; k < 24; ++k) o[k] = 0.0;
    if (x < v3) {
        const int s = j / 3, c = j % 3;
        o[2 * (3 * s + c)] = 0.5;
        o[2 * (3 * (s + 2) + c)] = -0.5;
    }
}

void wall_sources_p_plus(lqcd_lattice_s *lat, double *aos, cudaStream_t st)
{
    const long n = 6 * lat->V;
    ProfScope prof("wall_source", double(n) * 192.0, st);
    wall_source_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(lat->V, lat->V / lat->dims[3], aos);
    LQCD_CHECK_LAUNCH();
}

// SF boundary sources W_j(1, yvec) = U_t(0, yvec)^dag P+ e_j on the slice 1
// (host layout, 6 columns): component (alpha, a) = P+[alpha][s] conj(U_t(0, yvec)[c][a])
__global__ void wall_source_sf_kernel(Geom g, long V, long v3, LinkField<F64> U, double *aos)
{
    const long i = long(blockIdx.x) * blockDim.x + threadIdx.x;  // (j, site) over 6 V
    if (i >= 6 * V) return;
    const int j = int(i / V);
    const long x = i - long(j) * V;
    double *o = aos + i * 24;
    for (int k = 0; k < 24; ++k) o[k] = 0.0;
    if (x >= v3 && x < 2 * v3) {
        const long y = x - v3;  // the site below on the boundary slice
        int xc[4];
        lex_coords(g, y, xc);
        const int p = (xc[0] + xc[1] + xc[2] + xc[3]) & 1;
        const long cb = y >> 1;
        const int s = j / 3, c = j % 3;
        for (int a = 0; a < 3; ++a) {
            const double2 u = U.p[((long)(p * 4 + 3) * 9 + 3 * c + a) * U.stride + cb];
            o[2 * (3 * s + a)] = 0.5 * u.x;
            o[2 * (3 * s + a) + 1] = -0.5 * u.y;
            o[2 * (3 * (s + 2) + a)] = -0.5 * u.x;
            o[2 * (3 * (s + 2) + a) + 1] = 0.5 * u.y;
        }
    }
}

void wall_sources_sf(lqcd_lattice_s *lat, const GaugeSet &g, double *aos, cudaStream_t st)
{
    const long n = 6 * lat->V;
    ProfScope prof("wall_source", double(n) * 192.0, st);
    wall_source_sf_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(lat->geom, lat->V, lat->V / lat->dims[3],
                                                                     link_field<F64>(g, lat->stride), aos);
    LQCD_CHECK_LAUNCH();
}

// per site: sum_j |h_j|^2 and -sum_j Re <h_j, g_t h_j>; with g_t mixing spin s and s + 2 by -1:
// <h, g_t h> = -sum_{s<2, c} 2 Re(conj(h_s) h_{s+2})
__global__ void __launch_bounds__(128) boundary_contract_kernel(long V, long v3, int T, const double *H,
                                                                double *partial, unsigned *counter, double *fP,
                                                                double *fA)
{
    const int t = blockIdx.y, c = blockIdx.x, nchunk = gridDim.x;
    const long x = long(c) * blockDim.x + threadIdx.x;
    double p = 0.0, a = 0.0;
    if (x < v3) {
        for (int j = 0; j < 6; ++j) {
            const double *h = H + ((long)j * V + (long)t * v3 + x) * 24;
            for (int k = 0; k < 24; ++k) p += h[k] * h[k];
            for (int q = 0; q < 6; ++q) {  // q = 3 s + colour, s < 2: pair with 3 (s + 2) + colour
                const double ur = h[2 * q], ui = h[2 * q + 1], dr = h[2 * (q + 6)], di = h[2 * (q + 6) + 1];
                a += 2.0 * (ur * dr + ui * di);  // -Re <h, g_t h>
            }
        }
    }
    slice_finish(p, t, c, nchunk, T, 0, partial, counter, fP);
    slice_finish(a, t, c, nchunk, T, 0, partial + (long)T * nchunk, counter + T, fA);
}

void boundary_contract(lqcd_lattice_s *lat, const double *H_dev, double *fP, double *fA, double *partial,
                       unsigned *counter, cudaStream_t st)
{
    const int T = lat->dims[3];
    const long v3 = lat->V / T;
    const int nchunk = int((v3 + kBlock - 1) / kBlock);
    ProfScope prof("boundary_contract", double(lat->V) * 6 * 192.0, st);
    boundary_contract_kernel<<<dim3(nchunk, T), kBlock, 0, st>>>(lat->V, v3, T, H_dev, partial, counter, fP, fA);
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
