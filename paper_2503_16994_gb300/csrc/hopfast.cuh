// Hopping kernel built to issue few instructions per site, for every
// storage format (FP16 and FP32 storage with FP32 arithmetic, FP64 storage
// with FP64 arithmetic):
//   * complex multiply-adds as explicit fmaf chains (4 FFMA each);
//   * neighbour sites as cb-index offsets with wrap corrections, site
//     coordinates by multiply-high division, all constants in FP32/int;
//   * the FP16 per-site scale applied to the projected two-spinor (12
//     multiplies instead of 24);
//   * NR right-hand sides per thread: each link is loaded, decoded and
//     completed (third row) once and used for all NR right-hand sides;
//   * GPB groups of NR right-hand sides per block, run one after the other,
//     so a tile's links and clover come from L1 after the first group.
// The arithmetic is the one of hop_kernel (kernels.cuh); only the
// instruction schedule differs.
#pragma once
#include "kernels.cuh"

namespace lqcd {

// n / d for 0 <= n < 2^31 as (umulhi(n, m) + n) >> s (Granlund-Montgomery),
// with m, s prepared on the host by make_fastdiv.
struct FastDiv {
    unsigned d, m, s;
};

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f) { return (__umulhi(n, f.m) + n) >> f.s; }

inline FastDiv make_fastdiv(unsigned d)
{
    unsigned l = 0;
    while ((1ull << l) < d) ++l;
    unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{d, unsigned(m), l};
}

template <class S>
struct FastHop {
    int L[4];
    int Lxh, vh, nrhs, ntiles, parity;
    FastDiv dx, dy, dz;          // divide by Lx/2, Ly, Lz
    int oy, oz, ot;              // cb offsets of one step in y, z, t
    double coef;
    double th_re[4], th_im[4];
    int gpb;                     // groups of NR right-hand sides per block
    int minb;                    // register cap: minimum resident blocks per SM (1, 4 or 6)
    int swz;                     // tiles per super-tile in the block order (1: tile-major)
    int theta_mask;              // bit mu set: theta_mu != 1
    SpinorField<S> in, self, out, b;  // b: RESID only
    LinkField<S> U;
    CloverField<S> clov;
    const RhsState *gate_st;
    int gate;
    Reduce red;
};

// tiles rounded up to whole super-tiles (the grid covers padded tiles)
template <class S>
inline long padded_tiles(const FastHop<S> &f)
{
    return long((f.ntiles + f.swz - 1) / f.swz) * f.swz;
}

// ---------------------------------------------------------------------------
// float complex helpers on (re, im) pairs held in plain floats
// ---------------------------------------------------------------------------
template <typename R> struct real_of { using type = float; };
template <> struct real_of<F64> { using type = double; };

// acc += u * v
template <typename R>
__device__ __forceinline__ void cmad(R &ar, R &ai, R ur, R ui, R vr, R vi)
{
    ar = fma(ur, vr, ar);
    ar = fma(-ui, vi, ar);
    ai = fma(ur, vi, ai);
    ai = fma(ui, vr, ai);
}
// acc += conj(u) * v
template <typename R>
__device__ __forceinline__ void cmadc(R &ar, R &ai, R ur, R ui, R vr, R vi)
{
    ar = fma(ur, vr, ar);
    ar = fma(ui, vi, ar);
    ai = fma(ur, vi, ai);
    ai = fma(-ui, vr, ai);
}

// load the 24 reals of a spinor; for FP16 the values are returned unscaled
// and the per-site scale separately (1 for FP32)
template <class S, typename R>
__device__ __forceinline__ R load_raw(const SpinorField<S> &f, int j, int i, R v[24])
{
    constexpr int NP = spinor_planes<S>::n;
    const typename S::word *b = f.p + (long)j * NP * f.stride + i;
    if constexpr (S::W == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            double2 w = __ldg(b + k * f.stride);
            v[2 * k] = w.x;
            v[2 * k + 1] = w.y;
        }
        return R(1);
    } else if constexpr (S::W == 4) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float4 w = __ldg(b + k * f.stride);
            v[4 * k] = w.x;
            v[4 * k + 1] = w.y;
            v[4 * k + 2] = w.z;
            v[4 * k + 3] = w.w;
        }
        return 1.0f;
    } else {
        const float sc = __ldg(f.scale + (long)j * f.stride + i);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            uint4 w = __ldg(b + k * f.stride);
            const __half2 *h = reinterpret_cast<const __half2 *>(&w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 t = __half22float2(h[q]);
                v[8 * k + 2 * q] = t.x;
                v[8 * k + 2 * q + 1] = t.y;
            }
        }
        return sc;
    }
}

// store 24 reals; returns the squared norm of the stored values
template <class S, typename R>
__device__ __forceinline__ double store_raw(const SpinorField<S> &f, int j, int i, const R v[24])
{
    constexpr int NP = spinor_planes<S>::n;
    typename S::word *b = f.p + (long)j * NP * f.stride + i;
    R n2 = R(0);
    if constexpr (S::W == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            b[k * f.stride] = make_double2(v[2 * k], v[2 * k + 1]);
            n2 = fma(v[2 * k], v[2 * k], n2);
            n2 = fma(v[2 * k + 1], v[2 * k + 1], n2);
        }
    } else if constexpr (S::W == 4) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            b[k * f.stride] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            n2 = fmaf(v[4 * k], v[4 * k], n2);
            n2 = fmaf(v[4 * k + 1], v[4 * k + 1], n2);
            n2 = fmaf(v[4 * k + 2], v[4 * k + 2], n2);
            n2 = fmaf(v[4 * k + 3], v[4 * k + 3], n2);
        }
    } else {
        float mx = 0.f;
#pragma unroll
        for (int q = 0; q < 24; ++q) mx = fmaxf(mx, fabsf(v[q]));
        if (!(mx >= 1e-30f)) mx = 0.f;  // see store_spinor: denormal sites are stored as zero
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        f.scale[(long)j * f.stride + i] = mx;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            uint4 w;
            __half2 *h = reinterpret_cast<__half2 *>(&w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] = __floats2half2_rn(v[8 * k + 2 * q] * inv, v[8 * k + 2 * q + 1] * inv);
                float2 t = __half22float2(h[q]);
                acc = fmaf(t.x, t.x, acc);
                acc = fmaf(t.y, t.y, acc);
            }
            b[k * f.stride] = w;
        }
        n2 = acc * mx * mx;
    }
    return double(n2);
}

// link as 18 floats (row-major re, im), third row completed from unitarity
template <class S, typename R>
__device__ __forceinline__ void load_link18(const LinkField<S> &f, int parity, int mu, int i, R u[18])
{
    if constexpr (S::W == 2) {
        const double2 *b = f.p + (long)(parity * 4 + mu) * 9 * f.stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 w = __ldg(b + k * f.stride);
            u[2 * k] = w.x;
            u[2 * k + 1] = w.y;
        }
        return;  // all 18 reals stored
    } else if constexpr (S::W == 4) {
        const float4 *b = f.p + (long)(parity * 4 + mu) * 3 * f.stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 w = __ldg(b + k * f.stride);
            u[4 * k] = w.x;
            u[4 * k + 1] = w.y;
            u[4 * k + 2] = w.z;
            u[4 * k + 3] = w.w;
        }
    } else {
        uint4 w = __ldg(f.p + (long)(parity * 4 + mu) * f.stride + i);
        uint2 w2 = __ldg(f.p2 + (long)(parity * 4 + mu) * f.stride + i);
        const __half2 *h = reinterpret_cast<const __half2 *>(&w);
        const __half2 *h2 = reinterpret_cast<const __half2 *>(&w2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float2 t = __half22float2(h[e]);
            u[2 * e] = t.x;
            u[2 * e + 1] = t.y;
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float2 t = __half22float2(h2[e]);
            u[8 + 2 * e] = t.x;
            u[9 + 2 * e] = t.y;
        }
    }
    // row2 = conj(row0 x row1): entry c = conj(r0[a] r1[b] - r0[b] r1[a]) for (a, b) = (1, 2), (2, 0), (0, 1)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        R re = R(0), im = R(0);
        cmad(re, im, u[2 * a], u[2 * a + 1], u[6 + 2 * b], u[7 + 2 * b]);
        cmad(re, im, -u[2 * b], -u[2 * b + 1], u[6 + 2 * a], u[7 + 2 * a]);
        u[12 + 2 * c] = re;
        u[13 + 2 * c] = -im;
    }
}

// ---------------------------------------------------------------------------
// one direction: project (1 + SG g_mu), scale, multiply by U or U^dag,
// optional phase, accumulate (chiral basis, see lqcd_dev.cuh)
// h[s][c] (s = 0, 1) as re/im float arrays
// ---------------------------------------------------------------------------
template <int MU, int SG, typename R>
__device__ __forceinline__ void project_f(const R v[24], R hr[2][3], R hi[2][3])
{
    // component index of spin s colour c: 2 (3 s + c)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R u0r = v[2 * c], u0i = v[2 * c + 1], u1r = v[6 + 2 * c], u1i = v[7 + 2 * c];
        const R d0r = v[12 + 2 * c], d0i = v[13 + 2 * c], d1r = v[18 + 2 * c], d1i = v[19 + 2 * c];
        // i s_mu (d0, d1) = (ta, tb); for t: (ta, tb) = (d0, d1)
        R tar, tai, tbr, tbi;
        if (MU == 0) { tar = -d1i; tai = d1r; tbr = -d0i; tbi = d0r; }
        if (MU == 1) { tar = d1r; tai = d1i; tbr = -d0r; tbi = -d0i; }
        if (MU == 2) { tar = -d0i; tai = d0r; tbr = d1i; tbi = -d1r; }
        if (MU == 3) { tar = d0r; tai = d0i; tbr = d1r; tbi = d1i; }
        // h = up - SG (i s_mu dn)   [t: h = up - SG dn]
        if (SG > 0) {
            hr[0][c] = u0r - tar; hi[0][c] = u0i - tai;
            hr[1][c] = u1r - tbr; hi[1][c] = u1i - tbi;
        } else {
            hr[0][c] = u0r + tar; hi[0][c] = u0i + tai;
            hr[1][c] = u1r + tbr; hi[1][c] = u1i + tbi;
        }
    }
}

template <int MU, int SG, typename R>
__device__ __forceinline__ void accumulate_f(R acc[24], const R gr[2][3], const R gi[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[2 * c] += gr[0][c];
        acc[2 * c + 1] += gi[0][c];
        acc[6 + 2 * c] += gr[1][c];
        acc[7 + 2 * c] += gi[1][c];
        // lower: t: -SG g ; k: SG i s_k g
        R tar, tai, tbr, tbi;
        if (MU == 0) { tar = -gi[1][c]; tai = gr[1][c]; tbr = -gi[0][c]; tbi = gr[0][c]; }
        if (MU == 1) { tar = gr[1][c]; tai = gi[1][c]; tbr = -gr[0][c]; tbi = -gi[0][c]; }
        if (MU == 2) { tar = -gi[0][c]; tai = gr[0][c]; tbr = gi[1][c]; tbi = -gr[1][c]; }
        if (MU == 3) { tar = gr[0][c]; tai = gi[0][c]; tbr = gr[1][c]; tbi = gi[1][c]; }
        const bool plus = (MU == 3) ? (SG < 0) : (SG > 0);
        if (plus) {
            acc[12 + 2 * c] += tar; acc[13 + 2 * c] += tai;
            acc[18 + 2 * c] += tbr; acc[19 + 2 * c] += tbi;
        } else {
            acc[12 + 2 * c] -= tar; acc[13 + 2 * c] -= tai;
            acc[18 + 2 * c] -= tbr; acc[19 + 2 * c] -= tbi;
        }
    }
}

// g = U h (DAGU = false) or U^dag h (DAGU = true), times `sc`
template <bool DAGU, typename R>
__device__ __forceinline__ void link_mul(const R u[18], R sc, const R hr[2][3], const R hi[2][3], R gr[2][3],
                                         R gi[2][3])
{
    R sr[2][3], si[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sr[s][c] = hr[s][c] * sc;
            si[s][c] = hi[s][c] * sc;
        }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R re = R(0), im = R(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (!DAGU)
                    cmad(re, im, u[2 * (3 * a + b)], u[2 * (3 * a + b) + 1], sr[s][b], si[s][b]);
                else
                    cmadc(re, im, u[2 * (3 * b + a)], u[2 * (3 * b + a) + 1], sr[s][b], si[s][b]);
            }
            gr[s][a] = re;
            gi[s][a] = im;
        }
}

// FP16 storage: the spin projection runs on the stored (re, im) half2 words
// of each right-hand side, before conversion, so only the 12 projected reals
// per right-hand side are converted to FP32 (rounding the projected sum to
// FP16 adds an error of the order of the storage rounding).
__device__ __forceinline__ __half2 h2_bits(unsigned b)
{
    __half2 h;
    *reinterpret_cast<unsigned *>(&h) = b;
    return h;
}
// u + s d for s = +-1
template <int SGN> __device__ __forceinline__ __half2 h_addsg(__half2 u, __half2 d)
{
    if constexpr (SGN > 0) return __hadd2(u, d);
    else return __hsub2(u, d);
}
// u + s i d = (u.re - s d.im, u.im + s d.re) for s = +-1
template <int SGN> __device__ __forceinline__ __half2 h_addi(__half2 u, __half2 d)
{
    // half2 (lo, hi) = (-1, +1) or (+1, -1)
    const __half2 m = h2_bits(SGN > 0 ? 0x3C00BC00u : 0xBC003C00u);
    return __hfma2(__lowhigh2highlow(d), m, u);
}

// the 12 half2 (re, im) words of right-hand side j at site y and its scale
__device__ __forceinline__ float load_words(const SpinorField<F16> &f, int j, int y, __half2 w[12])
{
    const uint4 *b = f.p + (long)j * 3 * f.stride + y;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 x = __ldg(b + k * f.stride);
        const __half2 *h = reinterpret_cast<const __half2 *>(&x);
#pragma unroll
        for (int q = 0; q < 4; ++q) w[4 * k + q] = h[q];
    }
    return __ldg(f.scale + (long)j * f.stride + y);
}

// h = up - S (i s_mu dn) (t: up - S dn) on half2 words; same cases as project_p
template <int MU, int S>
__device__ __forceinline__ void project_h(const __half2 v[12], __half2 h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const __half2 u0 = v[c], u1 = v[3 + c], d0 = v[6 + c], d1 = v[9 + c];
        if (MU == 0) {
            h[0][c] = h_addi<-S>(u0, d1);
            h[1][c] = h_addi<-S>(u1, d0);
        } else if (MU == 1) {
            h[0][c] = h_addsg<-S>(u0, d1);
            h[1][c] = h_addsg<S>(u1, d0);
        } else if (MU == 2) {
            h[0][c] = h_addi<-S>(u0, d0);
            h[1][c] = h_addi<S>(u1, d1);
        } else {
            h[0][c] = h_addsg<-S>(u0, d0);
            h[1][c] = h_addsg<-S>(u1, d1);
        }
    }
}

// one direction of one right-hand side from FP16 words: projection on the
// half2 words, unscaled link multiply, optional phase, then the per-site
// scale folded into the accumulation (acc += sc g, as fmas).  Per lane this
// is the arithmetic of the paired kernel, so every kernel shape gives the
// same bits.
template <bool DAGU>
__device__ __forceinline__ void link_mul_ns(const float u[18], const float hr[2][3], const float hi[2][3],
                                            float gr[2][3], float gi[2][3])
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (!DAGU)
                    cmad(re, im, u[2 * (3 * a + b)], u[2 * (3 * a + b) + 1], hr[s][b], hi[s][b]);
                else
                    cmadc(re, im, u[2 * (3 * b + a)], u[2 * (3 * b + a) + 1], hr[s][b], hi[s][b]);
            }
            gr[s][a] = re;
            gi[s][a] = im;
        }
}

// acc += sc (1 + S g_mu) psi from g (cases of accumulate_f)
template <int MU, int S>
__device__ __forceinline__ void accumulate_sc(float acc[24], const float gr[2][3], const float gi[2][3], float sc)
{
    const float ps = S > 0 ? sc : -sc, ms = -ps;  // S sc, -S sc
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[2 * c] = fmaf(gr[0][c], sc, acc[2 * c]);
        acc[2 * c + 1] = fmaf(gi[0][c], sc, acc[2 * c + 1]);
        acc[6 + 2 * c] = fmaf(gr[1][c], sc, acc[6 + 2 * c]);
        acc[7 + 2 * c] = fmaf(gi[1][c], sc, acc[7 + 2 * c]);
        float &l0r = acc[12 + 2 * c], &l0i = acc[13 + 2 * c], &l1r = acc[18 + 2 * c], &l1i = acc[19 + 2 * c];
        if (MU == 0) {  // lower += S (i g1, i g0)
            l0r = fmaf(gi[1][c], ms, l0r);
            l0i = fmaf(gr[1][c], ps, l0i);
            l1r = fmaf(gi[0][c], ms, l1r);
            l1i = fmaf(gr[0][c], ps, l1i);
        } else if (MU == 1) {  // lower += S (g1, -g0)
            l0r = fmaf(gr[1][c], ps, l0r);
            l0i = fmaf(gi[1][c], ps, l0i);
            l1r = fmaf(gr[0][c], ms, l1r);
            l1i = fmaf(gi[0][c], ms, l1i);
        } else if (MU == 2) {  // lower += S (i g0, -i g1)
            l0r = fmaf(gi[0][c], ms, l0r);
            l0i = fmaf(gr[0][c], ps, l0i);
            l1r = fmaf(gi[1][c], ps, l1r);
            l1i = fmaf(gr[1][c], ms, l1i);
        } else {  // lower -= S (g0, g1)
            l0r = fmaf(gr[0][c], ms, l0r);
            l0i = fmaf(gi[0][c], ms, l0i);
            l1r = fmaf(gr[1][c], ms, l1r);
            l1i = fmaf(gi[1][c], ms, l1i);
        }
    }
}

template <class S, int MU, int DIR, int SP>
__device__ __forceinline__ void half_dir_rhs(const FastHop<S> &a, const float u[18], const __half2 w[12], float sc,
                                             bool ph, float acc[24])
{
    __half2 hh[2][3];
    project_h<MU, SP>(w, hh);
    float hr[2][3], hi[2][3], gr[2][3], gi[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            hr[s][c] = __low2float(hh[s][c]);
            hi[s][c] = __high2float(hh[s][c]);
        }
    link_mul_ns<(DIR < 0)>(u, hr, hi, gr, gi);
    if (ph) {
        const float pr = float(a.th_re[MU]), pi = DIR > 0 ? float(a.th_im[MU]) : float(-a.th_im[MU]);
        const float npi = DIR > 0 ? float(-a.th_im[MU]) : float(a.th_im[MU]);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float xr = gr[s][c], xi = gi[s][c];
                gr[s][c] = fmaf(npi, xi, __fmul_rn(pr, xr));
                gi[s][c] = fmaf(pi, xr, __fmul_rn(pr, xi));
            }
    }
    accumulate_sc<MU, SP>(acc, gr, gi, sc);
}

// one direction for all NR right-hand sides of this thread
template <class S, int NR, int MU, int DIR, int SG, typename R>
__device__ __forceinline__ void dir_f(const FastHop<S> &a, const int (&jj)[NR], unsigned on, int i, int y, bool wrap,
                                      R (&acc)[NR][24])
{
    constexpr int SP = DIR > 0 ? -SG : SG;  // forward (1 - s g), backward (1 + s g)
    R u[18];
    load_link18<S, R>(a.U, DIR > 0 ? a.parity : (a.parity ^ 1), MU, DIR > 0 ? i : y, u);
    const bool ph = wrap && ((a.theta_mask >> MU) & 1);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (!((on >> r) & 1)) continue;
        if constexpr (S::W == 8) {
            __half2 w[12];
            const float sc = load_words(a.in, jj[r], y, w);
            half_dir_rhs<S, MU, DIR, SP>(a, u, w, sc, ph, acc[r]);
            continue;
        }
        R v[24];
        const R sc = load_raw<S, R>(a.in, jj[r], y, v);
        R hr[2][3], hi[2][3], gr[2][3], gi[2][3];
        project_f<MU, SP, R>(v, hr, hi);
        link_mul<DIR < 0, R>(u, sc, hr, hi, gr, gi);
        if (ph) {
            const R pr = R(a.th_re[MU]), pi = DIR > 0 ? R(a.th_im[MU]) : R(-a.th_im[MU]);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const R xr = gr[s][c], xi = gi[s][c];
                    gr[s][c] = pr * xr - pi * xi;
                    gi[s][c] = pr * xi + pi * xr;
                }
        }
        accumulate_f<MU, SP, R>(acc[r], gr, gi);
    }
}

// out = C v for one 6x6 Hermitian block (36 floats: d[6], then 15 upper (re, im))
template <typename R>
__device__ __forceinline__ void clov6(const R A[36], const R *v, R *o)
{
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        R re = A[r] * v[2 * r], im = A[r] * v[2 * r + 1];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (c > r) {
                const int k = 6 + 2 * (r * 5 - (r * (r - 1)) / 2 + (c - r - 1));
                cmad(re, im, A[k], A[k + 1], v[2 * c], v[2 * c + 1]);
            }
            if (c < r) {
                const int k = 6 + 2 * (c * 5 - (c * (c - 1)) / 2 + (r - c - 1));
                cmadc(re, im, A[k], A[k + 1], v[2 * c], v[2 * c + 1]);
            }
        }
        o[2 * r] = re;
        o[2 * r + 1] = im;
    }
}

template <class S, typename R>
__device__ __forceinline__ void load_clov_block(const CloverField<S> &f, int parity, int i, int blk, R A[36])
{
    if constexpr (S::W == 2) {
        const double2 *b = f.p + ((long)parity * 36 + blk * 18) * f.stride + i;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            double2 w = __ldg(b + k * f.stride);
            A[2 * k] = w.x;
            A[2 * k + 1] = w.y;
        }
    } else if constexpr (S::W == 4) {
        const float4 *b = f.p + ((long)parity * 18 + blk * 9) * f.stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float4 w = __ldg(b + k * f.stride);
            A[4 * k] = w.x;
            A[4 * k + 1] = w.y;
            A[4 * k + 2] = w.z;
            A[4 * k + 3] = w.w;
        }
    } else {
        // 36 reals of block blk start at real 36 blk = word 4.5 blk: load the
        // 5 words that cover them and pick
        const uint4 *b = f.p + (long)parity * 9 * f.stride + i;
        const int w0 = blk ? 4 : 0;
        float t[40];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            uint4 w = __ldg(b + (w0 + k) * f.stride);
            const __half2 *h = reinterpret_cast<const __half2 *>(&w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 x = __half22float2(h[q]);
                t[8 * k + 2 * q] = x.x;
                t[8 * k + 2 * q + 1] = x.y;
            }
        }
        const int off = blk ? 4 : 0;  // real 36 = word 4 + 4 reals
#pragma unroll
        for (int q = 0; q < 36; ++q) A[q] = t[off + q];
    }
}

template <class S, int NR, int MODE, bool DAG, bool NORM>
__device__ __forceinline__ void hopf_group(const FastHop<S> &a, int tile, int g)
{
    using R = typename real_of<S>::type;
    int jj[NR];
    unsigned on = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        jj[r] = g * NR + r;
        if (jj[r] < a.nrhs && (!a.gate_st || a.gate_st[jj[r]].status == a.gate)) on |= 1u << r;
        if (jj[r] >= a.nrhs) jj[r] = a.nrhs - 1;
    }
    if (!on) return;
    const int i = tile * blockDim.x + threadIdx.x;
    const bool valid = i < a.vh;
    R acc[NR][24];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[r][q] = R(0);
    if (valid) {
        const unsigned row = fdiv(unsigned(i), a.dx);
        const int xh = i - int(row) * a.Lxh;
        const unsigned q1 = fdiv(row, a.dy);
        const int y = int(row) - int(q1) * a.L[1];
        const unsigned q2 = fdiv(q1, a.dz);
        const int z = int(q1) - int(q2) * a.L[2];
        const int t = int(q2);
        const int x = 2 * xh + ((a.parity + y + z + t) & 1);
        const int rowbase = int(row) * a.Lxh;
        constexpr int SG = DAG ? -1 : 1;
        {
            const bool w = x == a.L[0] - 1;
            dir_f<S, NR, 0, +1, SG, R>(a, jj, on, i, rowbase + ((w ? 0 : x + 1) >> 1), w, acc);
        }
        {
            const bool w = x == 0;
            dir_f<S, NR, 0, -1, SG, R>(a, jj, on, i, rowbase + ((w ? a.L[0] - 1 : x - 1) >> 1), w, acc);
        }
        {
            const bool w = y == a.L[1] - 1;
            dir_f<S, NR, 1, +1, SG, R>(a, jj, on, i, i + (w ? -(a.L[1] - 1) * a.oy : a.oy), w, acc);
        }
        {
            const bool w = y == 0;
            dir_f<S, NR, 1, -1, SG, R>(a, jj, on, i, i - (w ? -(a.L[1] - 1) * a.oy : a.oy), w, acc);
        }
        {
            const bool w = z == a.L[2] - 1;
            dir_f<S, NR, 2, +1, SG, R>(a, jj, on, i, i + (w ? -(a.L[2] - 1) * a.oz : a.oz), w, acc);
        }
        {
            const bool w = z == 0;
            dir_f<S, NR, 2, -1, SG, R>(a, jj, on, i, i - (w ? -(a.L[2] - 1) * a.oz : a.oz), w, acc);
        }
        {
            const bool w = t == a.L[3] - 1;
            dir_f<S, NR, 3, +1, SG, R>(a, jj, on, i, i + (w ? -(a.L[3] - 1) * a.ot : a.ot), w, acc);
        }
        {
            const bool w = t == 0;
            dir_f<S, NR, 3, -1, SG, R>(a, jj, on, i, i - (w ? -(a.L[3] - 1) * a.ot : a.ot), w, acc);
        }
    }
    // epilogue, one right-hand side at a time
    const R coef = R(a.coef);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (!((on >> r) & 1)) continue;
        double n2 = 0.0;
        if (valid) {
            R res[24];
            if constexpr (MODE == SELF_PLAIN || MODE == CLOV_SUM) {
                // self + coef H in, then (CLOV_SUM) times C
                R sv[24];
                const R sc = load_raw<S, R>(a.self, jj[r], i, sv);
                if constexpr (S::W == 8) {
#pragma unroll
                    for (int q = 0; q < 24; ++q) sv[q] *= sc;
                }
#pragma unroll
                for (int q = 0; q < 24; ++q) sv[q] = fma(coef, acc[r][q], sv[q]);
                if constexpr (MODE == SELF_PLAIN) {
#pragma unroll
                    for (int q = 0; q < 24; ++q) res[q] = sv[q];
                } else {
                    R A[36];
#pragma unroll
                    for (int blk = 0; blk < 2; ++blk) {
                        load_clov_block<S, R>(a.clov, a.parity, i, blk, A);
                        clov6(A, sv + 12 * blk, res + 12 * blk);
                    }
                }
            } else if constexpr (MODE == HOP_CLOV) {
                // out = coef * C (H in)
                R A[36];
#pragma unroll
                for (int blk = 0; blk < 2; ++blk) {
                    load_clov_block<S, R>(a.clov, a.parity, i, blk, A);
                    clov6(A, acc[r] + 12 * blk, res + 12 * blk);
                }
#pragma unroll
                for (int q = 0; q < 24; ++q) res[q] *= coef;
            } else {
                // out = C self + coef * H in
                R sv[24];
                const R sc = load_raw<S, R>(a.self, jj[r], i, sv);
                if constexpr (S::W == 8) {
#pragma unroll
                    for (int q = 0; q < 24; ++q) sv[q] *= sc;
                }
                R A[36];
#pragma unroll
                for (int blk = 0; blk < 2; ++blk) {
                    load_clov_block<S, R>(a.clov, a.parity, i, blk, A);
                    clov6(A, sv + 12 * blk, res + 12 * blk);
                }
#pragma unroll
                for (int q = 0; q < 24; ++q) res[q] = fma(coef, acc[r][q], res[q]);
            }
            if constexpr (MODE == RESID) {
                // |b - (C self + coef H in)|^2, nothing stored
                R bv[24];
                const R sb = load_raw<S, R>(a.b, jj[r], i, bv);
                R t = R(0);
#pragma unroll
                for (int q = 0; q < 24; ++q) {
                    const R d = bv[q] * sb - res[q];
                    t = fma(d, d, t);
                }
                n2 = double(t);
            } else {
                n2 = store_raw<S, R>(a.out, jj[r], i, res);
            }
        }
        if (NORM) {
            if constexpr (S::W == 2) reduce_partial<double>(a.red, jj[r], tile, a.ntiles, n2);
            else reduce_partial<float>(a.red, jj[r], tile, a.ntiles, float(n2));  // n2 is an FP32 sum
        }
    }
}

// Block order: blocks are grouped in super-tiles of swz consecutive tiles;
// inside a super-tile the blocks run tile-fastest for each block-of-groups
// index, so neighbouring blocks work on neighbouring tiles of the same
// right-hand sides while a super-tile's links and clover stay in L2 for all
// right-hand sides.  swz = 1 puts the blocks of one tile next to each other.
// Returns false for the padding blocks of the last super-tile.
__device__ __forceinline__ bool block_tile(int ntiles, int nbt, int swz, int &tile, int &gb)
{
    const int per_super = swz * nbt;
    const int super = blockIdx.x / per_super, rem = blockIdx.x - super * per_super;
    gb = rem / swz;
    tile = super * swz + (rem - gb * swz);
    return tile < ntiles;
}

// Block handles one tile and groups [gb gpb, gb gpb + gpb) of NR right-hand
// sides, nbt = ceil(groups / gpb) blocks per tile; groups run in sequence.
template <class S, int NR, int MODE, bool DAG, bool NORM, int MINB>
__global__ void __launch_bounds__(128, MINB) hopf_kernel(const FastHop<S> a)
{
    const int ngr = (a.nrhs + NR - 1) / NR;
    const int nbt = (ngr + a.gpb - 1) / a.gpb;
    int tile, gb;
    if (!block_tile(a.ntiles, nbt, a.swz, tile, gb)) return;
    const int g0 = gb * a.gpb;
    const int g1 = min(ngr, g0 + a.gpb);
    for (int g = g0; g < g1; ++g) hopf_group<S, NR, MODE, DAG, NORM>(a, tile, g);
}

// ---------------------------------------------------------------------------
// Paired variant (FP16 / FP32 storage): two right-hand sides ride in the two
// lanes of a float2 and every arithmetic step is one packed FP32x2
// instruction (FFMA2 / FADD2 / FMUL2, sm_100 and later) for both.  Link and
// clover entries are shared by the two lanes (broadcast); the spin
// projection and the i sigma shuffles never cross lanes.
// ---------------------------------------------------------------------------
struct cp {
    float2 r, i;
};

__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a + s b for a compile-time sign s
template <int SGN> __device__ __forceinline__ float2 p_addsg(float2 a, float2 b)
{
    if constexpr (SGN > 0) return p_add(a, b);
    else return p_sub(a, b);
}

// the 24 reals of right-hand sides ja (lane x) and jb (lane y) at site y;
// FP16 values unscaled, the per-site scales returned as a pair
template <class S>
__device__ __forceinline__ float2 load_pair(const SpinorField<S> &f, int ja, int jb, int y, cp v[12])
{
    constexpr int NP = spinor_planes<S>::n;
    const typename S::word *ba = f.p + (long)ja * NP * f.stride + y;
    const typename S::word *bb = f.p + (long)jb * NP * f.stride + y;
    if constexpr (S::W == 4) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float4 A = __ldg(ba + k * f.stride), B = __ldg(bb + k * f.stride);
            v[2 * k] = cp{make_float2(A.x, B.x), make_float2(A.y, B.y)};
            v[2 * k + 1] = cp{make_float2(A.z, B.z), make_float2(A.w, B.w)};
        }
        return make_float2(1.f, 1.f);
    } else {
        const float2 sc =
            make_float2(__ldg(f.scale + (long)ja * f.stride + y), __ldg(f.scale + (long)jb * f.stride + y));
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const uint4 A = __ldg(ba + k * f.stride), B = __ldg(bb + k * f.stride);
            const __half2 *ha = reinterpret_cast<const __half2 *>(&A);
            const __half2 *hb = reinterpret_cast<const __half2 *>(&B);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[4 * k + q] = cp{__half22float2(__lows2half2(ha[q], hb[q])), __half22float2(__highs2half2(ha[q], hb[q]))};
        }
        return sc;
    }
}

// h = up - S (i s_mu dn) (t: up - S dn), components c of spins 0/1
template <int MU, int S>
__device__ __forceinline__ void project_p(const cp v[12], cp h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cp u0 = v[c], u1 = v[3 + c], d0 = v[6 + c], d1 = v[9 + c];
        if (MU == 0) {  // ta = i d1, tb = i d0
            h[0][c] = cp{p_addsg<S>(u0.r, d1.i), p_addsg<-S>(u0.i, d1.r)};
            h[1][c] = cp{p_addsg<S>(u1.r, d0.i), p_addsg<-S>(u1.i, d0.r)};
        } else if (MU == 1) {  // ta = d1, tb = -d0
            h[0][c] = cp{p_addsg<-S>(u0.r, d1.r), p_addsg<-S>(u0.i, d1.i)};
            h[1][c] = cp{p_addsg<S>(u1.r, d0.r), p_addsg<S>(u1.i, d0.i)};
        } else if (MU == 2) {  // ta = i d0, tb = -i d1
            h[0][c] = cp{p_addsg<S>(u0.r, d0.i), p_addsg<-S>(u0.i, d0.r)};
            h[1][c] = cp{p_addsg<-S>(u1.r, d1.i), p_addsg<S>(u1.i, d1.r)};
        } else {  // ta = d0, tb = d1
            h[0][c] = cp{p_addsg<-S>(u0.r, d0.r), p_addsg<-S>(u0.i, d0.i)};
            h[1][c] = cp{p_addsg<-S>(u1.r, d1.r), p_addsg<-S>(u1.i, d1.i)};
        }
    }
}

// acc += (1 + S g_mu) psi from g = projected, multiplied two-spinor
template <int MU, int S>
__device__ __forceinline__ void accumulate_p(cp acc[12], const cp g[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cp{p_add(acc[c].r, g[0][c].r), p_add(acc[c].i, g[0][c].i)};
        acc[3 + c] = cp{p_add(acc[3 + c].r, g[1][c].r), p_add(acc[3 + c].i, g[1][c].i)};
        cp &l0 = acc[6 + c], &l1 = acc[9 + c];
        if (MU == 0) {  // lower += S (i g1, i g0)
            l0 = cp{p_addsg<-S>(l0.r, g[1][c].i), p_addsg<S>(l0.i, g[1][c].r)};
            l1 = cp{p_addsg<-S>(l1.r, g[0][c].i), p_addsg<S>(l1.i, g[0][c].r)};
        } else if (MU == 1) {  // lower += S (g1, -g0)
            l0 = cp{p_addsg<S>(l0.r, g[1][c].r), p_addsg<S>(l0.i, g[1][c].i)};
            l1 = cp{p_addsg<-S>(l1.r, g[0][c].r), p_addsg<-S>(l1.i, g[0][c].i)};
        } else if (MU == 2) {  // lower += S (i g0, -i g1)
            l0 = cp{p_addsg<-S>(l0.r, g[0][c].i), p_addsg<S>(l0.i, g[0][c].r)};
            l1 = cp{p_addsg<S>(l1.r, g[1][c].i), p_addsg<-S>(l1.i, g[1][c].r)};
        } else {  // lower -= S (g0, g1)
            l0 = cp{p_addsg<-S>(l0.r, g[0][c].r), p_addsg<-S>(l0.i, g[0][c].i)};
            l1 = cp{p_addsg<-S>(l1.r, g[1][c].r), p_addsg<-S>(l1.i, g[1][c].i)};
        }
    }
}

// g = U (sc h) or U^dag (sc h) for both lanes
template <bool DAGU>
__device__ __forceinline__ void link_mul_p(const float u[18], float2 sc, const cp h[2][3], cp g[2][3])
{
    cp hs[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) hs[s][c] = cp{p_mul(h[s][c].r, sc), p_mul(h[s][c].i, sc)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cp acc0{bc(0.f), bc(0.f)}, acc1{bc(0.f), bc(0.f)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int k = DAGU ? 2 * (3 * b + a) : 2 * (3 * a + b);
            const float2 ur = bc(u[k]), ui = bc(u[k + 1]), nui = bc(-u[k + 1]);
            // U h:      re += ur hr - ui hi, im += ur hi + ui hr
            // U^dag h:  re += ur hr + ui hi, im += ur hi - ui hr
            const float2 x1 = DAGU ? ui : nui, x2 = DAGU ? nui : ui;
            acc0.r = p_fma(ur, hs[0][b].r, acc0.r);
            acc0.r = p_fma(x1, hs[0][b].i, acc0.r);
            acc0.i = p_fma(ur, hs[0][b].i, acc0.i);
            acc0.i = p_fma(x2, hs[0][b].r, acc0.i);
            acc1.r = p_fma(ur, hs[1][b].r, acc1.r);
            acc1.r = p_fma(x1, hs[1][b].i, acc1.r);
            acc1.i = p_fma(ur, hs[1][b].i, acc1.i);
            acc1.i = p_fma(x2, hs[1][b].r, acc1.i);
        }
        g[0][a] = acc0;
        g[1][a] = acc1;
    }
}

// g = U h or U^dag h for both lanes (no scale)
template <bool DAGU>
__device__ __forceinline__ void link_mul_u(const float u[18], const cp h[2][3], cp g[2][3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cp acc0{bc(0.f), bc(0.f)}, acc1{bc(0.f), bc(0.f)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int k = DAGU ? 2 * (3 * b + a) : 2 * (3 * a + b);
            const float2 ur = bc(u[k]), ui = bc(u[k + 1]), nui = bc(-u[k + 1]);
            const float2 x1 = DAGU ? ui : nui, x2 = DAGU ? nui : ui;
            acc0.r = p_fma(ur, h[0][b].r, acc0.r);
            acc0.r = p_fma(x1, h[0][b].i, acc0.r);
            acc0.i = p_fma(ur, h[0][b].i, acc0.i);
            acc0.i = p_fma(x2, h[0][b].r, acc0.i);
            acc1.r = p_fma(ur, h[1][b].r, acc1.r);
            acc1.r = p_fma(x1, h[1][b].i, acc1.r);
            acc1.i = p_fma(ur, h[1][b].i, acc1.i);
            acc1.i = p_fma(x2, h[1][b].r, acc1.i);
        }
        g[0][a] = acc0;
        g[1][a] = acc1;
    }
}

// acc += sc (1 + S g_mu) psi from g; the cases of accumulate_p with every
// add a packed fma by the per-site scale pair (sc, or nsc = -sc)
template <int MU, int S>
__device__ __forceinline__ void accumulate_s(cp acc[12], const cp g[2][3], float2 sc, float2 nsc)
{
    const float2 ps = S > 0 ? sc : nsc, ms = S > 0 ? nsc : sc;  // S sc, -S sc
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cp{p_fma(g[0][c].r, sc, acc[c].r), p_fma(g[0][c].i, sc, acc[c].i)};
        acc[3 + c] = cp{p_fma(g[1][c].r, sc, acc[3 + c].r), p_fma(g[1][c].i, sc, acc[3 + c].i)};
        cp &l0 = acc[6 + c], &l1 = acc[9 + c];
        if (MU == 0) {  // lower += S (i g1, i g0)
            l0 = cp{p_fma(g[1][c].i, ms, l0.r), p_fma(g[1][c].r, ps, l0.i)};
            l1 = cp{p_fma(g[0][c].i, ms, l1.r), p_fma(g[0][c].r, ps, l1.i)};
        } else if (MU == 1) {  // lower += S (g1, -g0)
            l0 = cp{p_fma(g[1][c].r, ps, l0.r), p_fma(g[1][c].i, ps, l0.i)};
            l1 = cp{p_fma(g[0][c].r, ms, l1.r), p_fma(g[0][c].i, ms, l1.i)};
        } else if (MU == 2) {  // lower += S (i g0, -i g1)
            l0 = cp{p_fma(g[0][c].i, ms, l0.r), p_fma(g[0][c].r, ps, l0.i)};
            l1 = cp{p_fma(g[1][c].i, ps, l1.r), p_fma(g[1][c].r, ms, l1.i)};
        } else {  // lower -= S (g0, g1)
            l0 = cp{p_fma(g[0][c].r, ms, l0.r), p_fma(g[0][c].i, ms, l0.i)};
            l1 = cp{p_fma(g[1][c].r, ms, l1.r), p_fma(g[1][c].i, ms, l1.i)};
        }
    }
}

// colour c of accumulate_s: acc += sc (1 + S g_mu) psi from (g0, g1) = g[0][c], g[1][c]
template <int MU, int S>
__device__ __forceinline__ void accumulate_row(cp acc[12], int c, const cp &g0, const cp &g1, float2 sc, float2 nsc)
{
    const float2 ps = S > 0 ? sc : nsc, ms = S > 0 ? nsc : sc;  // S sc, -S sc
    acc[c] = cp{p_fma(g0.r, sc, acc[c].r), p_fma(g0.i, sc, acc[c].i)};
    acc[3 + c] = cp{p_fma(g1.r, sc, acc[3 + c].r), p_fma(g1.i, sc, acc[3 + c].i)};
    cp &l0 = acc[6 + c], &l1 = acc[9 + c];
    if (MU == 0) {  // lower += S (i g1, i g0)
        l0 = cp{p_fma(g1.i, ms, l0.r), p_fma(g1.r, ps, l0.i)};
        l1 = cp{p_fma(g0.i, ms, l1.r), p_fma(g0.r, ps, l1.i)};
    } else if (MU == 1) {  // lower += S (g1, -g0)
        l0 = cp{p_fma(g1.r, ps, l0.r), p_fma(g1.i, ps, l0.i)};
        l1 = cp{p_fma(g0.r, ms, l1.r), p_fma(g0.i, ms, l1.i)};
    } else if (MU == 2) {  // lower += S (i g0, -i g1)
        l0 = cp{p_fma(g0.i, ms, l0.r), p_fma(g0.r, ps, l0.i)};
        l1 = cp{p_fma(g1.i, ps, l1.r), p_fma(g1.r, ms, l1.i)};
    } else {  // lower -= S (g0, g1)
        l0 = cp{p_fma(g0.r, ms, l0.r), p_fma(g0.i, ms, l0.i)};
        l1 = cp{p_fma(g1.r, ms, l1.r), p_fma(g1.i, ms, l1.i)};
    }
}

// row a of g = U h or U^dag h for both lanes: the operations of link_mul_u for one colour row
template <bool DAGU>
__device__ __forceinline__ void link_row_u(const float u[18], int a, const cp h[2][3], cp &g0, cp &g1)
{
    cp acc0{bc(0.f), bc(0.f)}, acc1{bc(0.f), bc(0.f)};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int k = DAGU ? 2 * (3 * b + a) : 2 * (3 * a + b);
        const float2 ur = bc(u[k]), ui = bc(u[k + 1]), nui = bc(-u[k + 1]);
        const float2 x1 = DAGU ? ui : nui, x2 = DAGU ? nui : ui;
        acc0.r = p_fma(ur, h[0][b].r, acc0.r);
        acc0.r = p_fma(x1, h[0][b].i, acc0.r);
        acc0.i = p_fma(ur, h[0][b].i, acc0.i);
        acc0.i = p_fma(x2, h[0][b].r, acc0.i);
        acc1.r = p_fma(ur, h[1][b].r, acc1.r);
        acc1.r = p_fma(x1, h[1][b].i, acc1.r);
        acc1.i = p_fma(ur, h[1][b].i, acc1.i);
        acc1.i = p_fma(x2, h[1][b].r, acc1.i);
    }
    g0 = acc0;
    g1 = acc1;
}

// one direction of a pair of right-hand sides from their FP16 words (wa, wb,
// scales sa, sb) and the decoded link u; each colour row of the link product
// is phased and accumulated as soon as it is formed (the element-wise
// operations of link_mul_u, the phase and accumulate_s, so the same bits)
template <class S, int MU, int DIR, int SP>
__device__ __forceinline__ void dir_words(const FastHop<S> &a, const float u[18], const __half2 wa[12],
                                          const __half2 wb[12], float sa, float sb, bool wrap, cp acc[12])
{
    cp h[2][3];
    __half2 ha[2][3], hb[2][3];
    project_h<MU, SP>(wa, ha);
    project_h<MU, SP>(wb, hb);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            h[s][c] = cp{make_float2(__low2float(ha[s][c]), __low2float(hb[s][c])),
                         make_float2(__high2float(ha[s][c]), __high2float(hb[s][c]))};
    const bool phase = wrap && ((a.theta_mask >> MU) & 1);
    const float2 sc = make_float2(sa, sb), nsc = make_float2(-sa, -sb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cp g0, g1;
        link_row_u<(DIR < 0)>(u, c, h, g0, g1);
        if (phase) {
            const float2 pr = bc(float(a.th_re[MU])), pi = bc(DIR > 0 ? float(a.th_im[MU]) : float(-a.th_im[MU]));
            const float2 npi = bc(DIR > 0 ? float(-a.th_im[MU]) : float(a.th_im[MU]));
            g0 = cp{p_fma(npi, g0.i, p_mul(pr, g0.r)), p_fma(pi, g0.r, p_mul(pr, g0.i))};
            g1 = cp{p_fma(npi, g1.i, p_mul(pr, g1.r)), p_fma(pi, g1.r, p_mul(pr, g1.i))};
        }
        accumulate_row<MU, SP>(acc, c, g0, g1, sc, nsc);
    }
}

template <class S, int MU, int DIR, int SG>
__device__ __forceinline__ void dir_p(const FastHop<S> &a, int ja, int jb, int i, int y, bool wrap, cp acc[12])
{
    constexpr int SP = DIR > 0 ? -SG : SG;
    float u[18];
    load_link18<S, float>(a.U, DIR > 0 ? a.parity : (a.parity ^ 1), MU, DIR > 0 ? i : y, u);
    cp h[2][3], g[2][3];
    if constexpr (S::W == 8) {
        __half2 wa[12], wb[12];
        const float sa = load_words(a.in, ja, y, wa), sb = load_words(a.in, jb, y, wb);
        dir_words<S, MU, DIR, SP>(a, u, wa, wb, sa, sb, wrap, acc);
        return;
    }
    cp v[12];
    const float2 sc = load_pair<S>(a.in, ja, jb, y, v);
    project_p<MU, SP>(v, h);
    link_mul_p<(DIR < 0)>(u, sc, h, g);
    if (wrap && ((a.theta_mask >> MU) & 1)) {
        const float2 pr = bc(float(a.th_re[MU])), pi = bc(DIR > 0 ? float(a.th_im[MU]) : float(-a.th_im[MU]));
        const float2 npi = bc(DIR > 0 ? float(-a.th_im[MU]) : float(a.th_im[MU]));
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cp x = g[s][c];
                g[s][c] = cp{p_fma(npi, x.i, p_mul(pr, x.r)), p_fma(pi, x.r, p_mul(pr, x.i))};
            }
    }
    accumulate_p<MU, SP>(acc, g);
}

// out = A v for one Hermitian 6x6 block (36 floats), both lanes
__device__ __forceinline__ void clov6_p(const float A[36], const cp *v, cp *o)
{
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const float2 d = bc(A[r]);
        cp acc{p_mul(d, v[r].r), p_mul(d, v[r].i)};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (c == r) continue;
            const int lo = c > r ? r : c, hi = c > r ? c : r;
            const int k = 6 + 2 * (lo * 5 - (lo * (lo - 1)) / 2 + (hi - lo - 1));
            const float2 ur = bc(A[k]);
            // entry (r, c) = A_k for c > r, conj(A_k) for c < r
            const float2 ui = bc(c > r ? A[k + 1] : -A[k + 1]), nui = bc(c > r ? -A[k + 1] : A[k + 1]);
            acc.r = p_fma(ur, v[c].r, acc.r);
            acc.r = p_fma(nui, v[c].i, acc.r);
            acc.i = p_fma(ur, v[c].i, acc.i);
            acc.i = p_fma(ui, v[c].r, acc.i);
        }
        o[r] = acc;
    }
}

// clover epilogue, store and norm partials of a pair of right-hand sides
template <class S, int MODE, bool NORM>
__device__ __forceinline__ void hopp_epilogue(const FastHop<S> &a, int tile, int i, bool valid, int ja, bool on_a,
                                              int jb, bool on_b, const cp acc[12])
{
    double n2a = 0.0, n2b = 0.0;
    if (valid) {
        cp res[12];
        const float2 cf = bc(float(a.coef));
        if constexpr (MODE == HOP_CLOV) {
            float A[36];
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                load_clov_block<S, float>(a.clov, a.parity, i, blk, A);
                clov6_p(A, acc + 6 * blk, res + 6 * blk);
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) res[q] = cp{p_mul(cf, res[q].r), p_mul(cf, res[q].i)};
        } else {
            cp sv[12];
            const float2 sc = load_pair<S>(a.self, ja, jb, i, sv);
            if constexpr (S::W == 8) {
#pragma unroll
                for (int q = 0; q < 12; ++q) sv[q] = cp{p_mul(sv[q].r, sc), p_mul(sv[q].i, sc)};
            }
            float A[36];
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                load_clov_block<S, float>(a.clov, a.parity, i, blk, A);
                clov6_p(A, sv + 6 * blk, res + 6 * blk);
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) res[q] = cp{p_fma(cf, acc[q].r, res[q].r), p_fma(cf, acc[q].i, res[q].i)};
        }
        float va[24], vb[24];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            va[2 * q] = res[q].r.x;
            va[2 * q + 1] = res[q].i.x;
            vb[2 * q] = res[q].r.y;
            vb[2 * q + 1] = res[q].i.y;
        }
        if (on_a) n2a = store_raw<S, float>(a.out, ja, i, va);
        if (on_b) n2b = store_raw<S, float>(a.out, jb, i, vb);
    }
    if (NORM) reduce_partial2(a.red, ja, on_a, jb, on_b, tile, a.ntiles, float(n2a), float(n2b));  // FP32 sums
}

template <class S, int MODE, bool DAG, bool NORM>
__device__ __forceinline__ void hopp_group(const FastHop<S> &a, int tile, int g)
{
    const int ja0 = 2 * g, jb0 = 2 * g + 1;
    const bool on_a = ja0 < a.nrhs && (!a.gate_st || a.gate_st[ja0].status == a.gate);
    const bool on_b = jb0 < a.nrhs && (!a.gate_st || a.gate_st[jb0].status == a.gate);
    if (!on_a && !on_b) return;
    const int ja = min(ja0, a.nrhs - 1), jb = min(jb0, a.nrhs - 1);
    const int i = tile * blockDim.x + threadIdx.x;
    const bool valid = i < a.vh;
    cp acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = cp{bc(0.f), bc(0.f)};
    if (valid) {
        const unsigned row = fdiv(unsigned(i), a.dx);
        const int xh = i - int(row) * a.Lxh;
        const unsigned q1 = fdiv(row, a.dy);
        const int y = int(row) - int(q1) * a.L[1];
        const unsigned q2 = fdiv(q1, a.dz);
        const int z = int(q1) - int(q2) * a.L[2];
        const int t = int(q2);
        const int x = 2 * xh + ((a.parity + y + z + t) & 1);
        const int rowbase = int(row) * a.Lxh;
        constexpr int SG = DAG ? -1 : 1;
        bool w;
        w = x == a.L[0] - 1;
        dir_p<S, 0, +1, SG>(a, ja, jb, i, rowbase + ((w ? 0 : x + 1) >> 1), w, acc);
        w = x == 0;
        dir_p<S, 0, -1, SG>(a, ja, jb, i, rowbase + ((w ? a.L[0] - 1 : x - 1) >> 1), w, acc);
        w = y == a.L[1] - 1;
        dir_p<S, 1, +1, SG>(a, ja, jb, i, i + (w ? -(a.L[1] - 1) * a.oy : a.oy), w, acc);
        w = y == 0;
        dir_p<S, 1, -1, SG>(a, ja, jb, i, i - (w ? -(a.L[1] - 1) * a.oy : a.oy), w, acc);
        w = z == a.L[2] - 1;
        dir_p<S, 2, +1, SG>(a, ja, jb, i, i + (w ? -(a.L[2] - 1) * a.oz : a.oz), w, acc);
        w = z == 0;
        dir_p<S, 2, -1, SG>(a, ja, jb, i, i - (w ? -(a.L[2] - 1) * a.oz : a.oz), w, acc);
        w = t == a.L[3] - 1;
        dir_p<S, 3, +1, SG>(a, ja, jb, i, i + (w ? -(a.L[3] - 1) * a.ot : a.ot), w, acc);
        w = t == 0;
        dir_p<S, 3, -1, SG>(a, ja, jb, i, i - (w ? -(a.L[3] - 1) * a.ot : a.ot), w, acc);
    }
    hopp_epilogue<S, MODE, NORM>(a, tile, i, valid, ja, on_a, jb, on_b, acc);
}

// Block b handles tile b / nbt and pair groups [(b % nbt) gpb, ... + gpb).
template <class S, int MODE, bool DAG, bool NORM, int MINB>
__global__ void __launch_bounds__(128, MINB) hopp_kernel(const FastHop<S> a)
{
    const int ngr = (a.nrhs + 1) / 2;
    const int nbt = (ngr + a.gpb - 1) / a.gpb;
    int tile, gb;
    if (!block_tile(a.ntiles, nbt, a.swz, tile, gb)) return;
    const int g0 = gb * a.gpb;
    const int g1 = min(ngr, g0 + a.gpb);
    for (int g = g0; g < g1; ++g) hopp_group<S, MODE, DAG, NORM>(a, tile, g);
}

// ---------------------------------------------------------------------------
// Prefetching variant (one right-hand side per thread, FP16 / FP32 storage):
// the raw words of the links and neighbour spinors of PF directions are
// loaded before any of them is used, so a thread has PF directions of loads
// in flight instead of one (the kernel is bound by load latency otherwise).
// ---------------------------------------------------------------------------
template <class S>
struct RawSpinor {
    typename S::word w[spinor_planes<S>::n];
    float sc;
};
template <class S>
struct RawLink {
    typename S::word w[S::W == 4 ? 3 : 1];
    uint2 w2;  // FP16 only
};

template <class S>
__device__ __forceinline__ void fetch_spinor(const SpinorField<S> &f, int j, int y, RawSpinor<S> &r)
{
    constexpr int NP = spinor_planes<S>::n;
    const typename S::word *b = f.p + (long)j * NP * f.stride + y;
#pragma unroll
    for (int k = 0; k < NP; ++k) r.w[k] = __ldg(b + k * f.stride);
    if constexpr (S::W == 8) r.sc = __ldg(f.scale + (long)j * f.stride + y);
    else r.sc = 1.f;
}

template <class S>
__device__ __forceinline__ void fetch_link(const LinkField<S> &f, int parity, int mu, int i, RawLink<S> &r)
{
    if constexpr (S::W == 4) {
        const float4 *b = f.p + (long)(parity * 4 + mu) * 3 * f.stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) r.w[k] = __ldg(b + k * f.stride);
    } else {
        r.w[0] = __ldg(f.p + (long)(parity * 4 + mu) * f.stride + i);
        r.w2 = __ldg(f.p2 + (long)(parity * 4 + mu) * f.stride + i);
    }
}

template <class S>
__device__ __forceinline__ void decode_spinor(const RawSpinor<S> &r, float v[24])
{
    constexpr int NP = spinor_planes<S>::n;
    if constexpr (S::W == 4) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            v[4 * k] = r.w[k].x;
            v[4 * k + 1] = r.w[k].y;
            v[4 * k + 2] = r.w[k].z;
            v[4 * k + 3] = r.w[k].w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const __half2 *h = reinterpret_cast<const __half2 *>(&r.w[k]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 t = __half22float2(h[q]);
                v[8 * k + 2 * q] = t.x;
                v[8 * k + 2 * q + 1] = t.y;
            }
        }
    }
}

template <class S>
__device__ __forceinline__ void decode_link(const RawLink<S> &r, float u[18])
{
    if constexpr (S::W == 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[4 * k] = r.w[k].x;
            u[4 * k + 1] = r.w[k].y;
            u[4 * k + 2] = r.w[k].z;
            u[4 * k + 3] = r.w[k].w;
        }
    } else {
        const __half2 *h = reinterpret_cast<const __half2 *>(&r.w[0]);
        const __half2 *h2 = reinterpret_cast<const __half2 *>(&r.w2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float2 t = __half22float2(h[e]);
            u[2 * e] = t.x;
            u[2 * e + 1] = t.y;
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float2 t = __half22float2(h2[e]);
            u[8 + 2 * e] = t.x;
            u[9 + 2 * e] = t.y;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        float re = 0.f, im = 0.f;
        cmad(re, im, u[2 * a], u[2 * a + 1], u[6 + 2 * b], u[7 + 2 * b]);
        cmad(re, im, -u[2 * b], -u[2 * b + 1], u[6 + 2 * a], u[7 + 2 * a]);
        u[12 + 2 * c] = re;
        u[13 + 2 * c] = -im;
    }
}

// direction d = 2 mu + (0 forward, 1 backward)
template <class S, int D, int SG>
__device__ __forceinline__ void compute_dir(const FastHop<S> &a, const RawLink<S> &rl, const RawSpinor<S> &rs,
                                            bool wrap, float acc[24])
{
    constexpr int MU = D / 2, DIR = (D & 1) ? -1 : 1;
    constexpr int SP = DIR > 0 ? -SG : SG;
    float u[18], v[24];
    decode_link<S>(rl, u);
    if constexpr (S::W == 8) {
        half_dir_rhs<S, MU, DIR, SP>(a, u, reinterpret_cast<const __half2 *>(rs.w), rs.sc,
                                     wrap && ((a.theta_mask >> MU) & 1), acc);
        return;
    }
    decode_spinor<S>(rs, v);
    float hr[2][3], hi[2][3], gr[2][3], gi[2][3];
    project_f<MU, SP, float>(v, hr, hi);
    link_mul<(DIR < 0), float>(u, rs.sc, hr, hi, gr, gi);
    if (wrap && ((a.theta_mask >> MU) & 1)) {
        const float pr = float(a.th_re[MU]), pi = DIR > 0 ? float(a.th_im[MU]) : float(-a.th_im[MU]);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float xr = gr[s][c], xi = gi[s][c];
                gr[s][c] = pr * xr - pi * xi;
                gi[s][c] = pr * xi + pi * xr;
            }
    }
    accumulate_f<MU, SP, float>(acc, gr, gi);
}

template <class S, int D0, int PF, int SG>
__device__ __forceinline__ void phase_dirs(const FastHop<S> &a, int j, int i, const int (&nb)[8], unsigned wrapm,
                                           float acc[24])
{
    RawLink<S> rl[PF];
    RawSpinor<S> rs[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q) {
        const int d = D0 + q;
        fetch_link<S>(a.U, (d & 1) ? (a.parity ^ 1) : a.parity, d / 2, (d & 1) ? nb[d] : i, rl[q]);
        fetch_spinor<S>(a.in, j, nb[d], rs[q]);
    }
    if constexpr (PF == 8) {
        compute_dir<S, D0 + 0, SG>(a, rl[0], rs[0], (wrapm >> (D0 + 0)) & 1, acc);
        compute_dir<S, D0 + 1, SG>(a, rl[1], rs[1], (wrapm >> (D0 + 1)) & 1, acc);
        compute_dir<S, D0 + 2, SG>(a, rl[2], rs[2], (wrapm >> (D0 + 2)) & 1, acc);
        compute_dir<S, D0 + 3, SG>(a, rl[3], rs[3], (wrapm >> (D0 + 3)) & 1, acc);
        compute_dir<S, D0 + 4, SG>(a, rl[4], rs[4], (wrapm >> (D0 + 4)) & 1, acc);
        compute_dir<S, D0 + 5, SG>(a, rl[5], rs[5], (wrapm >> (D0 + 5)) & 1, acc);
        compute_dir<S, D0 + 6, SG>(a, rl[6], rs[6], (wrapm >> (D0 + 6)) & 1, acc);
        compute_dir<S, D0 + 7, SG>(a, rl[7], rs[7], (wrapm >> (D0 + 7)) & 1, acc);
    } else if constexpr (PF == 4) {
        compute_dir<S, D0 + 0, SG>(a, rl[0], rs[0], (wrapm >> (D0 + 0)) & 1, acc);
        compute_dir<S, D0 + 1, SG>(a, rl[1], rs[1], (wrapm >> (D0 + 1)) & 1, acc);
        compute_dir<S, D0 + 2, SG>(a, rl[2], rs[2], (wrapm >> (D0 + 2)) & 1, acc);
        compute_dir<S, D0 + 3, SG>(a, rl[3], rs[3], (wrapm >> (D0 + 3)) & 1, acc);
    } else {
        compute_dir<S, D0 + 0, SG>(a, rl[0], rs[0], (wrapm >> (D0 + 0)) & 1, acc);
        compute_dir<S, D0 + 1, SG>(a, rl[1], rs[1], (wrapm >> (D0 + 1)) & 1, acc);
    }
}

template <class S, int MODE, bool DAG, bool NORM, int PF>
__device__ __forceinline__ void hopq_item(const FastHop<S> &a, int tile, int j)
{
    if (a.gate_st && a.gate_st[j].status != a.gate) return;
    const int i = tile * blockDim.x + threadIdx.x;
    const bool valid = i < a.vh;
    double n2 = 0.0;
    if (valid) {
        const unsigned row = fdiv(unsigned(i), a.dx);
        const int xh = i - int(row) * a.Lxh;
        const unsigned q1 = fdiv(row, a.dy);
        const int y = int(row) - int(q1) * a.L[1];
        const unsigned q2 = fdiv(q1, a.dz);
        const int z = int(q1) - int(q2) * a.L[2];
        const int t = int(q2);
        const int x = 2 * xh + ((a.parity + y + z + t) & 1);
        const int rowbase = int(row) * a.Lxh;
        int nb[8];
        unsigned wm = 0;
        bool w;
        w = x == a.L[0] - 1; wm |= unsigned(w) << 0; nb[0] = rowbase + ((w ? 0 : x + 1) >> 1);
        w = x == 0;          wm |= unsigned(w) << 1; nb[1] = rowbase + ((w ? a.L[0] - 1 : x - 1) >> 1);
        w = y == a.L[1] - 1; wm |= unsigned(w) << 2; nb[2] = i + (w ? -(a.L[1] - 1) * a.oy : a.oy);
        w = y == 0;          wm |= unsigned(w) << 3; nb[3] = i - (w ? -(a.L[1] - 1) * a.oy : a.oy);
        w = z == a.L[2] - 1; wm |= unsigned(w) << 4; nb[4] = i + (w ? -(a.L[2] - 1) * a.oz : a.oz);
        w = z == 0;          wm |= unsigned(w) << 5; nb[5] = i - (w ? -(a.L[2] - 1) * a.oz : a.oz);
        w = t == a.L[3] - 1; wm |= unsigned(w) << 6; nb[6] = i + (w ? -(a.L[3] - 1) * a.ot : a.ot);
        w = t == 0;          wm |= unsigned(w) << 7; nb[7] = i - (w ? -(a.L[3] - 1) * a.ot : a.ot);
        constexpr int SG = DAG ? -1 : 1;
        float acc[24];
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[q] = 0.f;
        if constexpr (PF == 8) {
            phase_dirs<S, 0, 8, SG>(a, j, i, nb, wm, acc);
        } else if constexpr (PF == 4) {
            phase_dirs<S, 0, 4, SG>(a, j, i, nb, wm, acc);
            phase_dirs<S, 4, 4, SG>(a, j, i, nb, wm, acc);
        } else {
            phase_dirs<S, 0, 2, SG>(a, j, i, nb, wm, acc);
            phase_dirs<S, 2, 2, SG>(a, j, i, nb, wm, acc);
            phase_dirs<S, 4, 2, SG>(a, j, i, nb, wm, acc);
            phase_dirs<S, 6, 2, SG>(a, j, i, nb, wm, acc);
        }
        float res[24];
        const float coef = float(a.coef);
        if constexpr (MODE == HOP_CLOV) {
            float A[36];
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                load_clov_block<S, float>(a.clov, a.parity, i, blk, A);
                clov6(A, acc + 12 * blk, res + 12 * blk);
            }
#pragma unroll
            for (int q = 0; q < 24; ++q) res[q] *= coef;
        } else {
            float sv[24];
            const float sc = load_raw<S, float>(a.self, j, i, sv);
            if constexpr (S::W == 8) {
#pragma unroll
                for (int q = 0; q < 24; ++q) sv[q] *= sc;
            }
            float A[36];
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                load_clov_block<S, float>(a.clov, a.parity, i, blk, A);
                clov6(A, sv + 12 * blk, res + 12 * blk);
            }
#pragma unroll
            for (int q = 0; q < 24; ++q) res[q] = fmaf(coef, acc[q], res[q]);
        }
        n2 = store_raw<S, float>(a.out, j, i, res);
    }
    if (NORM) reduce_partial<float>(a.red, j, tile, a.ntiles, float(n2));  // FP16/FP32 only: an FP32 sum
}

// Block b handles tile b / nbt and right-hand sides [(b % nbt) gpb, ... + gpb).
template <class S, int MODE, bool DAG, bool NORM, int PF>
__global__ void __launch_bounds__(128) hopq_kernel(const FastHop<S> a)
{
    const int nbt = (a.nrhs + a.gpb - 1) / a.gpb;
    int tile, gb;
    if (!block_tile(a.ntiles, nbt, a.swz, tile, gb)) return;
    const int j0 = gb * a.gpb;
    const int j1 = min(a.nrhs, j0 + a.gpb);
    for (int j = j0; j < j1; ++j) hopq_item<S, MODE, DAG, NORM, PF>(a, tile, j);
}

}  // namespace lqcd
