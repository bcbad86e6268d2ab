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

template <class S>
struct FastHop {
    int L[4];
    int Lxh, vh, nrhs, ntiles, parity;
    FastDiv dx, dy, dz;          // divide by Lx/2, Ly, Lz
    int oy, oz, ot;              // cb offsets of one step in y, z, t
    double coef;
    double th_re[4], th_im[4];
    int gpb;                     // groups of NR right-hand sides per block
    int theta_mask;              // bit mu set: theta_mu != 1
    SpinorField<S> in, self, out;
    LinkField<S> U;
    CloverField<S> clov;
    const RhsState *gate_st;
    int gate;
    Reduce red;
};

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
            if constexpr (MODE == HOP_CLOV) {
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
            n2 = store_raw<S, R>(a.out, jj[r], i, res);
        }
        if (NORM) reduce_finish(a.red, jj[r], tile, a.ntiles, n2);
    }
}

// Block b handles tile b / nbt and groups [(b % nbt) gpb, ... + gpb) of NR
// right-hand sides, nbt = ceil(groups / gpb); groups run one after another.
template <class S, int NR, int MODE, bool DAG, bool NORM>
__global__ void __launch_bounds__(128) hopf_kernel(const FastHop<S> a)
{
    const int ngr = (a.nrhs + NR - 1) / NR;
    const int nbt = (ngr + a.gpb - 1) / a.gpb;
    const int tile = blockIdx.x / nbt;
    const int g0 = (blockIdx.x % nbt) * a.gpb;
    const int g1 = min(ngr, g0 + a.gpb);
    for (int g = g0; g < g1; ++g) hopf_group<S, NR, MODE, DAG, NORM>(a, tile, g);
}

}  // namespace lqcd
