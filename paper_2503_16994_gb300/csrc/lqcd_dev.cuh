// Device-side building blocks for the Wilson-clover kernels (sm_103a).
//
// Layout in HBM (one lattice, V sites, Vh = V/2 per parity):
//   * sites are split by parity p = (x+y+z+t) & 1 and numbered within a parity
//     by cb = lex >> 1 (lex = x + Lx (y + Ly (z + Lz t)); Lx is even, so the
//     pair (x, x+1) shares cb);
//   * every field is structure-of-arrays: "planes" of vector words, one word
//     per site, plane k of a field holding reals [k W, (k+1) W) of the site's
//     real stream (W = 2 for double2, 4 for float4, 8 for 8 halves in a
//     uint4); consecutive threads read consecutive words, so every load is a
//     coalesced 16-byte access;
//   * planes are `stride` words long (Vh rounded up to a multiple of 64);
//     right-hand side j of a multi-RHS field starts at plane j * planes.
// Real streams:
//   spinor : 24 reals, complex component 3 spin + colour;
//   link   : FP64 all 18 reals (row-major 3x3); FP32/FP16 reconstruct-12:
//            rows 0 and 1 (12 reals), row 2 rebuilt as conj(row0 x row1);
//   clover : two Hermitian 6x6 chirality blocks (upper spins 0,1 then lower
//            spins 2,3), each 36 reals: 6 real diagonal entries, then the 15
//            complex entries above the diagonal, row by row.
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

namespace lqcd {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
    R re, im;
};

template <typename R> __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
// i * a
template <typename R> __device__ __forceinline__ cx<R> mul_i(cx<R> a) { return {-a.im, a.re}; }
// conj(a) * b
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b)
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R> __device__ __forceinline__ R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------------------
// colour matrices, spinors
// ---------------------------------------------------------------------------
template <typename R> struct su3 { cx<R> m[3][3]; };
template <typename R> struct spinor { cx<R> s[4][3]; };      // [spin][colour]
template <typename R> struct hspinor { cx<R> s[2][3]; };     // projected two-spinor

template <typename R> __device__ __forceinline__ void zero(spinor<R> &a)
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.s[i][c] = cx<R>{R(0), R(0)};
}

// v = U h (both spin components)
template <typename R> __device__ __forceinline__ hspinor<R> mul(const su3<R> &U, const hspinor<R> &h)
{
    hspinor<R> r;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) r.s[s][a] = U.m[a][0] * h.s[s][0] + U.m[a][1] * h.s[s][1] + U.m[a][2] * h.s[s][2];
    return r;
}

// v = U^dag h
template <typename R> __device__ __forceinline__ hspinor<R> mul_dag(const su3<R> &U, const hspinor<R> &h)
{
    hspinor<R> r;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            r.s[s][a] = cmul(U.m[0][a], h.s[s][0]) + cmul(U.m[1][a], h.s[s][1]) + cmul(U.m[2][a], h.s[s][2]);
    return r;
}

// ---------------------------------------------------------------------------
// spin projection in the chiral basis
//
// g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, -1], [-1, 0]] in 2x2 spin
// blocks (up = spins 0,1; dn = spins 2,3).  For sign s = +1 or -1,
//   (1 + s g_k) psi = (h, s i s_k h)  with h = up - s i s_k dn,
//   (1 + s g_t) psi = (h, -s h)       with h = up - s dn,
// since (i s_k)^2 = -1.  So the 4-spinor is carried as the two-spinor h
// through the colour multiplication and rebuilt afterwards.
// i s_x (a, b) = (i b, i a); i s_y (a, b) = (b, -a); i s_z (a, b) = (i a, -i b).
// ---------------------------------------------------------------------------
template <typename R, int MU>
__device__ __forceinline__ void isigma(const cx<R> a[3], const cx<R> b[3], cx<R> oa[3], cx<R> ob[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) { oa[c] = mul_i(b[c]); ob[c] = mul_i(a[c]); }
        if (MU == 1) { oa[c] = b[c]; ob[c] = -a[c]; }
        if (MU == 2) { oa[c] = mul_i(a[c]); ob[c] = -mul_i(b[c]); }
    }
}

template <typename R, int MU, int S>
__device__ __forceinline__ hspinor<R> project(const spinor<R> &p)
{
    hspinor<R> h;
    if (MU == 3) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) h.s[s][c] = (S > 0) ? p.s[s][c] - p.s[2 + s][c] : p.s[s][c] + p.s[2 + s][c];
    } else {
        cx<R> ta[3], tb[3];
        isigma<R, MU>(p.s[2], p.s[3], ta, tb);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h.s[0][c] = (S > 0) ? p.s[0][c] - ta[c] : p.s[0][c] + ta[c];
            h.s[1][c] = (S > 0) ? p.s[1][c] - tb[c] : p.s[1][c] + tb[c];
        }
    }
    return h;
}

// acc += (1 + S g_mu) psi given its projection h
template <typename R, int MU, int S>
__device__ __forceinline__ void accumulate(spinor<R> &acc, const hspinor<R> &h)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc.s[s][c] = acc.s[s][c] + h.s[s][c];
    if (MU == 3) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc.s[2 + s][c] = (S > 0) ? acc.s[2 + s][c] - h.s[s][c] : acc.s[2 + s][c] + h.s[s][c];
    } else {
        cx<R> ta[3], tb[3];
        isigma<R, MU>(h.s[0], h.s[1], ta, tb);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc.s[2][c] = (S > 0) ? acc.s[2][c] + ta[c] : acc.s[2][c] - ta[c];
            acc.s[3][c] = (S > 0) ? acc.s[3][c] + tb[c] : acc.s[3][c] - tb[c];
        }
    }
}

template <typename R> __device__ __forceinline__ void scale_h(hspinor<R> &h, cx<R> ph)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) h.s[s][c] = ph * h.s[s][c];
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Geom {
    int L[4];     // Lx, Ly, Lz, T
    int Lxh;      // Lx / 2
    int vh;       // sites per parity
    long stride;  // words per plane
};

// coordinates of site cb of parity p
__device__ __forceinline__ void cb_coords(const Geom &g, int p, int cb, int x[4])
{
    int r = cb / g.Lxh;
    int xh = cb - r * g.Lxh;
    x[1] = r % g.L[1];
    r /= g.L[1];
    x[2] = r % g.L[2];
    x[3] = r / g.L[2];
    x[0] = 2 * xh + ((p + x[1] + x[2] + x[3]) & 1);
}

__device__ __forceinline__ int cb_index(const Geom &g, const int x[4])
{
    return (x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]))) >> 1;
}

// cb index of the site x + dir * mu (periodic wrap)
__device__ __forceinline__ int cb_neighbour(const Geom &g, const int x[4], int mu, int dir)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    int v = y[mu] + dir;
    if (v < 0) v += g.L[mu];
    if (v >= g.L[mu]) v -= g.L[mu];
    y[mu] = v;
    return cb_index(g, y);
}

// ---------------------------------------------------------------------------
// storage formats
// ---------------------------------------------------------------------------
struct F64 { using word = double2; static constexpr int W = 2; };
struct F32 { using word = float4; static constexpr int W = 4; };
struct F16 { using word = uint4; static constexpr int W = 8; };

// A spinor field (one parity, nrhs right-hand sides).  `scale` is used by F16
// only: per-site FP32 scale (one float per site and RHS, plane of `stride`).
template <class S>
struct SpinorField {
    typename S::word *p;
    float *scale;
    long stride;
};

template <class S> struct spinor_planes { static constexpr int n = 24 / S::W; };

__device__ __forceinline__ void unpack_h8(uint4 w, float sc, float *o)
{
    const __half2 *h = reinterpret_cast<const __half2 *>(&w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __half22float2(h[k]);
        o[2 * k] = f.x * sc;
        o[2 * k + 1] = f.y * sc;
    }
}

__device__ __forceinline__ uint4 pack_h8(const float *v, float inv)
{
    uint4 w;
    __half2 *h = reinterpret_cast<__half2 *>(&w);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(v[2 * k] * inv, v[2 * k + 1] * inv);
    return w;
}

// load the 24 reals of site i, right-hand side j
template <class S, typename R>
__device__ __forceinline__ spinor<R> load_spinor(const SpinorField<S> &f, int j, int i)
{
    spinor<R> a;
    R *v = reinterpret_cast<R *>(&a);
    constexpr int NP = spinor_planes<S>::n;
    const typename S::word *b = f.p + (long)j * NP * f.stride + i;
    if constexpr (sizeof(typename S::word) == 16 && S::W == 2) {  // F64
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            double2 w = __ldg(b + k * f.stride);
            v[2 * k] = R(w.x);
            v[2 * k + 1] = R(w.y);
        }
    } else if constexpr (S::W == 4) {  // F32
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float4 w = __ldg(b + k * f.stride);
            v[4 * k] = R(w.x);
            v[4 * k + 1] = R(w.y);
            v[4 * k + 2] = R(w.z);
            v[4 * k + 3] = R(w.w);
        }
    } else {  // F16
        float sc = __ldg(f.scale + (long)j * f.stride + i);
        float t[8];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            unpack_h8(__ldg(b + k * f.stride), sc, t);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[8 * k + q] = R(t[q]);
        }
    }
    return a;
}

// store; returns the squared norm of the value actually stored
template <class S, typename R>
__device__ __forceinline__ double store_spinor(const SpinorField<S> &f, int j, int i, const spinor<R> &a)
{
    const R *v = reinterpret_cast<const R *>(&a);
    constexpr int NP = spinor_planes<S>::n;
    typename S::word *b = f.p + (long)j * NP * f.stride + i;
    double n2 = 0;
    if constexpr (S::W == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            double2 w = make_double2(double(v[2 * k]), double(v[2 * k + 1]));
            b[k * f.stride] = w;
            n2 += w.x * w.x + w.y * w.y;
        }
    } else if constexpr (S::W == 4) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float4 w = make_float4(float(v[4 * k]), float(v[4 * k + 1]), float(v[4 * k + 2]), float(v[4 * k + 3]));
            b[k * f.stride] = w;
            acc += w.x * w.x + w.y * w.y + w.z * w.z + w.w * w.w;
        }
        n2 = acc;
    } else {
        float mx = 0.f;
        float fv[24];
#pragma unroll
        for (int q = 0; q < 24; ++q) {
            fv[q] = float(v[q]);
            mx = fmaxf(mx, fabsf(fv[q]));
        }
        // Sites whose largest component is below 1e-30 are stored as zero:
        // the exponentially decaying point-source propagator leaves FP32
        // denormals far from the source, where 1/mx would overflow.
        if (!(mx >= 1e-30f)) mx = 0.f;
        float inv = mx > 0.f ? 1.0f / mx : 0.f;
        f.scale[(long)j * f.stride + i] = mx;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            uint4 w = pack_h8(fv + 8 * k, inv);
            b[k * f.stride] = w;
            float t[8];
            unpack_h8(w, mx, t);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc += t[q] * t[q];
        }
        n2 = acc;
    }
    return n2;
}

// ---------------------------------------------------------------------------
// links
// ---------------------------------------------------------------------------
// Gauge field in one storage format: planes indexed [parity][mu][plane].
template <class S>
struct LinkField {
    const typename S::word *p;   // F64: 9 planes; F32: 3 planes; F16: 1 plane of 8 halves
    const uint2 *p2;             // F16 only: 1 plane of 4 halves (entries 4, 5 of rows 0-1)
    long stride;
};

template <typename R>
__device__ __forceinline__ void reconstruct_row2(su3<R> &U)
{
    // row2 = conj(row0 x row1) for a special unitary matrix
    U.m[2][0] = conj(U.m[0][1] * U.m[1][2] - U.m[0][2] * U.m[1][1]);
    U.m[2][1] = conj(U.m[0][2] * U.m[1][0] - U.m[0][0] * U.m[1][2]);
    U.m[2][2] = conj(U.m[0][0] * U.m[1][1] - U.m[0][1] * U.m[1][0]);
}

template <class S, typename R>
__device__ __forceinline__ su3<R> load_link(const LinkField<S> &f, int parity, int mu, int i)
{
    su3<R> U;
    if constexpr (S::W == 2) {
        const double2 *b = f.p + (long)(parity * 4 + mu) * 9 * f.stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 w = __ldg(b + k * f.stride);
            U.m[k / 3][k % 3] = cx<R>{R(w.x), R(w.y)};
        }
    } else if constexpr (S::W == 4) {
        const float4 *b = f.p + (long)(parity * 4 + mu) * 3 * f.stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 w = __ldg(b + k * f.stride);
            int e0 = 2 * k, e1 = 2 * k + 1;
            U.m[e0 / 3][e0 % 3] = cx<R>{R(w.x), R(w.y)};
            U.m[e1 / 3][e1 % 3] = cx<R>{R(w.z), R(w.w)};
        }
        reconstruct_row2(U);
    } else {
        uint4 w = __ldg(f.p + (long)(parity * 4 + mu) * f.stride + i);
        uint2 w2 = __ldg(f.p2 + (long)(parity * 4 + mu) * f.stride + i);
        const __half2 *h = reinterpret_cast<const __half2 *>(&w);
        const __half2 *h2 = reinterpret_cast<const __half2 *>(&w2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float2 v = __half22float2(h[e]);
            U.m[e / 3][e % 3] = cx<R>{R(v.x), R(v.y)};
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float2 v = __half22float2(h2[e]);
            U.m[(e + 4) / 3][(e + 4) % 3] = cx<R>{R(v.x), R(v.y)};
        }
        reconstruct_row2(U);
    }
    return U;
}

// ---------------------------------------------------------------------------
// clover blocks
// ---------------------------------------------------------------------------
template <class S>
struct CloverField {
    const typename S::word *p;  // [parity][72 / W planes]
    long stride;
};

template <typename R> struct clover_block { R d[6]; cx<R> o[15]; };

__device__ __forceinline__ int tri(int i, int j)  // i < j, index into the 15 upper entries
{
    return i * 5 - (i * (i - 1)) / 2 + (j - i - 1);
}

template <class S, typename R>
__device__ __forceinline__ void load_clover(const CloverField<S> &f, int parity, int i, clover_block<R> blk[2])
{
    R *v = reinterpret_cast<R *>(blk);  // 72 reals: d[6], o[15] x2 (layout matches the stream)
    constexpr int NP = 72 / S::W;
    const typename S::word *b = f.p + (long)parity * NP * f.stride + i;
    if constexpr (S::W == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            double2 w = __ldg(b + k * f.stride);
            v[2 * k] = R(w.x);
            v[2 * k + 1] = R(w.y);
        }
    } else if constexpr (S::W == 4) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float4 w = __ldg(b + k * f.stride);
            v[4 * k] = R(w.x);
            v[4 * k + 1] = R(w.y);
            v[4 * k + 2] = R(w.z);
            v[4 * k + 3] = R(w.w);
        }
    } else {
        float t[8];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            unpack_h8(__ldg(b + k * f.stride), 1.0f, t);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[8 * k + q] = R(t[q]);
        }
    }
}

// out = A v for one 6x6 Hermitian block; v, out indexed 3 s + a (s = 0, 1)
template <typename R>
__device__ __forceinline__ void clover_mul6(const clover_block<R> &A, const cx<R> v[6], cx<R> out[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        cx<R> acc = A.d[i] * v[i];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            if (j > i) acc = acc + A.o[tri(i, j)] * v[j];
            if (j < i) acc = acc + cmul(A.o[tri(j, i)], v[j]);
        }
        out[i] = acc;
    }
}

template <typename R>
__device__ __forceinline__ spinor<R> clover_apply(const clover_block<R> blk[2], const spinor<R> &a)
{
    spinor<R> r;
    const cx<R> *in = &a.s[0][0];
    cx<R> *out = &r.s[0][0];
    clover_mul6(blk[0], in, out);
    clover_mul6(blk[1], in + 6, out + 6);
    return r;
}

// ---------------------------------------------------------------------------
// reductions: per-block FP64 partials, finished by the last block
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block (result valid in thread 0).  `sh` holds 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}

}  // namespace lqcd
