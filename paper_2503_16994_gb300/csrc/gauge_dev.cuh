// Device helpers on FP64 links (3x3 complex matrices in the even-odd SoA
// layout): products, adjoints, neighbours and the clover field strength.
// Used by the clover construction and by the gauge flow and observables.
#pragma once
#include "kernels.cuh"

namespace lqcd {

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

// link U_mu(y); with an open time boundary the time links leaving the last
// slice are absent (zero)
__device__ __forceinline__ m3 link_xy(const Geom &g, const LinkField<F64> &U, const int y[4], int mu, bool open)
{
    if (open && mu == 3 && y[3] == g.L[3] - 1) {
        m3 z;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) z.m[i][j] = cd{0.0, 0.0};
        return z;
    }
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
__device__ __forceinline__ m3 field_strength(const Geom &g, const LinkField<F64> &U, const int x[4], int mu, int nu, bool open)
{
    int xpm[4], xpn[4], xmm[4], xmn[4], a[4], b[4], c[4];
    shift(g, x, mu, +1, xpm);
    shift(g, x, nu, +1, xpn);
    shift(g, x, mu, -1, xmm);
    shift(g, x, nu, -1, xmn);
    shift(g, xmm, nu, +1, a);  // x - mu + nu
    shift(g, xmm, nu, -1, b);  // x - mu - nu
    shift(g, xpm, nu, -1, c);  // x + mu - nu
    m3 Umx = link_xy(g, U, x, mu, open), Unx = link_xy(g, U, x, nu, open);
    m3 q = mm(mm(Umx, link_xy(g, U, xpm, nu, open)), mm(md(link_xy(g, U, xpn, mu, open)), md(Unx)));
    m3 t = mm(mm(Unx, md(link_xy(g, U, a, mu, open))), mm(md(link_xy(g, U, xmm, nu, open)), link_xy(g, U, xmm, mu, open)));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + t.m[i][j];
    t = mm(mm(md(link_xy(g, U, xmm, mu, open)), md(link_xy(g, U, b, nu, open))), mm(link_xy(g, U, b, mu, open), link_xy(g, U, xmn, nu, open)));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + t.m[i][j];
    t = mm(mm(md(link_xy(g, U, xmn, nu, open)), link_xy(g, U, xmn, mu, open)), mm(link_xy(g, U, c, nu, open), md(Umx)));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + t.m[i][j];
    m3 f;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f.m[i][j] = 0.125 * (q.m[i][j] - conj(q.m[j][i]));
    cd tr = (1.0 / 3.0) * (f.m[0][0] + f.m[1][1] + f.m[2][2]);
    for (int i = 0; i < 3; ++i) f.m[i][i] = f.m[i][i] - tr;
    return f;
}

// Per-slice sums in a fixed order: every block writes its chunk's sum, the
// last block of slice t to arrive adds the chunks in order and writes
// corr[(t - src_t) mod T].  counter[t] is zero between uses.
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

}  // namespace lqcd
