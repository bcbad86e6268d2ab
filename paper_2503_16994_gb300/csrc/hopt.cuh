// Tile hopping kernel (FP16 storage, two right-hand sides per thread in the
// lanes of packed FP32x2 instructions).  A block covers 32 consecutive output
// sites of one parity and NPW pairs of right-hand sides, one warp per pair
// (lane = site).  What the pairs of a tile share is prepared once per block in
// shared memory, ready to be used as FP32x2 operands:
//   * the neighbour cb indices of the 32 sites and their wrap bits;
//   * the 8 links of every site, decoded from FP16 reconstruct-12 (third row
//     completed), each complex entry stored as (re, re, im, im);
//   * the 72 clover reals of every output site, stored as (a, a, b, b).
// The warps then read only their own spinor words from global memory.  Per
// lane the arithmetic is the one of the paired kernels (spin projection on
// the stored half2 words, link product, boundary phase, accumulation with
// the per-site scale folded in, clover epilogue, FP16 store), and the norms
// are summed per 32 sites and combined four at a time like the 128-site
// blocks of the other shapes, so every kernel shape gives the same bits.
#pragma once
#include "hops.cuh"

namespace lqcd {

constexpr int kTileSites = 32;
constexpr int kTileMaxPairs = 6;  // warps per block at most (192 threads)

struct TileShared {
    float4 u[8][9][kTileSites];  // link of direction d (0 +x, 1 -x, 2 +y, ...), entry 3a + b: (re, re, im, im)
    float4 c[36][kTileSites];    // clover reals (2q, 2q, 2q + 1, 2q + 1) of the output site
    int nb[8][kTileSites];       // neighbour cb index per direction
    unsigned wm[kTileSites];     // bit d: the hop in direction d crosses the boundary
};

constexpr int tile_smem_bytes() { return int(sizeof(TileShared)); }

// Row a of g = U h or U^dag h for both lanes, U from shared memory (entry k
// at u[k * kTileSites]); the operations and their order are those of
// link_mul_u, one colour row at a time
template <bool DAGU>
__device__ __forceinline__ void link_row_tile(const float4 *u, int a, const cp h[2][3], cp &g0, cp &g1)
{
    cp acc0{bc(0.f), bc(0.f)}, acc1{bc(0.f), bc(0.f)};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int k = DAGU ? (3 * b + a) : (3 * a + b);
        const float4 e = u[k * kTileSites];
        const float2 ur = make_float2(e.x, e.y), ui = make_float2(e.z, e.w), nui = make_float2(-e.z, -e.w);
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

// out = A v for one Hermitian 6x6 block from shared memory (float4 q of the
// block at A[q * kTileSites]); the operations and their order are those of clov6_p
__device__ __forceinline__ void clov6_tile(const float4 *A, const cp *v, cp *o)
{
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const float4 dq = A[(r / 2) * kTileSites];
        const float2 d = (r & 1) ? make_float2(dq.z, dq.w) : make_float2(dq.x, dq.y);
        cp acc{p_mul(d, v[r].r), p_mul(d, v[r].i)};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (c == r) continue;
            const int lo = c > r ? r : c, hi = c > r ? c : r;
            const int q = 3 + (lo * 5 - (lo * (lo - 1)) / 2 + (hi - lo - 1));
            const float4 e = A[q * kTileSites];
            const float2 ur = make_float2(e.x, e.y);
            const float2 ui = c > r ? make_float2(e.z, e.w) : make_float2(-e.z, -e.w);
            const float2 nui = c > r ? make_float2(-e.z, -e.w) : make_float2(e.z, e.w);
            acc.r = p_fma(ur, v[c].r, acc.r);
            acc.r = p_fma(nui, v[c].i, acc.r);
            acc.i = p_fma(ur, v[c].i, acc.i);
            acc.i = p_fma(ui, v[c].r, acc.i);
        }
        o[r] = acc;
    }
}

// the words of one direction for the pair (ja, jb) at neighbour site y
struct TileWords {
    uint4 w[6];  // RHS ja planes 0-2, RHS jb planes 0-2
    float sa, sb;
};

__device__ __forceinline__ void tile_load(const SpinorField<F16> &f, int ja, int jb, int y, TileWords &t)
{
    const long st = f.stride;
    const uint4 *pa = f.p + (long)ja * 3 * st + y;
    const uint4 *pb = f.p + (long)jb * 3 * st + y;
    t.w[0] = __ldg(pa);
    t.w[1] = __ldg(pa + st);
    t.w[2] = __ldg(pa + 2 * st);
    t.w[3] = __ldg(pb);
    t.w[4] = __ldg(pb + st);
    t.w[5] = __ldg(pb + 2 * st);
    t.sa = __ldg(f.scale + (long)ja * st + y);
    t.sb = __ldg(f.scale + (long)jb * st + y);
}

// one direction of the pair: the arithmetic of dir_words with the link from shared memory
template <int D, int SG>
__device__ __forceinline__ void tile_dir(const FastHop<F16> &a, const TileShared &sh, int s, const TileWords &t,
                                         cp acc[12])
{
    constexpr int MU = D / 2, DIR = (D & 1) ? -1 : 1;
    constexpr int SP = DIR > 0 ? -SG : SG;
    __half2 wa[12], wb[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const __half2 *ha = reinterpret_cast<const __half2 *>(&t.w[k]);
        const __half2 *hb = reinterpret_cast<const __half2 *>(&t.w[3 + k]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            wa[4 * k + q] = ha[q];
            wb[4 * k + q] = hb[q];
        }
    }
    cp h[2][3];
    __half2 ha[2][3], hb[2][3];
    project_h<MU, SP>(wa, ha);
    project_h<MU, SP>(wb, hb);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            h[q][c] = cp{make_float2(__low2float(ha[q][c]), __low2float(hb[q][c])),
                         make_float2(__high2float(ha[q][c]), __high2float(hb[q][c]))};
    const bool phase = ((sh.wm[s] >> D) & 1) && ((a.theta_mask >> MU) & 1);
    const float2 sc = make_float2(t.sa, t.sb), nsc = make_float2(-t.sa, -t.sb);
    const float4 *u = &sh.u[D][0][s];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cp g0, g1;
        link_row_tile<(DIR < 0)>(u, c, h, g0, g1);
        if (phase) {
            const float2 pr = bc(float(a.th_re[MU])), pi = bc(DIR > 0 ? float(a.th_im[MU]) : float(-a.th_im[MU]));
            const float2 npi = bc(DIR > 0 ? float(-a.th_im[MU]) : float(a.th_im[MU]));
            g0 = cp{p_fma(npi, g0.i, p_mul(pr, g0.r)), p_fma(pi, g0.r, p_mul(pr, g0.i))};
            g1 = cp{p_fma(npi, g1.i, p_mul(pr, g1.r)), p_fma(pi, g1.r, p_mul(pr, g1.i))};
        }
        accumulate_row<MU, SP>(acc, c, g0, g1, sc, nsc);
    }
}

// the 8 directions; PF: the words of direction D + 1 are loaded before direction D is computed
template <int D, int SG, bool PF>
__device__ __forceinline__ void tile_dirs(const FastHop<F16> &a, const TileShared &sh, int s, int ja, int jb,
                                          TileWords &cur, cp acc[12])
{
    if constexpr (PF) {
        TileWords nxt;
        if constexpr (D < 7) tile_load(a.in, ja, jb, sh.nb[D + 1][s], nxt);
        tile_dir<D, SG>(a, sh, s, cur, acc);
        if constexpr (D < 7) tile_dirs<D + 1, SG, PF>(a, sh, s, ja, jb, nxt, acc);
    } else {
        tile_dir<D, SG>(a, sh, s, cur, acc);
        if constexpr (D < 7) {
            tile_load(a.in, ja, jb, sh.nb[D + 1][s], cur);
            tile_dirs<D + 1, SG, PF>(a, sh, s, ja, jb, cur, acc);
        }
    }
}

// Block b: 32-site tile b / nbt, pairs [(b % nbt) npw, ... + npw), npw = blockDim.x / 32.
// The grid covers 4 * ntiles 32-site tiles (ntiles counts 128-site tiles);
// tiles past the last site only write zero norm partials.
template <int MODE, bool DAG, bool NORM, int MINB, bool PF>
__global__ void __launch_bounds__(kTileSites * kTileMaxPairs, MINB) hopt_kernel(const FastHop<F16> a)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];
    TileShared &sh = *reinterpret_cast<TileShared *>(tile_smem);
    const int npairs = (a.nrhs + 1) / 2;
    const int npw = blockDim.x / kTileSites;
    const int nbt = (npairs + npw - 1) / npw;
    const int tile = blockIdx.x / nbt;
    const int warp = threadIdx.x / kTileSites, s = threadIdx.x % kTileSites;
    const int g = (blockIdx.x % nbt) * npw + warp;
    const int i0 = tile * kTileSites;
    const int i = i0 + s;
    const bool valid = i < a.vh;
    const int ja0 = 2 * g, jb0 = 2 * g + 1;
    const bool on_a = g < npairs && ja0 < a.nrhs && (!a.gate_st || a.gate_st[ja0].status == a.gate);
    const bool on_b = g < npairs && jb0 < a.nrhs && (!a.gate_st || a.gate_st[jb0].status == a.gate);
    const int ja = min(ja0, a.nrhs - 1), jb = min(jb0, a.nrhs - 1);
    float *const pf = a.red.partial_f;
    const long ntiles32 = 4L * a.ntiles;
    if (i0 >= a.vh) {  // padding tile: zero partials keep the four-tile groups complete
        if (NORM && s == 0) {
            if (on_a) pf[(long)ja * ntiles32 + tile] = 0.f;
            if (on_b) pf[(long)jb * ntiles32 + tile] = 0.f;
        }
        return;
    }
    // every warp of the block takes part in the preparation, whatever its pair
    if (warp == 0) {
        int nb[8];
        unsigned wm = 0;
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
            bool w;
            w = x == a.L[0] - 1;
            nb[0] = rowbase + ((w ? 0 : x + 1) >> 1);
            wm |= unsigned(w) << 0;
            w = x == 0;
            nb[1] = rowbase + ((w ? a.L[0] - 1 : x - 1) >> 1);
            wm |= unsigned(w) << 1;
            w = y == a.L[1] - 1;
            nb[2] = i + (w ? -(a.L[1] - 1) * a.oy : a.oy);
            wm |= unsigned(w) << 2;
            w = y == 0;
            nb[3] = i - (w ? -(a.L[1] - 1) * a.oy : a.oy);
            wm |= unsigned(w) << 3;
            w = z == a.L[2] - 1;
            nb[4] = i + (w ? -(a.L[2] - 1) * a.oz : a.oz);
            wm |= unsigned(w) << 4;
            w = z == 0;
            nb[5] = i - (w ? -(a.L[2] - 1) * a.oz : a.oz);
            wm |= unsigned(w) << 5;
            w = t == a.L[3] - 1;
            nb[6] = i + (w ? -(a.L[3] - 1) * a.ot : a.ot);
            wm |= unsigned(w) << 6;
            w = t == 0;
            nb[7] = i - (w ? -(a.L[3] - 1) * a.ot : a.ot);
            wm |= unsigned(w) << 7;
        } else {
#pragma unroll
            for (int d = 0; d < 8; ++d) nb[d] = i0;  // a valid site; its results are not stored
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) sh.nb[d][s] = nb[d];
        sh.wm[s] = wm;
    }
    // clover of the output sites: word k (8 halves) of site s -> float4 4k .. 4k + 3
    for (int task = threadIdx.x; task < 9 * kTileSites; task += blockDim.x) {
        const int k = task / kTileSites, ss = task % kTileSites;
        const int ii = min(i0 + ss, a.vh - 1);
        const uint4 w = __ldg(a.clov.p + ((long)a.parity * 9 + k) * a.clov.stride + ii);
        const __half2 *h = reinterpret_cast<const __half2 *>(&w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 v = __half22float2(h[q]);
            sh.c[4 * k + q][ss] = make_float4(v.x, v.x, v.y, v.y);
        }
    }
    __syncthreads();
    // links: direction d of site ss, decoded once for all pairs of the block
    for (int task = threadIdx.x; task < 8 * kTileSites; task += blockDim.x) {
        const int d = task / kTileSites, ss = task % kTileSites;
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int ii = min(i0 + ss, a.vh - 1);
        const int par = fwd ? a.parity : (a.parity ^ 1);
        const long lq = (long)(par * 4 + mu) * a.U.stride + (fwd ? ii : sh.nb[d][ss]);
        float u[18];
        decode_link16(__ldg(a.U.p + lq), __ldg(a.U.p2 + lq), u);
#pragma unroll
        for (int k = 0; k < 9; ++k) sh.u[d][k][ss] = make_float4(u[2 * k], u[2 * k], u[2 * k + 1], u[2 * k + 1]);
    }
    __syncthreads();
    if (!on_a && !on_b) return;  // no block-wide barrier follows
    cp acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = cp{bc(0.f), bc(0.f)};
    constexpr int SG = DAG ? -1 : 1;
    if (valid) {
        TileWords cur;
        tile_load(a.in, ja, jb, sh.nb[0][s], cur);
        tile_dirs<0, SG, PF>(a, sh, s, ja, jb, cur, acc);
    }
    float n2a = 0.f, n2b = 0.f;
    if (valid) {
        cp res[12];
        const float2 cf = bc(float(a.coef));
        if constexpr (MODE == HOP_CLOV) {
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) clov6_tile(&sh.c[18 * blk][s], acc + 6 * blk, res + 6 * blk);
#pragma unroll
            for (int q = 0; q < 12; ++q) res[q] = cp{p_mul(cf, res[q].r), p_mul(cf, res[q].i)};
        } else {
            // the arithmetic of hopp_epilogue (load_pair, scale, clov6_p, fma), one clover block at a time
            TileWords t;
            tile_load(a.self, ja, jb, i, t);
            const float2 sc = make_float2(t.sa, t.sb);
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                cp sv[6];
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    const int q = 6 * blk + r;  // complex component 0..11: word q / 4, half2 q % 4
                    const __half2 ha = reinterpret_cast<const __half2 *>(&t.w[q / 4])[q % 4];
                    const __half2 hb = reinterpret_cast<const __half2 *>(&t.w[3 + q / 4])[q % 4];
                    const cp v{__half22float2(__lows2half2(ha, hb)), __half22float2(__highs2half2(ha, hb))};
                    sv[r] = cp{p_mul(v.r, sc), p_mul(v.i, sc)};
                }
                clov6_tile(&sh.c[18 * blk][s], sv, res + 6 * blk);
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
        if (on_a) n2a = float(store_raw<F16, float>(a.out, ja, i, va));
        if (on_b) n2b = float(store_raw<F16, float>(a.out, jb, i, vb));
    }
    if (NORM) {
        // the 32-site sums of reduce_partial2's warps; partial_finish combines them four at a time
        n2a = warp_sum_t(n2a);
        n2b = warp_sum_t(n2b);
        if (s == 0) {
            if (on_a) pf[(long)ja * ntiles32 + tile] = n2a;
            if (on_b) pf[(long)jb * ntiles32 + tile] = n2b;
        }
    }
}

}  // namespace lqcd
