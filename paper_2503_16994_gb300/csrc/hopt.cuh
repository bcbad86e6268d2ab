// Tile hopping kernel (FP16 storage, two right-hand sides per thread in the
// lanes of packed FP32x2 instructions).  A block covers 32 consecutive output
// sites of one parity and NPW pairs of right-hand sides, one warp per pair
// (lane = site).  What the pairs of a tile share is prepared once per block in
// shared memory, ready to be used as FP32x2 operands:
//   * the 8 links of every site, decoded from FP16 reconstruct-12 (third row
//     completed), each complex entry stored as (re, re, im, im);
//   * the 72 clover reals of every output site, stored as (a, a, b, b).
// Each warp reads only its own pair's spinor words, copied by cp.async into
// the thread's own shared-memory slots PD directions before they are used.
// Per lane the arithmetic is the one of the paired kernels (spin projection on
// the stored half2 words, link product, boundary phase, accumulation with
// the per-site scale folded in, clover epilogue, FP16 store), and the norms
// are summed per 32 sites and combined four at a time like the 128-site
// blocks of the other shapes, so every kernel shape gives the same bits.
#pragma once
#include "hops.cuh"

namespace lqcd {

constexpr int kTileSites = 32;
constexpr int kTileMaxPairs = 6;  // warps per block at most (192 threads)

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

// Per-thread staging slots of the spinor words: slot q of thread t holds 7
// 16-byte words at stage[(q * 7 + k) * blockDim.x + t]: k 0-2 the words of
// RHS ja at the neighbour, 3-5 those of RHS jb, 6 the two scales (x, y).
constexpr int kTileSlotWords = 7;

// bytes of dynamic shared memory of a block of `threads` threads, PD directions staged ahead
constexpr int tile_smem_bytes(int threads, int pd)
{
    return int(sizeof(float4)) * (8 * 9 * kTileSites + 36 * kTileSites) + (pd + 1) * kTileSlotWords * 16 * threads;
}

struct TileShared {
    float4 u[8][9][kTileSites];  // link of direction d (0 +x, 1 -x, 2 +y, ...), entry 3a + b: (re, re, im, im)
    float4 c[36][kTileSites];    // clover reals (2q, 2q, 2q + 1, 2q + 1) of the output site
    uint4 stage[1];              // the staging slots follow
};

// copy the words of direction d of the pair (ja, jb) at neighbour y into slot `slot`
__device__ __forceinline__ void tile_issue(const SpinorField<F16> &f, int ja, int jb, int y, uint4 *stage, int slot)
{
    const long st = f.stride;
    const uint4 *pa = f.p + (long)ja * 3 * st + y;
    const uint4 *pb = f.p + (long)jb * 3 * st + y;
    const unsigned ws = blockDim.x * 16u;
    const unsigned dst = unsigned(__cvta_generic_to_shared(stage + slot * kTileSlotWords * blockDim.x + threadIdx.x));
    cp_async16(dst, pa);
    cp_async16(dst + ws, pa + st);
    cp_async16(dst + 2 * ws, pa + 2 * st);
    cp_async16(dst + 3 * ws, pb);
    cp_async16(dst + 4 * ws, pb + st);
    cp_async16(dst + 5 * ws, pb + 2 * st);
    cp_async4(dst + 6 * ws, f.scale + (long)ja * st + y);
    cp_async4(dst + 6 * ws + 4, f.scale + (long)jb * st + y);
    cp_async_commit();
}

// one direction of the pair from its staged words: the arithmetic of
// dir_words with the link from shared memory, one colour row at a time
template <int D, int SG>
__device__ __forceinline__ void tile_dir(const FastHop<F16> &a, const TileShared &sh, const uint4 *slot, int s,
                                         bool wrap, cp acc[12])
{
    constexpr int MU = D / 2, DIR = (D & 1) ? -1 : 1;
    constexpr int SP = DIR > 0 ? -SG : SG;
    const int nt = blockDim.x;
    __half2 wa[12], wb[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 xa = slot[k * nt], xb = slot[(3 + k) * nt];
        const __half2 *ha = reinterpret_cast<const __half2 *>(&xa);
        const __half2 *hb = reinterpret_cast<const __half2 *>(&xb);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            wa[4 * k + q] = ha[q];
            wb[4 * k + q] = hb[q];
        }
    }
    const uint4 xs = slot[6 * nt];
    const float sa = __uint_as_float(xs.x), sb = __uint_as_float(xs.y);
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
    const bool phase = wrap && ((a.theta_mask >> MU) & 1);
    const float2 sc = make_float2(sa, sb), nsc = make_float2(-sa, -sb);
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

// direction D: issue direction D + PD into the slot direction D - 1 used,
// wait for direction D's copies, compute it
template <int D, int PD, int SG>
__device__ __forceinline__ void tile_step(const FastHop<F16> &a, const TileShared &sh, uint4 *stage, int s, int ja,
                                          int jb, const int (&nb)[8], unsigned wm, cp acc[12])
{
    if constexpr (D + PD < 8) tile_issue(a.in, ja, jb, nb[D + PD], stage, (D + PD) % (PD + 1));
    constexpr int last = D + PD < 8 ? D + PD : 7;  // newest group issued
    cp_async_wait<last - D>();
    tile_dir<D, SG>(a, sh, stage + (D % (PD + 1)) * kTileSlotWords * blockDim.x + threadIdx.x, s, (wm >> D) & 1, acc);
    if constexpr (D < 7) tile_step<D + 1, PD, SG>(a, sh, stage, s, ja, jb, nb, wm, acc);
}

// Block b: 32-site tile b / nbt, pairs [(b % nbt) npw, ... + npw), npw = blockDim.x / 32.
// The grid covers 4 * ntiles 32-site tiles (ntiles counts 128-site tiles);
// tiles past the last site only write zero norm partials.  One barrier: the
// shared links and clover are decoded by the threads of their own site
// (warp w: directions w and w + 6, clover words w and w + 6) while the
// first PD directions of spinor words are already in flight.
template <int MODE, bool DAG, bool NORM, int MINB, int PD>
__global__ void __launch_bounds__(kTileSites * kTileMaxPairs, MINB) hopt_kernel(const FastHop<F16> a)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];
    TileShared &sh = *reinterpret_cast<TileShared *>(tile_smem);
    uint4 *const stage = sh.stage;
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
    // this thread's site (lanes past the last site take the tile's first site; nothing is stored for them)
    const int ic = valid ? i : i0;
    int nb[8];
    unsigned wm = 0;
    {
        const unsigned row = fdiv(unsigned(ic), a.dx);
        const int xh = ic - int(row) * a.Lxh;
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
        nb[2] = ic + (w ? -(a.L[1] - 1) * a.oy : a.oy);
        wm |= unsigned(w) << 2;
        w = y == 0;
        nb[3] = ic - (w ? -(a.L[1] - 1) * a.oy : a.oy);
        wm |= unsigned(w) << 3;
        w = z == a.L[2] - 1;
        nb[4] = ic + (w ? -(a.L[2] - 1) * a.oz : a.oz);
        wm |= unsigned(w) << 4;
        w = z == 0;
        nb[5] = ic - (w ? -(a.L[2] - 1) * a.oz : a.oz);
        wm |= unsigned(w) << 5;
        w = t == a.L[3] - 1;
        nb[6] = ic + (w ? -(a.L[3] - 1) * a.ot : a.ot);
        wm |= unsigned(w) << 6;
        w = t == 0;
        nb[7] = ic - (w ? -(a.L[3] - 1) * a.ot : a.ot);
        wm |= unsigned(w) << 7;
    }
    const bool active = on_a || on_b;
    if (active) {
#pragma unroll
        for (int d = 0; d < PD; ++d) tile_issue(a.in, ja, jb, nb[d], stage, d);
    }
    // links of this site: directions warp and warp + 6; clover words warp and warp + 6
    // (a block of fewer than 6 warps takes the rest in further rounds)
    for (int d = warp; d < 8; d += npw) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int par = fwd ? a.parity : (a.parity ^ 1);
        int idx = nb[0];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (e == d) idx = fwd ? ic : nb[e];
        const long lq = (long)(par * 4 + mu) * a.U.stride + idx;
        float u[18];
        decode_link16(__ldg(a.U.p + lq), __ldg(a.U.p2 + lq), u);
#pragma unroll
        for (int k = 0; k < 9; ++k) sh.u[d][k][s] = make_float4(u[2 * k], u[2 * k], u[2 * k + 1], u[2 * k + 1]);
    }
    for (int k = warp; k < 9; k += npw) {
        const uint4 w = __ldg(a.clov.p + ((long)a.parity * 9 + k) * a.clov.stride + ic);
        const __half2 *h = reinterpret_cast<const __half2 *>(&w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 v = __half22float2(h[q]);
            sh.c[4 * k + q][s] = make_float4(v.x, v.x, v.y, v.y);
        }
    }
    __syncthreads();
    if (!active) return;  // no barrier follows
    cp acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = cp{bc(0.f), bc(0.f)};
    constexpr int SG = DAG ? -1 : 1;
    tile_step<0, PD, SG>(a, sh, stage, s, ja, jb, nb, wm, acc);
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
            const long st = a.self.stride;
            const uint4 *pa = a.self.p + (long)ja * 3 * st + i;
            const uint4 *pb = a.self.p + (long)jb * 3 * st + i;
            uint4 wsa[3], wsb[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                wsa[k] = __ldg(pa + k * st);
                wsb[k] = __ldg(pb + k * st);
            }
            const float2 sc = make_float2(__ldg(a.self.scale + (long)ja * st + i), __ldg(a.self.scale + (long)jb * st + i));
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                cp sv[6];
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    const int q = 6 * blk + r;  // complex component 0..11: word q / 4, half2 q % 4
                    const __half2 ha = reinterpret_cast<const __half2 *>(&wsa[q / 4])[q % 4];
                    const __half2 hb = reinterpret_cast<const __half2 *>(&wsb[q / 4])[q % 4];
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
