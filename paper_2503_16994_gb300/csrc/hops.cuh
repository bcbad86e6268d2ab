// Staged paired hopping kernel (FP16 storage, two right-hand sides per
// thread in packed FP32x2 lanes).  The words each direction needs (three
// spinor words of each right-hand side, the reconstruct-12 link words and
// the two per-site scales) are copied by cp.async into slots of this
// thread's own shared memory PD directions before they are used, so the
// loads in flight occupy shared memory instead of registers.  Per lane the
// arithmetic is the paired kernel's (dir_words, hopp_epilogue), so both give
// the same bits.
#pragma once
#include "hopfast.cuh"

namespace lqcd {

constexpr int kStageWords = 8;  // 16-byte words per direction and thread

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// the link of load_link18<F16> from its two words
__device__ __forceinline__ void decode_link16(uint4 w, uint2 w2, float u[18])
{
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

// slot layout: word k of slot s of thread t at stage[(s * kStageWords + k) * blockDim.x + t]
//   k 0-2: spinor words of RHS ja at the neighbour; k 3-5: RHS jb
//   k 6: link word (rows 0-1, entries 0-3); k 7: link entries 4-5 (8 bytes), scale ja, scale jb
template <int D>
__device__ __forceinline__ void stage_issue(const FastHop<F16> &a, int ja, int jb, int i, int y, uint4 *stage,
                                            int slot)
{
    constexpr int MU = D / 2, DIR = (D & 1) ? -1 : 1;
    const long st = a.in.stride;
    const uint4 *pa = a.in.p + (long)ja * 3 * st + y;
    const uint4 *pb = a.in.p + (long)jb * 3 * st + y;
    const int par = DIR > 0 ? a.parity : (a.parity ^ 1);
    const long lq = (long)(par * 4 + MU) * a.U.stride + (DIR > 0 ? i : y);
    const unsigned ws = blockDim.x * 16u;
    const unsigned d = unsigned(__cvta_generic_to_shared(stage + slot * kStageWords * blockDim.x + threadIdx.x));
    cp_async16(d, pa);
    cp_async16(d + ws, pa + st);
    cp_async16(d + 2 * ws, pa + 2 * st);
    cp_async16(d + 3 * ws, pb);
    cp_async16(d + 4 * ws, pb + st);
    cp_async16(d + 5 * ws, pb + 2 * st);
    cp_async16(d + 6 * ws, a.U.p + lq);
    cp_async8(d + 7 * ws, a.U.p2 + lq);
    cp_async4(d + 7 * ws + 8, a.in.scale + (long)ja * st + y);
    cp_async4(d + 7 * ws + 12, a.in.scale + (long)jb * st + y);
    cp_async_commit();
}

template <int D, int SG>
__device__ __forceinline__ void stage_compute(const FastHop<F16> &a, const uint4 *stage, int slot, bool wrap,
                                              cp acc[12])
{
    constexpr int MU = D / 2, DIR = (D & 1) ? -1 : 1;
    constexpr int SP = DIR > 0 ? -SG : SG;
    const int nt = blockDim.x;
    const uint4 *s0 = stage + slot * kStageWords * nt + threadIdx.x;
    uint4 w[kStageWords];
#pragma unroll
    for (int k = 0; k < kStageWords; ++k) w[k] = s0[k * nt];
    __half2 wa[12], wb[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const __half2 *ha = reinterpret_cast<const __half2 *>(&w[k]);
        const __half2 *hb = reinterpret_cast<const __half2 *>(&w[3 + k]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            wa[4 * k + q] = ha[q];
            wb[4 * k + q] = hb[q];
        }
    }
    float u[18];
    decode_link16(w[6], make_uint2(w[7].x, w[7].y), u);
    dir_words<F16, MU, DIR, SP>(a, u, wa, wb, __uint_as_float(w[7].z), __uint_as_float(w[7].w), wrap, acc);
}

// direction D: issue direction D + PD (its slot was read by direction D - 1),
// wait for direction D's copies, compute it
template <int D, int PD, int SG>
__device__ __forceinline__ void stage_step(const FastHop<F16> &a, int ja, int jb, int i, const int (&nb)[8],
                                           unsigned wm, uint4 *stage, cp acc[12])
{
    if constexpr (D + PD < 8) stage_issue<D + PD>(a, ja, jb, i, nb[D + PD], stage, (D + PD) % (PD + 1));
    constexpr int last = D + PD < 8 ? D + PD : 7;  // newest group issued
    cp_async_wait<last - D>();
    stage_compute<D, SG>(a, stage, D % (PD + 1), (wm >> D) & 1, acc);
    if constexpr (D < 7) stage_step<D + 1, PD, SG>(a, ja, jb, i, nb, wm, stage, acc);
}

template <int PD, int SG, int D>
__device__ __forceinline__ void stage_prologue(const FastHop<F16> &a, int ja, int jb, int i, const int (&nb)[8],
                                               uint4 *stage)
{
    stage_issue<D>(a, ja, jb, i, nb[D], stage, D % (PD + 1));
    if constexpr (D + 1 < PD) stage_prologue<PD, SG, D + 1>(a, ja, jb, i, nb, stage);
}

template <int MODE, bool DAG, bool NORM, int PD>
__device__ __forceinline__ void hops_group(const FastHop<F16> &a, int tile, int g, uint4 *stage)
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
        int nb[8];
        unsigned wm = 0;
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
        constexpr int SG = DAG ? -1 : 1;
        stage_prologue<PD, SG, 0>(a, ja, jb, i, nb, stage);
        stage_step<0, PD, SG>(a, ja, jb, i, nb, wm, stage, acc);
    }
    hopp_epilogue<F16, MODE, NORM>(a, tile, i, valid, ja, on_a, jb, on_b, acc);
}

// bytes of dynamic shared memory per block of kBlock threads
constexpr int stage_bytes(int pd) { return (pd + 1) * kStageWords * 128 * 16; }

// Block b handles tile b / nbt and pair groups [(b % nbt) gpb, ... + gpb).
template <int MODE, bool DAG, bool NORM, int MINB, int PD>
__global__ void __launch_bounds__(128, MINB) hops_kernel(const FastHop<F16> a)
{
    extern __shared__ uint4 stage[];
    const int ngr = (a.nrhs + 1) / 2;
    const int nbt = (ngr + a.gpb - 1) / a.gpb;
    int tile, gb;
    if (!block_tile(a.ntiles, nbt, a.swz, tile, gb)) return;
    const int g0 = gb * a.gpb;
    const int g1 = min(ngr, g0 + a.gpb);
    for (int g = g0; g < g1; ++g) hops_group<MODE, DAG, NORM, PD>(a, tile, g, stage);
}

}  // namespace lqcd
