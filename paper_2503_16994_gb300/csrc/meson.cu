// Meson two-point functions for arbitrary spin matrices G, from the 12
// columns of a point-source propagator in the host layout (the correlation
// functions Sec. 3.3 leaves to the user of the propagator):
//
//   C_G(t) = - sum_xvec tr[ (G x 1) S(x) (Gbar x 1) g5 S(x)^dag g5 ],
//   Gbar = g_t G^dag g_t,  x = (xvec, src_t + t mod T).
//
// Writing S_{ad} for the 3x3 colour block of sink spin a and source spin d,
// the trace is a sum over spin indices of coefficients times colour inner
// products:
//   C_G = sum_{a,b,c,d} k_abcd <S_ad, S_bc>,  k_abcd = - G_ab Gbar_cd g5_d g5_a,
//   <A, B> = sum_ij conj(A_ij) B_ij.
// The host turns each G into its list of nonzero k (16 for a Clifford basis
// element, at most 256), and the kernel evaluates 9 complex products per
// term in FP64, one thread per site.
#include <vector>

#include "lqcd_impl.h"

namespace lqcd {

struct MesonTerm {
    int p, q;       // p = 4 a + d, q = 4 b + c
    double re, im;  // k_abcd
};

// chiral basis (spin index 0-3): g_t = [[0, -1], [-1, 0]] in 2x2 blocks, g5 = diag(1, 1, -1, -1)
static double gt_host(int a, int b) { return (a == b + 2 || b == a + 2) ? -1.0 : 0.0; }
static double g5_host(int a) { return a < 2 ? 1.0 : -1.0; }

// block (c, t): sites [c 128, (c + 1) 128) of slice t; partial[(t ng + g) nchunk + c] = (re, im)
__global__ void __launch_bounds__(128) meson_kernel(long V, long v3, int ng, const double2 *prop,
                                                    const MesonTerm *terms, const int *off, double2 *partial)
{
    __shared__ double sh[2][32];
    const int t = blockIdx.y, c = blockIdx.x, nchunk = gridDim.x;
    const long i = (long)c * blockDim.x + threadIdx.x;
    const bool valid = i < v3;
    const long x = (long)t * v3 + i;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int g = 0; g < ng; ++g) {
        double ar = 0.0, ai = 0.0;
        if (valid) {
            for (int k = off[g]; k < off[g + 1]; ++k) {
                const MesonTerm m = terms[k];
                const int a = m.p >> 2, d = m.p & 3, b = m.q >> 2, cs = m.q & 3;
                // <S_ad, S_bc> = sum_{u,v} conj(S[3a+u][3d+v]) S[3b+u][3c+v], S[i][j] = prop[j][x][i]
                double sr = 0.0, si = 0.0;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const double2 *pa = prop + ((long)(3 * d + v) * V + x) * 12 + 3 * a;
                    const double2 *pb = prop + ((long)(3 * cs + v) * V + x) * 12 + 3 * b;
#pragma unroll
                    for (int u = 0; u < 3; ++u) {
                        const double2 A = __ldg(pa + u), B = __ldg(pb + u);
                        sr = fma(A.x, B.x, fma(A.y, B.y, sr));
                        si = fma(A.x, B.y, fma(-A.y, B.x, si));
                    }
                }
                ar = fma(m.re, sr, fma(-m.im, si, ar));
                ai = fma(m.re, si, fma(m.im, sr, ai));
            }
        }
        ar = warp_sum(ar);
        ai = warp_sum(ai);
        __syncthreads();
        if (lane == 0) {
            sh[0][wid] = ar;
            sh[1][wid] = ai;
        }
        __syncthreads();
        if (wid == 0) {
            ar = warp_sum(lane < nw ? sh[0][lane] : 0.0);
            ai = warp_sum(lane < nw ? sh[1][lane] : 0.0);
            if (lane == 0) partial[((long)t * ng + g) * nchunk + c] = make_double2(ar, ai);
        }
    }
}

// corr[g T + (t - src_t) mod T] = sum of the chunks of (t, g), fixed order; one block per (t, g)
__global__ void __launch_bounds__(128) meson_finish_kernel(int T, int ng, int nchunk, int src_t,
                                                           const double2 *partial, double2 *corr)
{
    __shared__ double sh[32];
    const int t = blockIdx.x / ng, g = blockIdx.x % ng;
    double sr = 0.0, si = 0.0;
    for (int k = threadIdx.x; k < nchunk; k += blockDim.x) {
        const double2 v = partial[((long)t * ng + g) * nchunk + k];
        sr += v.x;
        si += v.y;
    }
    sr = block_sum(sr, sh);
    __syncthreads();
    si = block_sum(si, sh);
    if (threadIdx.x == 0) corr[(long)g * T + ((t - src_t) % T + T) % T] = make_double2(sr, si);
}

void meson_contract(lqcd_lattice_s *lat, const double *prop_dev, int src_t, const double *gammas, int ng,
                    double *corr_dev, cudaStream_t st)
{
    // host: term lists
    std::vector<MesonTerm> terms;
    std::vector<int> off(1, 0);
    for (int g = 0; g < ng; ++g) {
        double G[4][4][2], Gb[4][4][2];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                G[a][b][0] = gammas[2 * (16 * g + 4 * a + b)];
                G[a][b][1] = gammas[2 * (16 * g + 4 * a + b) + 1];
            }
        // Gbar = g_t G^dag g_t: (g_t)_{aa'} conj(G_{b'a'}) (g_t)_{b'b}
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                double re = 0.0, im = 0.0;
                for (int a2 = 0; a2 < 4; ++a2)
                    for (int b2 = 0; b2 < 4; ++b2) {
                        const double w = gt_host(a, a2) * gt_host(b2, b);
                        re += w * G[b2][a2][0];
                        im -= w * G[b2][a2][1];
                    }
                Gb[a][b][0] = re;
                Gb[a][b][1] = im;
            }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                for (int c = 0; c < 4; ++c)
                    for (int d = 0; d < 4; ++d) {
                        // k = - G_ab Gbar_cd g5_d g5_a
                        const double s = -g5_host(d) * g5_host(a);
                        const double re = s * (G[a][b][0] * Gb[c][d][0] - G[a][b][1] * Gb[c][d][1]);
                        const double im = s * (G[a][b][0] * Gb[c][d][1] + G[a][b][1] * Gb[c][d][0]);
                        if (re != 0.0 || im != 0.0) terms.push_back(MesonTerm{4 * a + d, 4 * b + c, re, im});
                    }
        off.push_back(int(terms.size()));
    }
    const int T = lat->dims[3];
    const long v3 = lat->V / T;
    const int nchunk = int((v3 + kBlock - 1) / kBlock);
    const size_t tbytes = sizeof(MesonTerm) * std::max<size_t>(terms.size(), 1);
    const size_t obytes = sizeof(int) * off.size();
    const size_t pbytes = sizeof(double2) * (size_t)T * ng * nchunk;
    void *buf = nullptr;
    LQCD_CUDA(cudaMallocAsync(&buf, tbytes + obytes + pbytes + 64, st));
    char *b = static_cast<char *>(buf);
    MesonTerm *dterms = reinterpret_cast<MesonTerm *>(b);
    int *doff = reinterpret_cast<int *>(b + tbytes);
    double2 *dpart = reinterpret_cast<double2 *>(b + ((tbytes + obytes + 15) / 16) * 16);
    if (!terms.empty())
        LQCD_CUDA(cudaMemcpyAsync(dterms, terms.data(), sizeof(MesonTerm) * terms.size(), cudaMemcpyHostToDevice, st));
    LQCD_CUDA(cudaMemcpyAsync(doff, off.data(), obytes, cudaMemcpyHostToDevice, st));
    {
        // algorithmic bytes: the 12 columns once; flops: 8 per complex product, 9 per term, per site
        ProfScope prof("meson_contract", double(lat->V) * 12 * 192.0, st);
        meson_kernel<<<dim3(unsigned(nchunk), unsigned(T)), kBlock, 0, st>>>(
            lat->V, v3, ng, reinterpret_cast<const double2 *>(prop_dev), dterms, doff, dpart);
        LQCD_CHECK_LAUNCH();
    }
    meson_finish_kernel<<<unsigned(T * ng), kBlock, 0, st>>>(T, ng, nchunk, src_t, dpart,
                                                               reinterpret_cast<double2 *>(corr_dev));
    LQCD_CHECK_LAUNCH();
    LQCD_CUDA(cudaFreeAsync(buf, st));
}

}  // namespace lqcd
