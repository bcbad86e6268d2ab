// Host-side internals of the library: lattice handle, resident gauge and
// clover fields, solver workspaces, kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/lqcd.h"
#include "kernels.cuh"

namespace lqcd {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define LQCD_CUDA(call)                                                                             \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            throw ::lqcd::Error{e_ == cudaErrorMemoryAllocation ? LQCD_ENOMEM : LQCD_ECUDA,         \
                                std::string(#call) + ": " + cudaGetErrorString(e_)};                \
    } while (0)

#define LQCD_CHECK_LAUNCH() LQCD_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// device memory owned by the library
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t async_st = nullptr;  // set: stream-ordered allocation (cudaMallocAsync / cudaFreeAsync)
    bool async = false;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) {
            if (async)
                cudaFreeAsync(p, async_st);
            else
                cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    // (re)allocates when smaller than `n` bytes; contents are not kept
    void ensure(size_t n)
    {
        if (bytes >= n) return;
        release();
        if (async)
            LQCD_CUDA(cudaMallocAsync(&p, n, async_st));
        else
            LQCD_CUDA(cudaMalloc(&p, n));
        bytes = n;
    }
    // later allocations of this buffer are stream-ordered on `st` (no device-wide synchronisation)
    void set_async(cudaStream_t st)
    {
        async = true;
        async_st = st;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// resident fields
// ---------------------------------------------------------------------------
// Clover site terms of one (gauge field, kappa csw, twisted mass): A, the
// Hermitian chirality blocks, and the inverse of A + i tau g5 (tau = 2 kappa
// mu).  tau = 0: ainv = A^-1.  tau != 0: per block (sign s = +1 upper, -1
// lower) (A + i s tau)^-1 = B - i s tau C with C = (A^2 + tau^2)^-1 and
// B = A C, both Hermitian; ainv holds B and cinv holds C.
struct CloverSet {
    double tau = 0.0;
    DevBuf a64, ainv64, cinv64;  // [parity][36 double2 planes]
    DevBuf a32, ainv32, cinv32;  // [parity][18 float4 planes]
    DevBuf a16, ainv16, cinv16;  // [parity][9 uint4 planes]
};

struct GaugeSet {
    DevBuf u64;             // [parity][mu][9 double2 planes]
    DevBuf u32;             // [parity][mu][3 float4 planes]
    DevBuf u16, u16b;       // [parity][mu] uint4 plane + uint2 plane
    // the hopping links of Schroedinger-functional boundaries: the same copies
    // with every link that touches the boundary slice x_t = 0 set to zero
    // (built on first use; sf_ready false once the links change)
    DevBuf u64sf, u32sf, u16sf, u16bsf;
    bool sf_ready = false;
    // keyed by (kappa csw, kappa mu, bc, kappa (cF - 1))
    std::map<std::tuple<double, double, int, double>, std::unique_ptr<CloverSet>> clover;
};

// Storage-format-specific field pointers for one (gauge, clover) pair.
template <class S> LinkField<S> link_field(const GaugeSet &g, long stride);
// the links the hopping kernels use under the boundary condition bc (the
// zeroed copies for LQCD_BC_SF, which clover_get builds)
template <class S> LinkField<S> hop_links(const GaugeSet &g, long stride, int bc);
template <class S> CloverField<S> clover_field(const CloverSet &c, bool inverse, long stride);
// the C blocks of a twisted inverse (null pointers when tau = 0)
template <class S> CloverField<S> clover_field_c(const CloverSet &c, long stride);

// Solver workspace for one (nrhs, precision): fields of one parity each.
struct Workspace {
    int nrhs = 0, prec = -1;
    DevBuf b_e, b_o, bhat, x_e, x_o, t64, w64;   // FP64
    DevBuf p, t, w, r, z;                        // inner precision
    DevBuf p_sc, t_sc, w_sc, r_sc, z_sc;         // FP16 scales
    DevBuf e;                                    // correction (FP32, or FP64 for the FP64 solver)
    DevBuf state;                                // RhsState[nrhs]
    DevBuf partial, counter;                     // reductions
    RhsState *host_state = nullptr;              // host mirror (pinned unless host_pageable)
    bool host_pageable = false;
    ~Workspace();
};

// Solver workspace for (nrhs, precision) on a lattice.  async: the device
// buffers are stream-ordered allocations on `st` (used by the server, whose
// requests come and go while other streams run) and the host mirror is
// pageable memory.
std::unique_ptr<Workspace> workspace_build(lqcd_lattice_s *lat, int nrhs, int prec, cudaStream_t st, bool async);
size_t workspace_bytes(const lqcd_lattice_s *lat, int nrhs, int prec);
std::unique_ptr<CloverSet> clover_build(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp,
                                        cudaStream_t st, bool async);
size_t clover_bytes(const lqcd_lattice_s *lat, bool twisted = false);
size_t gauge_bytes(const lqcd_lattice_s *lat);

}  // namespace lqcd

struct lqcd_lattice_s {
    int dims[4];
    int device;
    long V, vh, stride;
    lqcd::Geom geom;
    std::mutex mu;
    std::map<int, std::unique_ptr<lqcd::GaugeSet>> gauges;
    int next_gauge = 0;
    std::map<std::pair<int, int>, std::unique_ptr<lqcd::Workspace>> ws;  // keyed by (nrhs, precision)
    lqcd::DevBuf staging;         // host-layout fields on the device
    lqcd::DevBuf staging2;
    lqcd::DevBuf red_partial, red_counter, red_state;  // reductions outside the solver
};

namespace lqcd {

constexpr int kBlock = 128;

// Counts (and, when enabled, times) one kernel launch made in its lifetime.
struct ProfScope {
    std::string name;
    double bytes;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    bool timed = false;
    ProfScope(const char *name, double bytes, cudaStream_t st);
    ~ProfScope();
};

// records an autotuning decision (reported by lqcd_tune_report and
// lqcd_tune_export); ms < 0: taken from an imported table, not timed
void tune_record(const char *prec, int mode, int vh, int nrhs, int nr, int gpb, int minb, int swz, float ms);
// a shape imported by lqcd_tune_import for (format, mode, sites per parity,
// nrhs): shape = (nr, gpb, minb, swz); false when none was imported
bool tune_imported(const char *prec, int mode, int vh, int nrhs, int shape[4]);

// algorithmic bytes per site of one field in a storage format
template <class S> constexpr double spinor_bytes() { return S::W == 2 ? 192.0 : (S::W == 4 ? 96.0 : 52.0); }
template <class S> constexpr double link_bytes() { return S::W == 2 ? 144.0 : (S::W == 4 ? 48.0 : 24.0); }
template <class S> constexpr double clover_bytes() { return S::W == 2 ? 576.0 : (S::W == 4 ? 288.0 : 144.0); }
template <class S> constexpr const char *prec_name() { return S::W == 2 ? "f64" : (S::W == 4 ? "f32" : "f16"); }

inline int ntiles_of(long vh) { return int((vh + kBlock - 1) / kBlock); }



// gauge / clover setup (field_ops.cu)
void gauge_repack(lqcd_lattice_s *lat, GaugeSet &g, const double *U_dev_aos, cudaStream_t st);
// the clover fields of (g, dp), built on first use; for LQCD_BC_SF also the
// hopping links of hop_links
CloverSet &clover_get(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, cudaStream_t st);
// the boundary phases the hopping kernels use: theta, with theta_t = 0 for an open time boundary
void hop_theta(const lqcd_dirac_params &dp, double th_re[4], double th_im[4]);

// Wilson flow of the resident links (RK3, nsteps of eps; FP32/FP16 copies
// rebuilt, clover cache dropped), per-slice observables into out_dev[4 T]
// (plaquette / 3, plaquette and clover action densities, clover charge
// density), and the links in the host layout (gauge_flow.cu)
void gauge_flow(lqcd_lattice_s *lat, GaugeSet &g, double eps, int nsteps, cudaStream_t st);
// the same flow with nrhs quark fields (host layout, on the device) flowed
// alongside by the covariant Laplacian (theta of dp), in place
void fermion_flow(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, double *psi_dev, int nrhs,
                  double eps, int nsteps, cudaStream_t st);
// the exact adjoint of fermion_flow's steps, run backwards from t = nsteps eps
// to 0 through the flow that starts at the resident links (left unchanged);
// nsave gauge-field checkpoints
void fermion_backflow(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, double *eta_dev, int nrhs,
                      double eps, int nsteps, int nsave, cudaStream_t st);
void gauge_observables(lqcd_lattice_s *lat, GaugeSet &g, double *out_dev, cudaStream_t st);
void gauge_download(lqcd_lattice_s *lat, GaugeSet &g, double *U_dev, cudaStream_t st);
// one leapfrog HMC trajectory of the resident links with the caller's momenta
// (device, [site][mu][8]); returns accepted (1) or rejected (0, links restored)
int hmc_trajectory(lqcd_lattice_s *lat, GaugeSet &g, double beta, double eps, int nsteps, const double *mom_dev,
                   double u, double *dH, cudaStream_t st);

// host-layout <-> even-odd SoA FP64 (field_ops.cu)
void spinor_to_soa(lqcd_lattice_s *lat, const double *aos, int nrhs, SpinorField<F64> even, SpinorField<F64> odd,
                   cudaStream_t st);
void spinor_from_soa(lqcd_lattice_s *lat, double *aos, int nrhs, SpinorField<F64> even, SpinorField<F64> odd,
                     cudaStream_t st);
void point_sources(lqcd_lattice_s *lat, const int src[4], SpinorField<F64> even, SpinorField<F64> odd,
                   cudaStream_t st);
// corr[t] (device, T doubles) from 12 FP64 SoA columns, t relative to src_t
void pion_contract_soa(lqcd_lattice_s *lat, SpinorField<F64> even, SpinorField<F64> odd, int src_t,
                       double *corr_dev, double *partial, unsigned *counter, cudaStream_t st);
// corr[t] from 12 host-layout columns already on the device
void pion_contract_aos(lqcd_lattice_s *lat, const double *prop_dev, int src_t, double *corr_dev,
                       double *partial, unsigned *counter, cudaStream_t st);
// the six boundary wall sources delta_{y_t,0} P+ e_j (j = 3 s + c, s < 2), host layout, on the device
void wall_sources_p_plus(lqcd_lattice_s *lat, double *aos, cudaStream_t st);
// the six SF boundary sources U_t(0, yvec)^dag P+ e_j on the slice 1, host layout, on the device
void wall_sources_sf(lqcd_lattice_s *lat, const GaugeSet &g, double *aos, cudaStream_t st);
// fP[t], fA[t] (device, T doubles each) from six host-layout columns on the device
void boundary_contract(lqcd_lattice_s *lat, const double *H_dev, double *fP, double *fA, double *partial,
                       unsigned *counter, cudaStream_t st);
// corr[g][t] (complex) for ng host 4x4 spin matrices, 12 host-layout columns on the device (meson.cu)
void meson_contract(lqcd_lattice_s *lat, const double *prop_dev, int src_t, const double *gammas, int ng,
                    double *corr_dev, cudaStream_t st);

// hopping kernels (dslash_f64.cu, dslash_f32.cu, dslash_f16.cu)
template <class S, class L, class C>
void launch_hop(const HopArgs<S, L, C> &a, int mode, bool dag, bool norm, cudaStream_t st);

// vector kernels (blas_*.cu)
template <class W, class E>
void launch_er_update(const VecArgs &v, SpinorField<W> p, SpinorField<W> w, SpinorField<W> r, SpinorField<E> e,
                      cudaStream_t st);
template <class W>
void launch_p_update(const VecArgs &v, const RhsState *s, SpinorField<W> z, SpinorField<W> p, cudaStream_t st);
template <class E>
void launch_x_update(const VecArgs &v, const RhsState *s, SpinorField<E> e, SpinorField<F64> x, cudaStream_t st);
template <class W, class WI>
void launch_r_replace(const VecArgs &v, SpinorField<F64> src, SpinorField<WI> w, SpinorField<W> r,
                      SpinorField<F64> save, bool w_scaled, cudaStream_t st);
void launch_norm2_f64(const VecArgs &v, SpinorField<F64> x, cudaStream_t st);
// finishes the per-tile partials a hopping kernel wrote with reduce_partial
// (quad: the FP32 32-site partials of the tile kernel in r.partial_f)
void launch_partial_finish(const Reduce &r, int ntiles, int nrhs, const RhsState *gate_st, int gate, cudaStream_t st,
                           bool quad = false);
// out = C in, or with tau != 0 the twisted inverse (B - i s tau Cc) in (cl = B, cl2 = Cc)
template <class S, class C>
void launch_clover_apply(long vh, int nrhs, int parity, CloverField<C> cl, SpinorField<S> in, SpinorField<S> out,
                         cudaStream_t st, double tau = 0.0, CloverField<C> cl2 = CloverField<C>{});

template <class SI, class SO>
void launch_convert(long vh, int nrhs, SpinorField<SI> in, SpinorField<SO> out, cudaStream_t st);

// solver (solver.cu)
void schur_apply_dev(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, int precision, const double *in,
                     double *out, int nrhs, int repeat, bool dag, cudaStream_t st);
void dirac_apply_dev(lqcd_lattice_s *lat, GaugeSet &g, const lqcd_dirac_params &dp, const double *in, double *out,
                     bool dag, cudaStream_t st);
// guess: x_dev holds an initial guess on entry (host layout, device memory);
// otherwise the solve starts from zero
int solve(lqcd_lattice_s *lat, int gauge_id, const lqcd_dirac_params &dp, const lqcd_solver_params &sp,
          const double *b_dev, double *x_dev, const int *src, int nrhs, lqcd_solve_info *info, double *corr_dev,
          cudaStream_t st, bool guess = false);
// Batched propagators over uneven lattices (lqcd_pion_corr_batch); returns
// the number of jobs with a column that did not converge.
int pion_batch(lqcd_pion_job *jobs, int n, const lqcd_solver_params &sp, int chunk, cudaStream_t origin);

// The same on explicit clover fields and workspace (no lattice caches); stops
// early when *cancel becomes true (then returns nrhs).
int solve_on(lqcd_lattice_s *lat, GaugeSet &g, CloverSet &cl, Workspace &ws, const lqcd_dirac_params &dp,
             const lqcd_solver_params &sp, const double *b_dev, double *x_dev, const int *src, int nrhs,
             lqcd_solve_info *info, double *corr_dev, cudaStream_t st, const volatile bool *cancel,
             bool guess = false);

}  // namespace lqcd
