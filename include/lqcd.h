/*
 * lqcd.h -- C ABI of a GB300 (sm_103a) library for the O(a)-improved Wilson
 * (clover) point-source propagator of LatticeGPU.jl (arXiv:2503.16994).
 *
 * What the calls compute (the paper's Sec. 3.3, with the reading below):
 *
 *   (D psi)(x) = psi(x)
 *       - kappa sum_mu [ (1 - g_mu) U~_mu(x) psi(x+mu) + (1 + g_mu) U~_mu(x-mu)^dag psi(x-mu) ]
 *       + i kappa csw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) psi(x)
 *
 *   kappa-normalised (m0 = 1/(2 kappa) - 4, D = 2 kappa Dw); U~_mu(x) carries
 *   the boundary phase factor theta_mu on the link from x_mu = L_mu - 1 to
 *   x_mu = 0 (theta holds full phase factors, Sec. 3.3 footnote); the default
 *   theta = (1,1,1,-1) gives periodic space and antiperiodic time.
 *   sigma_{mu nu} = (i/2)[g_mu, g_nu]; F_{mu nu} = (Q - Q^dag)/8 made
 *   traceless, Q the four-leaf clover (the Csw! term of Sec. 3.3).
 *   Gamma matrices, chiral basis, 2x2 spin blocks: g_k = [[0, -i s_k], [i s_k, 0]]
 *   (k = x, y, z), g_t = [[0, -1], [-1, 0]], g5 = g_t g_x g_y g_z = diag(1,1,-1,-1).
 *
 * Host layouts (all calls): lexicographic sites, x fastest and t slowest
 * (time is the last extent, Sec. 2.1).  Complex numbers are interleaved
 * (re, im) doubles.
 *   gauge field : U[t][z][y][x][mu][a][b]     (mu = 0..3 = x,y,z,t; 3x3 row-major; 72 doubles/site)
 *   spinor field: psi[t][z][y][x][spin][colour] (24 doubles/site; component 3*spin + colour)
 *   nrhs fields : stored one after another, field j at offset j * 24 * V doubles.
 *
 * Conventions:
 *   - Every call returns LQCD_OK (0) or a negative status; it never aborts,
 *     traps or exits.  lqcd_last_error() gives a message for the calling thread.
 *   - The caller owns every buffer it passes.  Host pointers are read or
 *     written only during the call.  With LQCD_DEVICE_PTRS the pointers are
 *     device memory of the lattice's device (for example PyTorch tensors),
 *     used in stream order on `stream`; the call returns after the work on
 *     `stream` has completed.
 *   - The library owns lattices, resident gauge fields (with their clover
 *     fields) and solver workspaces; they live until the matching destroy/free.
 *   - A lattice handle may be used from one thread at a time (calls on one
 *     lattice are serialised internally).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LQCD_ABI_VERSION 3

/* status codes */
enum {
    LQCD_OK = 0,
    LQCD_EINVAL = -1,    /* bad argument (null pointer, odd extent, unknown id, ...) */
    LQCD_ENOMEM = -2,    /* device memory or HBM budget exhausted */
    LQCD_ECUDA = -3,     /* a CUDA call failed (message has the CUDA error string) */
    LQCD_ENOCONV = -4,   /* a solve did not reach the tolerance within maxiter (info is filled in) */
    LQCD_EBUSY = -5,     /* request still pending (serve poll) */
    LQCD_ETIMEOUT = -6,  /* a bounded wait ran out (poll timeout, device-side wait cap) */
    LQCD_ENOTFOUND = -7, /* unknown ticket */
    LQCD_ENOTIMPL = -8   /* feature not available in this build */
};

/* solver precisions */
enum {
    LQCD_PREC_FP64 = 0,       /* every vector and operator in FP64 */
    LQCD_PREC_MIXED_FP32 = 1, /* inner Krylov vectors FP32, FP32 math, recon-12 FP32 links; FP64 outer */
    LQCD_PREC_MIXED_FP16 = 2  /* inner vectors FP16 + per-site FP32 scale, FP16 recon-12 links and
                                 clover, FP32 math; FP64 outer */
};

/* flags for lqcd_dirac_apply / lqcd_pion_contract / lqcd_cg_solve */
enum {
    LQCD_DAG = 1,         /* apply D^dag = g5 D g5 instead of D */
    LQCD_DEVICE_PTRS = 2, /* psi_in / psi_out (or prop / corr, b / x) are device pointers */
    LQCD_GUESS = 4        /* lqcd_cg_solve: x holds an initial guess on input (resume, warm start) */
};

/* boundary conditions in time (SpaceParm's BC of Sec. 2.1) */
enum {
    LQCD_BC_PERIODIC = 0, /* every direction closes on itself, the hops across carry theta_mu */
    LQCD_BC_OPEN = 1,     /* open in time: no link from the slice x_t = T - 1 to x_t = 0 (hops and clover
                             leaves across vanish, theta_t plays no part); the slices x_t = 0 and T - 1 get
                             the boundary improvement term 2 kappa (cF - 1) */
    LQCD_BC_SF = 2        /* Schroedinger functional (BC_SF_ORBI / BC_SF_AFWB, which read the same for the
                             quark fields), homogeneous quark boundary values: the slice x_t = 0 is the
                             boundary at x_t = 0 and at x_t = T (its links, set by the caller to the
                             boundary field, serve both); the operator is the identity there and no hop
                             reaches it; the clover term on 1 .. T-1 uses every link; the slices 1 and
                             T - 1 get 2 kappa (cF - 1); theta_t plays no part; mu must be 0 */
};

typedef struct lqcd_lattice_s *lqcd_lattice; /* opaque; owns all device memory it allocates */
typedef struct lqcd_server_s *lqcd_server;   /* opaque serving loop */

/* DiracParam of Sec. 3.3 (kappa instead of m0).  theta: the four boundary
 * phase factors (|theta_mu| = 1), re and im parts.  mu: twisted mass in mass
 * units, one flavour: the kappa-normalised site term gains 2 i kappa mu g5
 * (the paper's D_w gains i mu g5 and D = 2 kappa D_w), so
 *   D(mu) = D + 2 i kappa mu g5,   D(mu)^dag = g5 D(-mu) g5;
 * every call takes it (0: the Wilson-clover operator).  Per chirality block
 * A_s (s = +1 spins 0-1, -1 spins 2-3) the site term A_s + i s tau, tau =
 * 2 kappa mu, is inverted as B_s - i s tau C_s with C_s = (A_s^2 + tau^2)^-1
 * and B_s = A_s C_s.  Solves at mu != 0 run on the generic (untuned) hopping
 * kernel in every storage format.  mu must be finite (LQCD_EINVAL).
 * bc: LQCD_BC_PERIODIC (0), LQCD_BC_OPEN or LQCD_BC_SF; cF: the boundary
 * improvement coefficient of DiracParam (Sec. 3.3, c~_t), used with LQCD_BC_OPEN
 * and LQCD_BC_SF only (for LQCD_BC_OPEN the T
 * slices of the lattice are all dynamical; the paper's iL[4] - 1 effective
 * slices are this T).  A zero-initialised struct is the periodic operator. */
typedef struct {
    double kappa;
    double csw;
    double theta_re[4];
    double theta_im[4];
    double mu;
    double cF;
    int bc;
} lqcd_dirac_params;

/* tol: stop when the true relative residual |b - D x|_2 / |b|_2 of the full
 * (unpreconditioned) system is <= tol.  maxiter: cap on inner iterations
 * (applications of the normal operator) per right-hand side.  precision:
 * LQCD_PREC_*.  inner_tol: the reliable-update factor delta (the residual is
 * recomputed in FP64 whenever the low-precision one has dropped by delta;
 * 0 selects the default: 0.1 for FP16, 0.005 for FP32 inner vectors).  nrhs: right-hand sides solved together
 * (batched per launch), >= 1. */
typedef struct {
    double tol;
    int maxiter;
    int precision;
    double inner_tol;
    int nrhs;
} lqcd_solver_params;

/* Per right-hand-side result.  iters_inner: normal-operator applications;
 * iters_outer: FP64 residual recomputations (reliable updates); true_resid:
 * final |b - D x| / |b| computed in FP64 on the full lattice; status: LQCD_OK
 * or LQCD_ENOCONV. */
typedef struct {
    int iters_inner;
    int iters_outer;
    double true_resid;
    int status;
} lqcd_solve_info;

/* Thread-local message describing the last failing call of this thread. */
const char *lqcd_last_error(void);

/* LQCD_ABI_VERSION of the loaded library. */
int lqcd_abi_version(void);

/* Lattice geometry (SpaceParm of Sec. 2.1).  dims = {Lx, Ly, Lz, T}, each even
 * and >= 2 (even-odd preconditioning needs even extents; extents of 2 are
 * allowed, psi(x+mu) and psi(x-mu) are then the same site and both terms
 * count).  device: CUDA ordinal.  Allocates nothing large; gauge fields and
 * workspaces are allocated by later calls.
 * Errors: LQCD_EINVAL (null out, odd or < 2 extent, V/2 >= 2^31),
 * LQCD_ECUDA (bad device). */
int lqcd_lattice_create(const int dims[4], int device, lqcd_lattice *out);

/* Frees every device buffer of the lattice (gauge fields, clover fields,
 * workspaces).  NULL is accepted. */
int lqcd_lattice_destroy(lqcd_lattice lat);

/* Makes a gauge field resident (Sec. 2.2: SU(3) links, stored on the device
 * as FP64 and as reconstruct-12 FP32/FP16 copies keeping the first two rows;
 * the third row is rebuilt from unitarity as conj(row0 x row1)).  U: host
 * array in the layout above (72 doubles per site), copied; the caller keeps
 * it.  The links must be special unitary for the recon-12 copies to be exact.
 * *gauge_id receives an id >= 0 used by the other calls.
 * Errors: LQCD_EINVAL, LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_gauge_upload(lqcd_lattice lat, const double *U, int *gauge_id);

/* Releases a resident gauge field and its cached clover fields. */
int lqcd_gauge_free(lqcd_lattice lat, int gauge_id);

/* psi_out = D psi_in (or D^dag psi_in with LQCD_DAG), in FP64, out of place
 * (Dw! of Sec. 3.3: both fields preallocated by the caller).  The clover
 * field for (gauge_id, kappa, csw) is computed on first use and cached
 * (Csw! of Sec. 3.3).  psi_in, psi_out: 24 V doubles each, host layout; host
 * memory, or device memory with LQCD_DEVICE_PTRS.  psi_in and psi_out must
 * not overlap.
 * Errors: LQCD_EINVAL (null, unknown id, non-finite parameters), LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_dirac_apply(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp,
                     const double *psi_in, double *psi_out, int flags, void *stream);

/* The even-odd preconditioned operator used by the solver (the Schur
 * complement of D on the even sites; the paper's Dw! restricted to one
 * parity block, Sec. 3.3):
 *   Dhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe     (Dhat^dag = g5 Dhat g5 with LQCD_DAG)
 * where A is the clover site term and H the hopping term of D, applied in
 * the storage format of `precision` (LQCD_PREC_*: FP64; FP32; FP16 spinors
 * with a per-site scale, FP16 reconstruct-12 links and FP16 clover, FP32
 * arithmetic).  in, out: nrhs full-lattice fields in the host layout (host
 * memory, or device memory with LQCD_DEVICE_PTRS); only the even sites of in
 * are read (converted to `precision` first); out receives Dhat in on the even
 * sites (converted back to FP64) and zero on the odd sites.  repeat >= 1:
 * the operator is applied `repeat` times to the same input (same result),
 * so its kernels can be timed with lqcd_profile_*.
 * Errors: LQCD_EINVAL, LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_schur_apply(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, int precision,
                     const double *in, double *out, int nrhs, int repeat, int flags, void *stream);

/* Solves D x_j = b_j for j = 0..nrhs-1 (CG! of Sec. 3.3) by CG on the normal
 * equations of the even-odd preconditioned (Schur) operator
 *   Dhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe
 * (A = clover site term, H = hopping term), with FP64 residual recomputation
 * (reliable updates) and an FP64 final true-residual check on the full
 * lattice.  b, x: nrhs * 24 V doubles, host layout; host memory, or device
 * memory when flags has LQCD_DEVICE_PTRS.  x on input: with LQCD_GUESS in
 * flags, the initial guess x_0 (the CG! of Sec. 3.3 works on a given field:
 * a solve resumed from a saved x_0, or warm-started from a nearby solution);
 * the first FP64 residual is b - D x_0, so a guess that already meets tol
 * returns after that check with iters_inner = 0.  Only the even-site part of
 * x_0 enters (the odd part is rebuilt from it, x_o = A_oo^-1 (b_o +
 * kappa H_oe x_e)).  Without LQCD_GUESS, x on input is ignored (zero start).
 * x may not overlap b.  info: nrhs entries (may be NULL).  sp->nrhs is
 * ignored; nrhs is the argument.
 * Returns LQCD_OK when every column reached sp->tol, LQCD_ENOCONV when one
 * did not (x and info still filled), or an error. */
int lqcd_cg_solve(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp,
                  const lqcd_solver_params *sp, const double *b, double *x, int nrhs,
                  lqcd_solve_info *info, int flags, void *stream);

/* Point-source propagator and pion correlator (propagator! of Sec. 3.3 and
 * the contraction it enables; Sec. 4 example).  Solves the 12 columns
 * eta_j(x) = delta_{x,src} e_j, j = 3*spin + colour, as one batch, then
 *   corr[t] = sum_{x vec} sum_j sum_{spin,colour} |S_j(x vec, (src_t + t) mod T)|^2
 * (t counted from the source time slice; no 1/V).  src = {x, y, z, t}.
 * corr: T doubles (host, or device with LQCD_DEVICE_PTRS).  prop: NULL or
 * 12 * 24 V doubles receiving the 12 columns (same memory kind as corr).
 * info: 12 entries or NULL.  Return as lqcd_cg_solve. */
int lqcd_pion_corr(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp,
                   const lqcd_solver_params *sp, const int src[4], double *corr, double *prop,
                   lqcd_solve_info *info, int flags, void *stream);

/* One job of a batch of point-source propagators: its lattice and resident
 * gauge field, Dirac parameters, source, and outputs. */
typedef struct {
    lqcd_lattice lat;           /* in: lattice of this job (jobs may share one) */
    int gauge_id;               /* in: resident gauge field on lat */
    lqcd_dirac_params dp;       /* in: kappa, csw, theta of this job */
    int src[4];                 /* in: source position {x, y, z, t} */
    double *corr;               /* out: host array of T doubles (T of this lattice) */
    lqcd_solve_info info[12];   /* out: per column */
    int status;                 /* out: LQCD_OK or LQCD_ENOCONV */
} lqcd_pion_job;

/* Many point-source propagators (lqcd_pion_corr per job) on lattices of
 * different sizes, gauge fields and kappa, solved together: every job's 12
 * columns iterate in the same CUDA graph (one branch per job, `chunk`
 * iterations per graph launch, 0 = 8), so the device runs all lattices at
 * once and the host issues one launch per chunk instead of one per kernel.
 * The paper solves one propagator at a time (Sec. 4 example); this batches
 * uneven lattices into one device schedule.  All jobs use sp (precision, tol, maxiter) and
 * the device of their lattices (one device for the batch).  The call locks
 * every lattice involved and returns when all jobs are done; `stream` work
 * queued before the call completes first.
 * Returns LQCD_OK, LQCD_ENOCONV when a job has a column that did not
 * converge (its status says which), or an error (LQCD_EINVAL, LQCD_ENOMEM,
 * LQCD_ECUDA). */
int lqcd_pion_corr_batch(lqcd_pion_job *jobs, int njobs, const lqcd_solver_params *sp, int chunk, void *stream);

/* The pion contraction alone: corr[t] as above from 12 columns prop (12 * 24 V
 * doubles, host layout) with the source on time slice src_t.  Host pointers,
 * or device pointers with LQCD_DEVICE_PTRS.  Uses a device scratch buffer
 * owned by the lattice. */
int lqcd_pion_contract(lqcd_lattice lat, const double *prop, int src_t, double *corr, int flags,
                       void *stream);

/* Meson two-point functions for arbitrary spin matrices (the "any
 * contraction" of a propagator, Sec. 3.3): for each of the ng 4x4 complex
 * matrices G (gammas: ng * 16 complex = 32 ng doubles, row-major, chiral
 * basis of lqcd_dirac_apply, always a host pointer),
 *     corr[g][t] = - sum_xvec tr[ (G x 1) S(x) (Gbar x 1) g5 S(x)^dag g5 ],
 *     Gbar = g_t G^dag g_t,  x = (xvec, src_t + t mod T),
 * the connected correlator of psibar G psi with its conjugate at the source
 * (S(x0, x) = g5 S(x, x0)^dag g5).  S(x)[3 spin + colour][j] is column j of
 * prop (12 * 24 V doubles, host layout, source on slice src_t).  corr:
 * ng * T complex values (2 ng T doubles, re then im), t counted from the
 * source slice.  G = g5 gives the pion contraction.  Host pointers for prop
 * and corr, or device pointers with LQCD_DEVICE_PTRS (then on `stream`).
 * FP64 throughout; a G with one nonzero per row (the 16 Clifford basis
 * elements) costs 16 terms of 9 complex products per site, a dense G 256.
 * Returns LQCD_EINVAL for null pointers, src_t outside the lattice, ng
 * outside 1..LQCD_MESON_MAX_GAMMAS or non-finite entries of gammas. */
#define LQCD_MESON_MAX_GAMMAS 64
int lqcd_meson_contract(lqcd_lattice lat, const double *prop, int src_t, const double *gammas, int ng, double *corr,
                        int flags, void *stream);

/* Boundary-to-bulk correlators (Sec. 3.3: the propagators from the boundary
 * that give f_P and f_A), on the operator of dp (meant for LQCD_BC_OPEN or
 * LQCD_BC_SF): the six sources W_j, j = 3 s + c with spin s in {0, 1} and
 * colour c, P+ = (1 + g_t) / 2, zero spatial momentum (P+ e_{j+6} = -P+ e_j
 * adds nothing) -- W_j(y) = delta_{y_t, 0} P+ e_j on every site of the slice
 * y_t = 0 (open, periodic), or W_j(y) = delta_{y_t, 1} U_t(0, yvec)^dag P+ e_j
 * on the slice 1 (SF: the boundary quark field carried in by the time link)
 * -- are solved as one batch, H_j = D^-1 W_j, and per slice
 *   fP[x_t] = sum_xvec sum_j |H_j(x)|^2,
 *   fA[x_t] = - sum_xvec sum_j Re <H_j(x), g_t H_j(x)>.
 * fP, fA: T doubles each; H: NULL or 6 * 24 V doubles receiving the columns;
 * all host memory, or device memory with LQCD_DEVICE_PTRS.  info: 6 entries
 * or NULL.  Returns as lqcd_cg_solve. */
int lqcd_boundary_corr(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, const lqcd_solver_params *sp,
                       double *fP, double *fA, double *H, lqcd_solve_info *info, int flags, void *stream);

/* ---------------- gauge observables and the Wilson flow (Sec. 3.2) ---- */

/* Wilson flow of a resident gauge field, in place (flw with the wfl_rk3
 * scheme of Sec. 3.2): nsteps steps of size eps of the third-order
 * Runge-Kutta integrator of Luescher (JHEP 2010, the reference the paper
 * cites), flow time t = nsteps eps:
 *   W1 = exp(Z0/4) W0,  W2 = exp(8 Z1/9 - 17 Z0/36) W1,
 *   V(t + eps) = exp(3 Z2/4 - 8 Z1/9 + 17 Z0/36) W2,   Z_i = eps Z(W_i),
 * Z_mu(x) = -(1/2)(Omega - Omega^dag) + (1/6) tr(Omega - Omega^dag), Omega =
 * U_mu(x) times the sum of its six staples (the force of the Wilson action
 * over oriented plaquettes); periodic in every direction; FP64 on the GPU.
 * The FP32/FP16 copies are rebuilt and the cached clover fields dropped.
 * Errors: LQCD_EINVAL (unknown id, eps <= 0, nsteps < 0), LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_gauge_flow(lqcd_lattice lat, int gauge_id, double eps, int nsteps, void *stream);

/* Fermion gradient flow (Sec. 3.2: the flow of quark fields following
 * Luescher's 2013 construction, which the paper cites): the resident links
 * are flowed exactly as by lqcd_gauge_flow and the nrhs quark fields psi
 * alongside, d psi/dt = Delta psi with the covariant Laplacian
 *   (Delta psi)(x) = sum_mu [U~_mu(x) psi(x+mu) + U~_mu(x-mu)^dag psi(x-mu) - 2 psi(x)]
 * (colour only; U~ carries the boundary phases theta of dp, the other fields
 * of dp are not used), by the third-order scheme on the gauge stages W0, W1,
 * W2 of each step:
 *   lambda1 = psi + eps/4 Delta(W0) psi,
 *   lambda2 = psi + 8 eps/9 Delta(W1) lambda1 - 2 eps/9 Delta(W0) psi,
 *   psi(t + eps) = lambda1 + 3 eps/4 Delta(W2) lambda2;  FP64.
 * psi: nrhs full-lattice fields in the host layout, overwritten with the
 * flowed fields (host memory, or device memory with LQCD_DEVICE_PTRS).
 * Errors: LQCD_EINVAL (unknown id, null pointer, eps <= 0, nsteps < 0,
 * nrhs < 1, bc other than periodic), LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_fermion_flow(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, double *psi, int nrhs,
                      double eps, int nsteps, int flags, void *stream);

/* Fermion backflow (Sec. 3.2: correlators of flowed quark fields need "the
 * integration of the adjoint flow equations", the fermion field backflowed
 * through stored gauge fields): the exact adjoint of the steps of
 * lqcd_fermion_flow, applied to eta from flow time t = nsteps eps back to 0
 * through the Wilson flow that starts at the resident links.  With one
 * forward step psi' = M psi, one backward step is eta <- M^dag eta =
 *   u + z2 + Delta(W0) (eps/4 u - 2 eps/9 z2),  u = eta + z1,
 *   z2 = 3 eps/4 Delta(W2) eta,  z1 = 8 eps/9 Delta(W1) z2,
 * so <eta, F psi> = <B eta, psi> holds for the discrete flows F and B.  The
 * gauge field at the start of every step is rebuilt from nsave >= 1
 * checkpoints (one every ceil(nsteps / nsave) steps), each segment being
 * flowed again from its checkpoint: device memory for nsave + ceil(nsteps /
 * nsave) + 3 gauge fields and 5 nrhs-field quark fields.  The resident links
 * are not changed.  eta: nrhs full-lattice fields in the host layout (host
 * memory, or device memory with LQCD_DEVICE_PTRS), overwritten.
 * Errors: LQCD_EINVAL (unknown id, null pointer, eps <= 0, nsteps < 0,
 * nrhs < 1, nsave < 1, bc other than periodic), LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_fermion_backflow(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, double *eta, int nrhs,
                          double eps, int nsteps, int nsave, int flags, void *stream);

/* Gauge observables of a resident field (plaquette, Eoft_plaq, Eoft_clover
 * and Qtop of Sec. 3.2), FP64, host outputs (any may be NULL):
 *   *plaq    = (1 / 6V) sum_x sum_{mu<nu} Re tr U_p(x) / 3   (1 for the unit field),
 *   Eplaq[t] = sum_xvec 2 sum_{mu<nu} Re tr (1 - U_p(x)),
 *   Eclov[t] = sum_xvec - sum_{mu<nu} tr F_{mu nu}(x)^2,
 *   Q[t]     = sum_xvec -(1 / 32 pi^2) eps_{mu nu rho sigma} tr F_{mu nu}(x) F_{rho sigma}(x),
 * per time slice t (T values each), F the antihermitian clover field of
 * lqcd_dirac_apply; divide by L^3 for the densities. */
int lqcd_gauge_observables(lqcd_lattice lat, int gauge_id, double *plaq, double *Eplaq, double *Eclov, double *Q,
                           void *stream);

/* One trajectory of the quenched Hybrid Monte Carlo (HMC! of Sec. 3.1) on a
 * resident gauge field, in place, with the leapfrog integrator of nsteps
 * steps of size eps, for the Wilson gauge action with beta = 2N / g0^2,
 * read as S = (beta / 3) sum_x sum_{mu<nu} Re tr (1 - U_p(x)) (c0 = 1):
 *   P += eps/2 F(U);  [U = exp(eps P) U;  P += eps F(U)] x (nsteps - 1);
 *   U = exp(eps P) U;  P += eps/2 F(U),      F = -dS (Lie derivative),
 * H = -sum tr P^2 + S.  mom: the initial momenta, host, 8 V 4 doubles
 * [site][mu][a] = coordinates on the generators i lambda_a / 2 (standard
 * Gell-Mann order), drawn by the caller (normal for the HMC).  u: a uniform
 * number in (0, 1) drawn by the caller; the trajectory is accepted when
 * u < exp(-dH), otherwise the links are restored.  *dH receives H(end) -
 * H(start), *accepted 1 or 0.  FP64; the FP32/FP16 copies are rebuilt and
 * the cached clover fields dropped.  Omelyan integrators and the c1 (1x2
 * loop) terms of the paper's action are not built. */
int lqcd_hmc_trajectory(lqcd_lattice lat, int gauge_id, double beta, double eps, int nsteps, const double *mom,
                        double u, double *dH, int *accepted, void *stream);

/* The resident FP64 links in the host layout of lqcd_gauge_upload (72 V
 * doubles; host memory, or device memory with LQCD_DEVICE_PTRS). */
int lqcd_gauge_download(lqcd_lattice lat, int gauge_id, double *U, int flags, void *stream);

/* ---------------- launch accounting and timing ------------------------- */

/* Per-kernel statistics since the last lqcd_profile_reset.  launches and
 * bytes count every launch of the kind (bytes = algorithmic bytes: each
 * operand of the launch read or written once, for the right-hand sides
 * expected to pass the launch's gate by the last host poll, all of them when
 * unknown).  Launches replayed from a CUDA graph (small solves below 2^20
 * site-RHS and batched solves) are counted once, when the graph is
 * captured, and are not timed.  timed_*: launches bracketed by CUDA events
 * on their stream while timing was enabled, with their summed device time.  Not part of the
 * paper; this is the library's tracing facility (the paper times methods
 * with TimerOutputs.jl, Sec. 3.4). */
typedef struct {
    char name[48];
    long long launches;
    double bytes;
    long long timed_launches;
    double timed_ms;
    double timed_bytes;
} lqcd_kernel_stat;

/* Clears the statistics; enable_timing != 0 brackets every following launch
 * with CUDA events (a small host overhead per launch). */
int lqcd_profile_reset(int enable_timing);

/* Copies up to max entries into out; *count receives the number of kernel
 * kinds seen.  Waits for the timed launches to complete. */
int lqcd_profile_read(lqcd_kernel_stat *out, int max, int *count);

/* Autotuning decisions taken so far in this process, as a JSON array
 * written into buf (len bytes, NUL-terminated).  Each entry names a kernel,
 * the problem (sites per parity, right-hand sides) and the chosen shape
 * with its time: variant ("scalar": 1..3 right-hand sides per thread in
 * scalar arithmetic; "paired": two right-hand sides in the lanes of packed
 * FP32x2 instructions; "paired_staged": the same with each direction's words
 * copied into shared memory by cp.async, FP16 only; "prefetch": one
 * right-hand side with the loads of several directions issued ahead),
 * rhs_per_thread, directions_ahead, rhs_groups_per_block (groups run in
 * sequence by one block), min_blocks_per_sm (register cap),
 * tiles_per_supertile (block order) and block (threads).  The hopping
 * kernels time these candidates on their first launch for each (sites,
 * nrhs, format, mode) and keep the fastest; the environment variables
 * LQCD_HOP_NR (shape code: 1..3 scalar, 0 paired, -2/-4/-8 prefetch, 12/13
 * staged 2/3 directions ahead), LQCD_HOP_GPB, LQCD_HOP_MINB and LQCD_HOP_SWZ
 * force a shape instead.  Returns LQCD_EINVAL
 * if buf is too small (the text is truncated). */
int lqcd_tune_report(char *buf, size_t len);

/* The autotuner's decisions of this process (timed or imported) as text
 * that lqcd_tune_import reads back, so that a later process (a restarted
 * server) skips the timing: a header line "lqcd-tune 1", then one line per
 * decision "<format> <mode> <sites per parity> <nrhs> <nr> <gpb> <minb> <swz>"
 * (format f64, f32 or f16; mode 0 = t = kappa A^-1 H in, 1 = A self -
 * kappa H in; nr the shape code of lqcd_tune_report, gpb its
 * rhs_groups_per_block, minb min_blocks_per_sm, swz tiles_per_supertile).
 * The shapes are valid on the GPU model that timed them.  Returns LQCD_EINVAL
 * if buf is too small (the text is truncated). */
int lqcd_tune_export(char *buf, size_t len);

/* Loads decisions in the format of lqcd_tune_export: the first launch of a
 * listed (format, mode, sites, nrhs) uses the shape without timing the
 * candidates (reported with "source": "imported").  Every line is checked
 * first (header, field count, a shape the launcher accepts for the format);
 * on any error nothing is loaded and LQCD_EINVAL is returned.  Shapes already
 * chosen in this process are kept.  Host-only: needs no GPU. */
int lqcd_tune_import(const char *text);

/* The pion contraction of lqcd_pion_contract without any device allocation,
 * for callers that cannot allocate: processes whose device memory belongs
 * to another allocator (a framework's caching allocator or a fixed pool,
 * where a cudaMalloc can fail or fragment it) and loops that must not call
 * cudaMalloc/cudaFree per call because those can synchronize the device.
 * The paper has no counterpart: this is a library service.
 *
 * dims = {Lx, Ly, Lz, T} (host array, extents >= 1); prop: 12 * 24 V
 * doubles, device memory of the current device, host layout; corr: T
 * doubles, device memory of the current device; src_t: source time slice.
 * No lattice handle is needed.  The work is queued on `stream` and the call
 * returns without waiting; corr is valid once the stream reaches it.
 *
 * Scratch: a fixed array compiled into the library's device image (2 MiB of
 * partial sums and 8192 counters), held by every GPU that loads the library
 * until the process exits.  The lattice must satisfy
 * T * ceil(12 V / (512 T)) <= 262144 and T <= 8192 (32^3 x 64 needs
 * 49152); larger lattices get LQCD_EINVAL with the counts
 * in the message (use lqcd_pion_contract there).  The first call on a
 * device looks up the device address of the array (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture on that
 * device.  Every call shares the array, and the counters are cleared at the
 * start of each call: calls that overlap on the GPU (other streams, other
 * threads) race and give wrong results, so serialize them.
 * Errors: LQCD_EINVAL (null pointer, bad extent or source, too large),
 * LQCD_ECUDA. */
int lqcd_pion_contract_noalloc(const int dims[4], const double *prop, int src_t, double *corr, void *stream);

/* ---------------- serving loop (continuous batching) ------------------- */

/* A server owns one device thread that admits propagator requests
 * (lqcd_pion_corr work units) while HBM budget and slots allow, runs all
 * admitted requests' iterations interleaved on the device, and retires each
 * one independently as it converges.  hbm_budget_bytes: device memory the
 * server may use for gauge fields and per-request workspaces (0 = 90% of
 * free memory).  max_slots: requests resident at once (>= 1). */
int lqcd_serve_create(int device, size_t hbm_budget_bytes, int max_slots, lqcd_server *out);

/* Makes a gauge field of the given dims resident on the server (charged
 * to the budget).  U: host, layout as lqcd_gauge_upload.  Errors as there,
 * plus LQCD_ENOMEM when the budget cannot hold it. */
int lqcd_serve_gauge(lqcd_server srv, const int dims[4], const double *U, int *gauge_id);

/* Queues one 12-column point-source propagator + pion correlator request.
 * Copies its arguments; non-blocking.  *ticket identifies the request.
 * Errors: LQCD_EINVAL (unknown gauge id, bad source or params, bc other than
 * LQCD_BC_PERIODIC or LQCD_BC_OPEN). */
int lqcd_serve_submit(lqcd_server srv, int gauge_id, const lqcd_dirac_params *dp,
                      const lqcd_solver_params *sp, const int src[4], uint64_t *ticket);

/* Waits up to timeout_ms (0 = just look, < 0 = forever) for a request.
 * On completion fills corr (T doubles), info (12 entries) and timestamps
 * {arrive, admit, start, finish} (seconds on a monotonic clock; any of the
 * three pointers may be NULL) and forgets the ticket.  Returns LQCD_OK when
 * done, LQCD_ENOCONV when done but a column did not converge, LQCD_EBUSY when
 * still queued or running and timeout_ms == 0, LQCD_ETIMEOUT when the wait
 * ran out, LQCD_ENOTFOUND for an unknown ticket, or the request's error. */
int lqcd_serve_poll(lqcd_server srv, uint64_t ticket, double *corr, lqcd_solve_info *info,
                    double timestamps[4], int timeout_ms);

/* Stops the device threads: queued requests finish at once and running ones
 * at their next poll, all with LQCD_ETIMEOUT ("server stopped"), so a
 * lqcd_serve_poll already waiting returns; destroy waits for such polls to
 * leave, then frees everything.  No call on srv may start once destroy has
 * begun.  NULL is accepted. */
int lqcd_serve_destroy(lqcd_server srv);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
