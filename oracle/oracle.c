/*
 * FP64 CPU oracle for the O(a)-improved (clover) Wilson propagator path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the library never calls
 * it and shares no code, header, table or helper with it.
 *
 * What it follows (LatticeGPU.jl, arXiv:2503.16994):
 *   - Sec. 3.3: DiracParam(m0, csw, theta, ...), Dw! (the Wilson-clover
 *     operator), Csw! (the Sheikholeslami-Wohlert term stored as a clover
 *     field and added at every application), CG! and propagator! (point
 *     source of given spin, colour and position), and the footnote there
 *     that theta holds the full boundary phase factors.
 *   - Sec. 2.1: lattice extents with time last.
 *   - Sec. 2.2: SU(3) links and 4-spinor x 3-colour fermion fields.
 * The paper prints no formula for the operator.  The reading used here is
 * the standard kappa-normalised O(a)-improved Wilson operator:
 *
 *   (D psi)(x) = psi(x)
 *       - kappa sum_mu [ (1 - g_mu) U~_mu(x) psi(x+mu)
 *                        + (1 + g_mu) U~_mu(x-mu)^dag psi(x-mu) ]
 *       + i kappa csw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) psi(x)
 *
 * with U~_mu(x) = theta_mu U_mu(x) on the link that leaves the last slice in
 * direction mu (x_mu = L_mu - 1), sigma_{mu nu} = (i/2)[g_mu, g_nu], and
 * F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag)/8 made traceless, Q being the sum of
 * the four plaquette leaves around x (the clover).  Gamma matrices are in the
 * chiral basis: g_t = [[0,-1],[-1,0]], g_k = [[0,-i s_k],[i s_k,0]] in 2x2
 * spin blocks, so g5 = g_t g_x g_y g_z = diag(1,1,-1,-1).
 *
 * Layouts (host, lexicographic with x fastest and t slowest, mu = 0..3 =
 * x,y,z,t): gauge U[site][mu][a][b], spinor psi[site][spin][colour], complex
 * numbers as interleaved (re, im) doubles.
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Lattice geometry (Sec. 2.1: iL with the time extent last)           */
/* ------------------------------------------------------------------ */

static long volume_of(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int L[4], long s, int x[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

static long index_of(const int L[4], const int x[4])
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

/* site reached from s by one step of dir = +1 or -1 in direction mu */
static long step(const int L[4], long s, int mu, int dir)
{
    int x[4];
    coords_of(L, s, x);
    x[mu] = (x[mu] + dir + L[mu]) % L[mu];
    return index_of(L, x);
}

/* ------------------------------------------------------------------ */
/* Gamma matrices in the chiral basis, built from the Pauli matrices    */
/* ------------------------------------------------------------------ */

static cplx G[5][4][4];     /* g_x, g_y, g_z, g_t, g5 */
static cplx SIGMA[4][4][4][4]; /* sigma_{mu nu} = (i/2)[g_mu, g_nu] */
static int gamma_ready = 0;

static void init_gamma(void)
{
    if (gamma_ready) return;
    const cplx pauli[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(G, 0, sizeof G);
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G[k][i][2 + j] = -I * pauli[k][i][j];
                G[k][2 + i][j] = I * pauli[k][i][j];
            }
    for (int i = 0; i < 2; ++i) {
        G[3][i][2 + i] = -1;
        G[3][2 + i][i] = -1;
    }
    /* g5 = g_t g_x g_y g_z */
    cplx a[4][4], b[4][4];
    memcpy(a, G[3], sizeof a);
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                cplx acc = 0;
                for (int l = 0; l < 4; ++l) acc += a[i][l] * G[k][l][j];
                b[i][j] = acc;
            }
        memcpy(a, b, sizeof a);
    }
    memcpy(G[4], a, sizeof a);
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu)
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    cplx c = 0;
                    for (int l = 0; l < 4; ++l)
                        c += G[mu][i][l] * G[nu][l][j] - G[nu][i][l] * G[mu][l][j];
                    SIGMA[mu][nu][i][j] = 0.5 * I * c;
                }
    gamma_ready = 1;
}

/* gamma matrix mu (0..3 = x,y,z,t; 4 = gamma5) as 4x4 complex, row-major */
void oracle_gamma(int mu, double *out)
{
    init_gamma();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            out[2 * (4 * i + j)] = creal(G[mu][i][j]);
            out[2 * (4 * i + j) + 1] = cimag(G[mu][i][j]);
        }
}

/* ------------------------------------------------------------------ */
/* 3x3 complex matrices (Sec. 2.2: SU(3) link variables)               */
/* ------------------------------------------------------------------ */

typedef struct { cplx m[3][3]; } mat3;

static mat3 link_at(const double *U, long s, int mu)
{
    mat3 r;
    const double *p = U + 18 * (4 * s + mu);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) r.m[a][b] = p[2 * (3 * a + b)] + I * p[2 * (3 * a + b) + 1];
    return r;
}

static mat3 mul(mat3 a, mat3 b)
{
    mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx c = 0;
            for (int k = 0; k < 3; ++k) c += a.m[i][k] * b.m[k][j];
            r.m[i][j] = c;
        }
    return r;
}

static mat3 dag(mat3 a)
{
    mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

static mat3 add(mat3 a, mat3 b)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.m[i][j] += b.m[i][j];
    return a;
}

/* ------------------------------------------------------------------ */
/* Clover field (Sec. 3.3, Csw!): F_{mu nu}(x) for the 6 planes mu<nu   */
/* ------------------------------------------------------------------ */

/* Sum of the four plaquette leaves in the (mu, nu) plane that start and end
 * at x, all with the same orientation (mu first, then nu). */
static mat3 clover_leaves(const int L[4], const double *U, long x, int mu, int nu)
{
    long xpm = step(L, x, mu, +1), xpn = step(L, x, nu, +1);
    long xmm = step(L, x, mu, -1), xmn = step(L, x, nu, -1);
    long xmm_pn = step(L, xmm, nu, +1);  /* x - mu + nu */
    long xmm_mn = step(L, xmm, nu, -1);  /* x - mu - nu */
    long xpm_mn = step(L, xpm, nu, -1);  /* x + mu - nu */

    /* x -> x+mu -> x+mu+nu -> x+nu -> x */
    mat3 q1 = mul(mul(link_at(U, x, mu), link_at(U, xpm, nu)),
                  mul(dag(link_at(U, xpn, mu)), dag(link_at(U, x, nu))));
    /* x -> x+nu -> x+nu-mu -> x-mu -> x */
    mat3 q2 = mul(mul(link_at(U, x, nu), dag(link_at(U, xmm_pn, mu))),
                  mul(dag(link_at(U, xmm, nu)), link_at(U, xmm, mu)));
    /* x -> x-mu -> x-mu-nu -> x-nu -> x */
    mat3 q3 = mul(mul(dag(link_at(U, xmm, mu)), dag(link_at(U, xmm_mn, nu))),
                  mul(link_at(U, xmm_mn, mu), link_at(U, xmn, nu)));
    /* x -> x-nu -> x-nu+mu -> x+mu -> x */
    mat3 q4 = mul(mul(dag(link_at(U, xmn, nu)), link_at(U, xmn, mu)),
                  mul(link_at(U, xpm_mn, nu), dag(link_at(U, x, mu))));
    return add(add(q1, q2), add(q3, q4));
}

/* F_{mu nu}(x) = (Q - Q^dag)/8, then made traceless */
static mat3 field_strength(const int L[4], const double *U, long x, int mu, int nu)
{
    mat3 q = clover_leaves(L, U, x, mu, nu);
    mat3 f;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f.m[i][j] = (q.m[i][j] - conj(q.m[j][i])) / 8.0;
    cplx tr = (f.m[0][0] + f.m[1][1] + f.m[2][2]) / 3.0;
    for (int i = 0; i < 3; ++i) f.m[i][i] -= tr;
    return f;
}

/* The six planes in the order (x,y) (x,z) (x,t) (y,z) (y,t) (z,t). */
static const int PLANE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

/* F[site][plane][3][3] complex for all sites (the stored clover field). */
void oracle_field_strength(const int *L, const double *U, double *F)
{
    long V = volume_of(L);
    for (long x = 0; x < V; ++x)
        for (int p = 0; p < 6; ++p) {
            mat3 f = field_strength(L, U, x, PLANE[p][0], PLANE[p][1]);
            double *o = F + 18 * (6 * x + p);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    o[2 * (3 * a + b)] = creal(f.m[a][b]);
                    o[2 * (3 * a + b) + 1] = cimag(f.m[a][b]);
                }
        }
}

/* ------------------------------------------------------------------ */
/* The Dirac operator (Sec. 3.3, Dw!)                                  */
/* ------------------------------------------------------------------ */

typedef struct { cplx c[4][3]; } spinor;

static spinor spinor_at(const double *psi, long s)
{
    spinor r;
    const double *p = psi + 24 * s;
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) r.c[al][a] = p[2 * (3 * al + a)] + I * p[2 * (3 * al + a) + 1];
    return r;
}

static void spinor_store(double *psi, long s, const spinor *v)
{
    double *p = psi + 24 * s;
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) {
            p[2 * (3 * al + a)] = creal(v->c[al][a]);
            p[2 * (3 * al + a) + 1] = cimag(v->c[al][a]);
        }
}

/* colour matrix m acting on every spin component, times a scalar phase */
static spinor colour_mul(mat3 m, cplx phase, spinor v)
{
    spinor r;
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) {
            cplx c = 0;
            for (int b = 0; b < 3; ++b) c += m.m[a][b] * v.c[al][b];
            r.c[al][a] = phase * c;
        }
    return r;
}

/* out += coef * (1 + sgn g_mu) v */
static void add_projected(spinor *out, cplx coef, int sgn, int mu, const spinor *v)
{
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) {
            cplx c = v->c[al][a];
            for (int be = 0; be < 4; ++be) c += sgn * G[mu][al][be] * v->c[be][a];
            out->c[al][a] += coef * c;
        }
}

typedef struct {
    int L[4];
    const double *U;
    double kappa, csw;
    double mu; /* twisted mass (mass units): site term + 2 i kappa mu g5; 0 for the Wilson-clover D */
    cplx theta[4];
    double *F; /* clover field F[site][plane][3][3], NULL when csw == 0 */
    int open;   /* open boundary in time: the links U_t(x) with x_t = T - 1 are absent */
    int sf;     /* Schroedinger-functional boundary: slice x_t = 0 is the boundary (identity there) */
    double cF;  /* boundary improvement coefficient on the slices x_t = 0 and T - 1 (open only) */
    double *Uopen; /* the gauge field with the absent links set to zero (owned; open only) */
} dirac_ctx;

static void ctx_init(dirac_ctx *c, const int *L, const double *U, double kappa, double csw,
                     const double *theta)
{
    init_gamma();
    memcpy(c->L, L, sizeof c->L);
    c->U = U;
    c->kappa = kappa;
    c->csw = csw;
    c->mu = 0.0;
    for (int mu = 0; mu < 4; ++mu) c->theta[mu] = theta[2 * mu] + I * theta[2 * mu + 1];
    c->F = NULL;
    c->open = 0;
    c->sf = 0;
    c->cF = 1.0;
    c->Uopen = NULL;
    if (csw != 0.0) {
        c->F = malloc(sizeof(double) * 108 * volume_of(L));
        oracle_field_strength(L, U, c->F);
    }
}

/* Open boundary conditions in time (Sec. 2.1, BC_OPEN): the lattice has no
 * link from the slice x_t = T - 1 to x_t = 0.  Read plainly: that link is
 * zero, so every hop across the time boundary and every clover leaf through
 * it vanish; the slices x_t = 0 and T - 1 get the boundary improvement term
 * (cF - 1) of D_w, i.e. 2 kappa (cF - 1) in the kappa normalisation (cF of
 * DiracParam, Sec. 3.3). */
static void ctx_init_open(dirac_ctx *c, const int *L, const double *U, double kappa, double csw,
                          const double *theta, double cF)
{
    long V = volume_of(L), V3 = (long)L[0] * L[1] * L[2];
    double *Uz = malloc(sizeof(double) * 72 * V);
    memcpy(Uz, U, sizeof(double) * 72 * V);
    for (long s = (long)(L[3] - 1) * V3; s < V; ++s) memset(Uz + 18 * (4 * s + 3), 0, sizeof(double) * 18);
    ctx_init(c, L, Uz, kappa, csw, theta);
    c->Uopen = Uz;
    c->open = 1;
    c->cF = cF;
}

/* Schroedinger-functional boundary conditions (Sec. 2.1, BC_SF_ORBI and
 * BC_SF_AFWB; the two differ only in the boundary weights of improved gauge
 * actions, so for the quark fields of the Wilson-clover operator they read
 * the same).  Read as the standard SF with homogeneous quark boundary values:
 * the time extent T runs from the boundary x_t = 0 to the boundary x_t = T,
 * which is stored as the slice x_t = 0 again (so both boundaries carry the
 * field's links of slice 0); the quark field lives on the slices 1 .. T - 1
 * and vanishes on the boundaries.  So every hop that reaches the slice 0 is
 * absent, the operator is the identity on the slice 0 (which then decouples:
 * a source that vanishes there gives a solution that vanishes there), the
 * clover term on 1 .. T - 1 is built from all links (the boundary ones
 * included), and the slices 1 and T - 1 get the boundary improvement term
 * 2 kappa (cF - 1) (cF = c~_t of DiracParam, Sec. 3.3).  theta_t plays no part. */
static void ctx_init_sf(dirac_ctx *c, const int *L, const double *U, double kappa, double csw,
                        const double *theta, double cF)
{
    long V = volume_of(L), V3 = (long)L[0] * L[1] * L[2];
    ctx_init(c, L, U, kappa, csw, theta); /* the clover field from every link */
    double *Uz = malloc(sizeof(double) * 72 * V);
    memcpy(Uz, U, sizeof(double) * 72 * V);
    for (long s = 0; s < V3; ++s) memset(Uz + 18 * 4 * s, 0, sizeof(double) * 72);   /* links at x_t = 0 */
    for (long s = (long)(L[3] - 1) * V3; s < V; ++s) memset(Uz + 18 * (4 * s + 3), 0, sizeof(double) * 18);
    c->U = Uz; /* the hops */
    c->Uopen = Uz;
    c->sf = 1;
    c->cF = cF;
}

/* slices that carry the boundary improvement term */
static int improved_slice(const dirac_ctx *c, int t)
{
    if (c->open) return t == 0 || t == c->L[3] - 1;
    if (c->sf) return t == 1 || t == c->L[3] - 1;
    return 0;
}

static void ctx_free(dirac_ctx *c)
{
    free(c->F);
    c->F = NULL;
    free(c->Uopen);
    c->Uopen = NULL;
}

static mat3 stored_F(const dirac_ctx *c, long x, int p)
{
    mat3 f;
    const double *q = c->F + 18 * (6 * x + p);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) f.m[a][b] = q[2 * (3 * a + b)] + I * q[2 * (3 * a + b) + 1];
    return f;
}

/* (D psi)(x) for one site x */
static spinor dirac_site(const dirac_ctx *c, const double *psi, long x)
{
    const int *L = c->L;
    int xc[4];
    coords_of(L, x, xc);
    spinor out = spinor_at(psi, x);
    if (c->sf && xc[3] == 0) return out; /* the SF boundary slice */
    for (int mu = 0; mu < 4; ++mu) {
        /* forward: -kappa (1 - g_mu) U~_mu(x) psi(x+mu) */
        long y = step(L, x, mu, +1);
        cplx ph = (xc[mu] == L[mu] - 1) ? c->theta[mu] : 1.0;
        spinor v = colour_mul(link_at(c->U, x, mu), ph, spinor_at(psi, y));
        add_projected(&out, -c->kappa, -1, mu, &v);
        /* backward: -kappa (1 + g_mu) U~_mu(x-mu)^dag psi(x-mu) */
        y = step(L, x, mu, -1);
        ph = (xc[mu] == 0) ? conj(c->theta[mu]) : 1.0;
        v = colour_mul(dag(link_at(c->U, y, mu)), ph, spinor_at(psi, y));
        add_projected(&out, -c->kappa, +1, mu, &v);
    }
    if (c->F) {
        /* + i kappa csw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x) psi(x) */
        spinor s = spinor_at(psi, x);
        for (int p = 0; p < 6; ++p) {
            int mu = PLANE[p][0], nu = PLANE[p][1];
            spinor fs = colour_mul(stored_F(c, x, p), 1.0, s);
            for (int al = 0; al < 4; ++al)
                for (int a = 0; a < 3; ++a) {
                    cplx acc = 0;
                    for (int be = 0; be < 4; ++be) acc += SIGMA[mu][nu][al][be] * fs.c[be][a];
                    out.c[al][a] += I * c->kappa * c->csw * acc;
                }
        }
    }
    if (c->mu != 0.0) {
        /* twisted mass, kappa-normalised: + 2 i kappa mu g5 psi(x) */
        spinor s = spinor_at(psi, x);
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) out.c[al][a] += 2.0 * I * c->kappa * c->mu * G[4][al][al] * s.c[al][a];
    }
    if (improved_slice(c, xc[3])) {
        /* boundary improvement: + 2 kappa (cF - 1) psi(x) on the first and last slice */
        spinor s = spinor_at(psi, x);
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) out.c[al][a] += 2.0 * c->kappa * (c->cF - 1.0) * s.c[al][a];
    }
    return out;
}

static void dirac_apply(const dirac_ctx *c, const double *in, double *out)
{
    long V = volume_of(c->L);
    for (long x = 0; x < V; ++x) {
        spinor r = dirac_site(c, in, x);
        spinor_store(out, x, &r);
    }
}

/* D^dag by definition: every term D(x, y) of the operator adds its conjugate
 * transpose D(x, y)^dag psi(x) into out(y).  Gamma matrices are Hermitian, so
 * (1 -/+ g_mu)^dag = (1 -/+ g_mu); the clover term is Hermitian. */
static void dirac_dagger_apply(const dirac_ctx *c, const double *in, double *out)
{
    const int *L = c->L;
    long V = volume_of(L);
    spinor *acc = calloc((size_t)V, sizeof(spinor));
    for (long x = 0; x < V; ++x) {
        int xc[4];
        coords_of(L, x, xc);
        spinor px = spinor_at(in, x);
        /* diagonal: 1 + clover^dag */
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) acc[x].c[al][a] += px.c[al][a];
        if (c->sf && xc[3] == 0) continue; /* the SF boundary slice: identity, no hops */
        if (c->F) {
            for (int p = 0; p < 6; ++p) {
                int mu = PLANE[p][0], nu = PLANE[p][1];
                /* (i k csw sigma (x) F)^dag = -i k csw sigma (x) F^dag */
                spinor fs = colour_mul(dag(stored_F(c, x, p)), 1.0, px);
                for (int al = 0; al < 4; ++al)
                    for (int a = 0; a < 3; ++a) {
                        cplx s = 0;
                        for (int be = 0; be < 4; ++be) s += conj(SIGMA[mu][nu][be][al]) * fs.c[be][a];
                        acc[x].c[al][a] += -I * c->kappa * c->csw * s;
                    }
            }
        }
        if (c->mu != 0.0) {
            /* (2 i kappa mu g5)^dag = -2 i kappa mu g5 */
            for (int al = 0; al < 4; ++al)
                for (int a = 0; a < 3; ++a)
                    acc[x].c[al][a] += -2.0 * I * c->kappa * c->mu * G[4][al][al] * px.c[al][a];
        }
        if (improved_slice(c, xc[3])) {
            /* the boundary term is real and diagonal: its own adjoint */
            for (int al = 0; al < 4; ++al)
                for (int a = 0; a < 3; ++a) acc[x].c[al][a] += 2.0 * c->kappa * (c->cF - 1.0) * px.c[al][a];
        }
        for (int mu = 0; mu < 4; ++mu) {
            /* term D(x, x+mu) = -kappa (1 - g_mu) U~_mu(x): adjoint goes to x+mu */
            long y = step(L, x, mu, +1);
            cplx ph = (xc[mu] == L[mu] - 1) ? c->theta[mu] : 1.0;
            spinor v = colour_mul(dag(link_at(c->U, x, mu)), conj(ph), px);
            add_projected(&acc[y], -c->kappa, -1, mu, &v);
            /* term D(x, x-mu) = -kappa (1 + g_mu) U~_mu(x-mu)^dag: adjoint to x-mu */
            y = step(L, x, mu, -1);
            ph = (xc[mu] == 0) ? conj(c->theta[mu]) : 1.0;
            v = colour_mul(link_at(c->U, y, mu), conj(ph), px);
            add_projected(&acc[y], -c->kappa, +1, mu, &v);
        }
    }
    for (long x = 0; x < V; ++x) spinor_store(out, x, &acc[x]);
    free(acc);
}

/* theta: 4 complex boundary phase factors as (re, im) pairs */
void oracle_dirac(const int *L, const double *U, double kappa, double csw, const double *theta,
                  const double *in, double *out, int dagger)
{
    dirac_ctx c;
    ctx_init(&c, L, U, kappa, csw, theta);
    if (dagger)
        dirac_dagger_apply(&c, in, out);
    else
        dirac_apply(&c, in, out);
    ctx_free(&c);
}

/* D (or D^dag) applied to n fields stored one after another (used to build
 * the dense matrix of D on tiny lattices column by column). */
void oracle_dirac_many(const int *L, const double *U, double kappa, double csw, const double *theta,
                       long n, const double *in, double *out, int dagger)
{
    dirac_ctx c;
    ctx_init(&c, L, U, kappa, csw, theta);
    long len = 24 * volume_of(L);
    for (long k = 0; k < n; ++k) {
        if (dagger)
            dirac_dagger_apply(&c, in + k * len, out + k * len);
        else
            dirac_apply(&c, in + k * len, out + k * len);
    }
    ctx_free(&c);
}

/* (D psi)(x) at the listed sites only: out[k] is the 12-component spinor at
 * sites[k].  The clover term is computed at those sites only, so this works
 * on large lattices where a full application would be slow. */
void oracle_dirac_sites(const int *L, const double *U, double kappa, double csw,
                        const double *theta, const double *in, long nsites, const long *sites,
                        double *out)
{
    dirac_ctx c;
    memset(&c, 0, sizeof c); /* the periodic Wilson-clover D: no twist, no open boundary */
    init_gamma();
    memcpy(c.L, L, sizeof c.L);
    c.U = U;
    c.kappa = kappa;
    c.csw = csw;
    c.cF = 1.0;
    for (int mu = 0; mu < 4; ++mu) c.theta[mu] = theta[2 * mu] + I * theta[2 * mu + 1];
    double Fx[108];
    for (long k = 0; k < nsites; ++k) {
        long x = sites[k];
        c.F = NULL;
        spinor r = dirac_site(&c, in, x);
        if (csw != 0.0) {
            spinor s = spinor_at(in, x);
            for (int p = 0; p < 6; ++p) {
                mat3 f = field_strength(L, U, x, PLANE[p][0], PLANE[p][1]);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        Fx[18 * p + 2 * (3 * a + b)] = creal(f.m[a][b]);
                        Fx[18 * p + 2 * (3 * a + b) + 1] = cimag(f.m[a][b]);
                    }
            }
            for (int p = 0; p < 6; ++p) {
                int mu = PLANE[p][0], nu = PLANE[p][1];
                mat3 f;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        f.m[a][b] = Fx[18 * p + 2 * (3 * a + b)] + I * Fx[18 * p + 2 * (3 * a + b) + 1];
                spinor fs = colour_mul(f, 1.0, s);
                for (int al = 0; al < 4; ++al)
                    for (int a = 0; a < 3; ++a) {
                        cplx acc = 0;
                        for (int be = 0; be < 4; ++be) acc += SIGMA[mu][nu][al][be] * fs.c[be][a];
                        r.c[al][a] += I * kappa * csw * acc;
                    }
            }
        }
        spinor_store(out, k, &r);
    }
}

/* ------------------------------------------------------------------ */
/* Conjugate gradient on the normal equations (Sec. 3.3, CG!)          */
/* ------------------------------------------------------------------ */

static double norm2(const double *v, long n)
{
    double s = 0;
    for (long i = 0; i < n; ++i) s += v[i] * v[i];
    return s;
}

/* Solves D x = b by CG on D^dag D x = D^dag b (CGNR), starting from the x
 * passed in.  The recursion tracks r = b - D x.  When its norm falls below
 * tol * |b| the residual is recomputed from scratch; the solve stops when
 * that true relative residual |b - D x| / |b| is <= tol, otherwise CG is
 * restarted from the current x.  Returns 0 on convergence, 1 if maxiter was
 * reached; *iters is the number of D^dag D applications, *resid the last true
 * relative residual. */
static int cgnr_ctx(dirac_ctx *cp, const int *L, const double *b, double *x, double tol, int maxiter, int *iters,
                    double *resid)
{
    dirac_ctx c = *cp;
    long n = 24 * volume_of(L);
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    double bnorm = sqrt(norm2(b, n));
    int it = 0, status = 1;
    double rel = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0;
        *resid = 0;
        free(r); free(z); free(p); free(w);
        return 0;
    }
    for (;;) {
        /* (re)start: r = b - D x, z = D^dag r, p = z */
        dirac_apply(&c, x, w);
        for (long i = 0; i < n; ++i) r[i] = b[i] - w[i];
        rel = sqrt(norm2(r, n)) / bnorm;
        if (rel <= tol) { status = 0; break; }
        if (it >= maxiter) break;
        dirac_dagger_apply(&c, r, z);
        memcpy(p, z, sizeof(double) * n);
        double gam = norm2(z, n);
        while (it < maxiter) {
            dirac_apply(&c, p, w);
            double alpha = gam / norm2(w, n);
            for (long i = 0; i < n; ++i) {
                x[i] += alpha * p[i];
                r[i] -= alpha * w[i];
            }
            ++it;
            if (sqrt(norm2(r, n)) <= tol * bnorm) break;
            dirac_dagger_apply(&c, r, z);
            double gnew = norm2(z, n);
            double beta = gnew / gam;
            gam = gnew;
            for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
    }
    *iters = it;
    *resid = rel;
    free(r); free(z); free(p); free(w);
    return status;
}

int oracle_cgnr(const int *L, const double *U, double kappa, double csw, const double *theta,
                const double *b, double *x, double tol, int maxiter, int *iters, double *resid)
{
    dirac_ctx c;
    ctx_init(&c, L, U, kappa, csw, theta);
    int st = cgnr_ctx(&c, L, b, x, tol, maxiter, iters, resid);
    ctx_free(&c);
    return st;
}

/* Twisted-mass Wilson-clover operator (DiracParam's mu, Sec. 3.3), read in
 * the kappa normalisation of oracle_dirac: D(mu) = D + 2 i kappa mu g5, mu in
 * mass units (the paper's D_w gains + i mu g5, and D = 2 kappa D_w).  The
 * twist is applied to a single flavour; D(mu)^dag = D^dag - 2 i kappa mu g5. */
void oracle_dirac_tm(const int *L, const double *U, double kappa, double csw, double mu, const double *theta,
                     const double *in, double *out, int dagger)
{
    dirac_ctx c;
    ctx_init(&c, L, U, kappa, csw, theta);
    c.mu = mu;
    if (dagger)
        dirac_dagger_apply(&c, in, out);
    else
        dirac_apply(&c, in, out);
    ctx_free(&c);
}

/* CGNR of oracle_cgnr on D(mu) */
int oracle_cgnr_tm(const int *L, const double *U, double kappa, double csw, double mu, const double *theta,
                   const double *b, double *x, double tol, int maxiter, int *iters, double *resid)
{
    dirac_ctx c;
    ctx_init(&c, L, U, kappa, csw, theta);
    c.mu = mu;
    int st = cgnr_ctx(&c, L, b, x, tol, maxiter, iters, resid);
    ctx_free(&c);
    return st;
}

/* The operator with open boundary conditions in time (see ctx_init_open):
 * D or D^dag on the T slices of the lattice, theta_t playing no part. */
void oracle_dirac_open(const int *L, const double *U, double kappa, double csw, double cF, const double *theta,
                       const double *in, double *out, int dagger)
{
    dirac_ctx c;
    ctx_init_open(&c, L, U, kappa, csw, theta, cF);
    if (dagger)
        dirac_dagger_apply(&c, in, out);
    else
        dirac_apply(&c, in, out);
    ctx_free(&c);
}

/* CGNR of oracle_cgnr on the open-boundary operator */
int oracle_cgnr_open(const int *L, const double *U, double kappa, double csw, double cF, const double *theta,
                     const double *b, double *x, double tol, int maxiter, int *iters, double *resid)
{
    dirac_ctx c;
    ctx_init_open(&c, L, U, kappa, csw, theta, cF);
    int st = cgnr_ctx(&c, L, b, x, tol, maxiter, iters, resid);
    ctx_free(&c);
    return st;
}

/* Boundary-to-bulk correlators with open boundaries (Sec. 3.3: the
 * propagators from the boundary that give f_P and f_A).  Read as: the six
 * sources W_j(y) = delta_{y_t, 0} P+ e_j, j = 3 s + c with spin s in {0, 1}
 * and colour c, P+ = (1 + g_t) / 2, on every site of the boundary slice
 * (zero spatial momentum); H_j = D^-1 W_j; then per slice x_t
 *   fP[x_t] = sum_xvec sum_j |H_j(x)|^2,
 *   fA[x_t] = - sum_xvec sum_j Re <H_j(x), g_t H_j(x)>   (spin-colour inner product).
 * (P+ e_{j+6} = -P+ e_j, so the six columns are all there is.)  H (may be
 * NULL) receives the columns [6][site][12] complex; iters, resid (may be
 * NULL) per column.  Returns the number of columns that did not converge. */
/* The boundary-to-bulk correlators on the operator of c; sf: the sources sit
 * on the slice 1, W_j(1, yvec) = U_t(0, yvec)^dag P+ e_j (the hop from the SF
 * boundary field), else on the slice 0, W_j(0, yvec) = P+ e_j. */
static int boundary_corr_ctx(dirac_ctx *c, const int *L, const double *U, int sf, double tol, int maxiter,
                             double *fP, double *fA, double *H, int *iters, double *resid)
{
    const long V = volume_of(L), V3 = (long)L[0] * L[1] * L[2], n = 24 * V;
    double *S = H ? H : malloc(sizeof(double) * 6 * n);
    double *w = calloc((size_t)n, sizeof(double));
    int failed = 0;
    for (int j = 0; j < 6; ++j) {
        memset(w, 0, sizeof(double) * n);
        const int s = j / 3, col = j % 3;
        for (long y = 0; y < V3; ++y) {
            const long site = sf ? y + V3 : y; /* the slice 1 or 0 */
            mat3 u = dag(link_at(U, y, 3));    /* U_t(0, yvec)^dag (sf only) */
            for (int al = 0; al < 4; ++al) {  /* (P+ e_j)_al = (delta_{al,s} + (g_t)_{al,s}) / 2 */
                cplx v = 0.5 * ((al == s ? 1.0 : 0.0) + G[3][al][s]);
                for (int a = 0; a < 3; ++a) {
                    cplx va = sf ? v * u.m[a][col] : (a == col ? v : 0.0);
                    w[24 * site + 2 * (3 * al + a)] = creal(va);
                    w[24 * site + 2 * (3 * al + a) + 1] = cimag(va);
                }
            }
        }
        double *x = S + (long)j * n;
        memset(x, 0, sizeof(double) * n);
        int it;
        double res;
        failed += cgnr_ctx(c, L, w, x, tol, maxiter, &it, &res);
        if (iters) iters[j] = it;
        if (resid) resid[j] = res;
    }
    for (int t = 0; t < L[3]; ++t) fP[t] = fA[t] = 0.0;
    for (int j = 0; j < 6; ++j)
        for (long x = 0; x < V; ++x) {
            const int t = (int)(x / V3);
            spinor h = spinor_at(S + (long)j * n, x);
            for (int al = 0; al < 4; ++al)
                for (int a = 0; a < 3; ++a) {
                    cplx gh = 0;
                    for (int be = 0; be < 4; ++be) gh += G[3][al][be] * h.c[be][a];
                    fP[t] += creal(conj(h.c[al][a]) * h.c[al][a]);
                    fA[t] -= creal(conj(h.c[al][a]) * gh);
                }
        }
    free(w);
    if (!H) free(S);
    return failed;
}

int oracle_boundary_corr(const int *L, const double *U, double kappa, double csw, double cF, const double *theta,
                         double tol, int maxiter, double *fP, double *fA, double *H, int *iters, double *resid)
{
    init_gamma();
    dirac_ctx c;
    ctx_init_open(&c, L, U, kappa, csw, theta, cF);
    int failed = boundary_corr_ctx(&c, L, U, 0, tol, maxiter, fP, fA, H, iters, resid);
    ctx_free(&c);
    return failed;
}

void oracle_dirac_sf(const int *L, const double *U, double kappa, double csw, double cF, const double *theta,
                     const double *in, double *out, int dagger)
{
    dirac_ctx c;
    ctx_init_sf(&c, L, U, kappa, csw, theta, cF);
    if (dagger)
        dirac_dagger_apply(&c, in, out);
    else
        dirac_apply(&c, in, out);
    ctx_free(&c);
}

/* CGNR of oracle_cgnr on the SF operator */
int oracle_cgnr_sf(const int *L, const double *U, double kappa, double csw, double cF, const double *theta,
                   const double *b, double *x, double tol, int maxiter, int *iters, double *resid)
{
    dirac_ctx c;
    ctx_init_sf(&c, L, U, kappa, csw, theta, cF);
    int st = cgnr_ctx(&c, L, b, x, tol, maxiter, iters, resid);
    ctx_free(&c);
    return st;
}

/* f_P, f_A with SF boundaries (Sec. 3.3: the boundary-to-bulk propagators of
 * the Dirichlet boundaries give f_P and f_A for SF boundary conditions):
 * H_j = D_SF^-1 W_j with the six sources W_j(1, yvec) = U_t(0, yvec)^dag P+ e_j
 * on every site of the first dynamical slice (the boundary quark field
 * P+ e_j at x_t = 0 carried in by the time link; zero spatial momentum), and
 * fP, fA per slice as for the open boundary (no 1/2, no 1/L^3). */
int oracle_boundary_corr_sf(const int *L, const double *U, double kappa, double csw, double cF, const double *theta,
                            double tol, int maxiter, double *fP, double *fA, double *H, int *iters, double *resid)
{
    init_gamma();
    dirac_ctx c;
    ctx_init_sf(&c, L, U, kappa, csw, theta, cF);
    int failed = boundary_corr_ctx(&c, L, U, 1, tol, maxiter, fP, fA, H, iters, resid);
    ctx_free(&c);
    return failed;
}

/* ------------------------------------------------------------------ */
/* Gauge observables and the Wilson flow (Sec. 3.2)                    */
/* ------------------------------------------------------------------ */

static mat3 scale3(mat3 a, cplx s)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.m[i][j] *= s;
    return a;
}

static cplx trace3(mat3 a) { return a.m[0][0] + a.m[1][1] + a.m[2][2]; }

/* U_p = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
static mat3 plaquette_at(const int L[4], const double *U, long x, int mu, int nu)
{
    long xpm = step(L, x, mu, +1), xpn = step(L, x, nu, +1);
    return mul(mul(link_at(U, x, mu), link_at(U, xpm, nu)), mul(dag(link_at(U, xpn, mu)), dag(link_at(U, x, nu))));
}

/* Gauge observables (plaquette, Eoft_plaq, Eoft_clover, Qtop of Sec. 3.2):
 *   plaq       = (1 / 6V) sum_x sum_{mu<nu} Re tr U_p / 3  (1 for the unit field);
 *   Eplaq[t]   = sum_xvec 2 sum_{mu<nu} Re tr (1 - U_p(x))  (the plaquette action density, summed per slice);
 *   Eclov[t]   = sum_xvec - sum_{mu<nu} tr F_{mu nu}(x)^2  (F the antihermitian clover field above);
 *   Q[t]       = sum_xvec - (1 / 32 pi^2) eps_{mu nu rho sigma} tr F_{mu nu}(x) F_{rho sigma}(x),
 * the epsilon sum written out as 8 [tr F_xy F_zt - tr F_xz F_yt + tr F_xt F_yz]. */
void oracle_gauge_obs(const int *L, const double *U, double *plaq, double *Eplaq, double *Eclov, double *Q)
{
    const long V = volume_of(L), V3 = (long)L[0] * L[1] * L[2];
    double psum = 0.0;
    for (int t = 0; t < L[3]; ++t) Eplaq[t] = Eclov[t] = Q[t] = 0.0;
    for (long x = 0; x < V; ++x) {
        const int t = (int)(x / V3);
        mat3 F[6];
        for (int p = 0; p < 6; ++p) {
            const int mu = PLANE[p][0], nu = PLANE[p][1];
            const double re = creal(trace3(plaquette_at(L, U, x, mu, nu)));
            psum += re / 3.0;
            Eplaq[t] += 2.0 * (3.0 - re);
            F[p] = field_strength(L, U, x, mu, nu);
            Eclov[t] -= creal(trace3(mul(F[p], F[p])));
        }
        /* planes (x,y) (x,z) (x,t) (y,z) (y,t) (z,t) = 0..5 */
        const double e = creal(trace3(mul(F[0], F[5]))) - creal(trace3(mul(F[1], F[4]))) +
                         creal(trace3(mul(F[2], F[3])));
        Q[t] -= 8.0 * e / (32.0 * PI * PI);
    }
    *plaq = psum / (6.0 * V);
}

/* exp(X) by its Taylor series, summed until the terms stop changing the sum */
static mat3 expm3(mat3 X)
{
    mat3 r, term;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.m[i][j] = term.m[i][j] = (i == j) ? 1.0 : 0.0;
    for (int k = 1; k < 60; ++k) {
        term = scale3(mul(term, X), 1.0 / k);
        double n = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                r.m[i][j] += term.m[i][j];
                n += creal(term.m[i][j] * conj(term.m[i][j]));
            }
        if (n < 1e-40) break;
    }
    return r;
}

/* The flow generator Z_mu(x) = -d_{x,mu} S(U) for the Wilson action summed
 * over oriented plaquettes, S = 2 sum_{mu<nu} Re tr (1 - U_p) (Luescher's
 * normalisation of the Wilson flow, cited by Sec. 3.2): with the staple sum
 * S_mu(x) such that Omega = U_mu(x) S_mu(x) closes every plaquette through
 * the link, Z = -(1/2) (Omega - Omega^dag) + (1/6) tr (Omega - Omega^dag). */
static mat3 flow_generator(const int L[4], const double *U, long x, int mu)
{
    mat3 S;
    memset(&S, 0, sizeof S);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        long xpm = step(L, x, mu, +1), xpn = step(L, x, nu, +1), xmn = step(L, x, nu, -1);
        long xpm_mn = step(L, xpm, nu, -1);
        S = add(S, mul(mul(link_at(U, xpm, nu), dag(link_at(U, xpn, mu))), dag(link_at(U, x, nu))));
        S = add(S, mul(mul(dag(link_at(U, xpm_mn, nu)), dag(link_at(U, xmn, mu))), link_at(U, xmn, nu)));
    }
    mat3 om = mul(link_at(U, x, mu), S), Z;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Z.m[i][j] = -0.5 * (om.m[i][j] - conj(om.m[j][i]));
    cplx tr = trace3(Z) / 3.0;
    for (int i = 0; i < 3; ++i) Z.m[i][i] -= tr;
    return Z;
}

static void store_link(double *U, long s, int mu, mat3 m)
{
    double *p = U + 18 * (4 * s + mu);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            p[2 * (3 * a + b)] = creal(m.m[a][b]);
            p[2 * (3 * a + b) + 1] = cimag(m.m[a][b]);
        }
}

/* Wilson flow (Sec. 3.2, flw with the wfl_rk3 scheme): nsteps steps of size
 * eps of the third-order Runge-Kutta integrator of Luescher (JHEP 2010):
 *   W1 = exp(Z0/4) W0,  W2 = exp(8 Z1/9 - 17 Z0/36) W1,
 *   V(t + eps) = exp(3 Z2/4 - 8 Z1/9 + 17 Z0/36) W2,   Z_i = eps Z(W_i),
 * every link updated together at each stage.  U in, Uout out (may alias). */
void oracle_wilson_flow(const int *L, const double *U, double eps, int nsteps, double *Uout)
{
    const long V = volume_of(L), n = 72 * V;
    double *W = malloc(sizeof(double) * n);
    mat3 *Z0 = malloc(sizeof(mat3) * 4 * V), *Z1 = malloc(sizeof(mat3) * 4 * V), *Z2 = malloc(sizeof(mat3) * 4 * V);
    memcpy(W, U, sizeof(double) * n);
    for (int k = 0; k < nsteps; ++k) {
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) Z0[4 * x + mu] = scale3(flow_generator(L, W, x, mu), eps);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu)
                store_link(W, x, mu, mul(expm3(scale3(Z0[4 * x + mu], 0.25)), link_at(W, x, mu)));
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) Z1[4 * x + mu] = scale3(flow_generator(L, W, x, mu), eps);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) {
                mat3 X = add(scale3(Z1[4 * x + mu], 8.0 / 9.0), scale3(Z0[4 * x + mu], -17.0 / 36.0));
                store_link(W, x, mu, mul(expm3(X), link_at(W, x, mu)));
            }
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) Z2[4 * x + mu] = scale3(flow_generator(L, W, x, mu), eps);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) {
                mat3 X = add(add(scale3(Z2[4 * x + mu], 0.75), scale3(Z1[4 * x + mu], -8.0 / 9.0)),
                             scale3(Z0[4 * x + mu], 17.0 / 36.0));
                store_link(W, x, mu, mul(expm3(X), link_at(W, x, mu)));
            }
    }
    memcpy(Uout, W, sizeof(double) * n);
    free(W);
    free(Z0);
    free(Z1);
    free(Z2);
}

/* Covariant lattice Laplacian on a quark field, the generator of the
 * fermion gradient flow (Sec. 3.2, "Gradient flow for fermion fields
 * following the lines of" Luescher, JHEP 2013):
 *   (Delta psi)(x) = sum_mu [ U~_mu(x) psi(x+mu) + U~_mu(x-mu)^dag psi(x-mu)
 *                             - 2 psi(x) ],
 * acting on colour only (the identity in spin), with the boundary phases
 * theta of the Dirac operator on the links that leave the last slice. */
static void laplacian(const int L[4], const double *U, const cplx th[4], const double *in, double *out)
{
    const long V = volume_of(L);
    for (long x = 0; x < V; ++x) {
        int xc[4];
        coords_of(L, x, xc);
        spinor acc = spinor_at(in, x);
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) acc.c[al][a] *= -8.0;
        for (int mu = 0; mu < 4; ++mu) {
            long y = step(L, x, mu, +1);
            cplx ph = (xc[mu] == L[mu] - 1) ? th[mu] : 1.0;
            spinor v = colour_mul(link_at(U, x, mu), ph, spinor_at(in, y));
            y = step(L, x, mu, -1);
            ph = (xc[mu] == 0) ? conj(th[mu]) : 1.0;
            spinor w = colour_mul(dag(link_at(U, y, mu)), ph, spinor_at(in, y));
            for (int al = 0; al < 4; ++al)
                for (int a = 0; a < 3; ++a) acc.c[al][a] += v.c[al][a] + w.c[al][a];
        }
        spinor_store(out, x, &acc);
    }
}

void oracle_laplacian(const int *L, const double *U, const double *theta, const double *in, double *out)
{
    cplx th[4];
    for (int mu = 0; mu < 4; ++mu) th[mu] = theta[2 * mu] + I * theta[2 * mu + 1];
    laplacian(L, U, th, in, out);
}

/* out = a x + b y (n doubles) */
static void axpby(long n, double a, const double *x, double b, const double *y, double *out)
{
    for (long k = 0; k < n; ++k) out[k] = a * x[k] + b * y[k];
}

/* Fermion gradient flow (Sec. 3.2): d chi / dt = Delta(V_t) chi with the gauge
 * field flowed alongside by the Wilson flow of oracle_wilson_flow.  Reading:
 * Luescher's third-order scheme for the pair, the fermion stages evaluated on
 * the gauge stages W0 = V_t, W1, W2 of the same step:
 *   lambda1 = chi + (1/4) eps Delta(W0) chi,
 *   lambda2 = chi + (8/9) eps Delta(W1) lambda1 - (2/9) eps Delta(W0) chi,
 *   chi(t + eps) = lambda1 + (3/4) eps Delta(W2) lambda2
 * (Butcher weights c = (0, 1/4, 2/3), b = (1/4, 0, 3/4): third order).
 * nrhs quark fields chi[nrhs][site][spin][colour]; U, chi in; Uout, chiout
 * out (chiout may alias chi, Uout may alias U). */
void oracle_fermion_flow(const int *L, const double *U, const double *theta, double eps, int nsteps,
                         const double *chi, int nrhs, double *Uout, double *chiout)
{
    const long V = volume_of(L), n = 72 * V, f = 24 * V;
    cplx th[4];
    for (int mu = 0; mu < 4; ++mu) th[mu] = theta[2 * mu] + I * theta[2 * mu + 1];
    double *W = malloc(sizeof(double) * n);
    double *c = malloc(sizeof(double) * f * nrhs), *d0 = malloc(sizeof(double) * f * nrhs);
    double *l1 = malloc(sizeof(double) * f * nrhs), *l2 = malloc(sizeof(double) * f * nrhs);
    double *tmp = malloc(sizeof(double) * f);
    mat3 *Z0 = malloc(sizeof(mat3) * 4 * V), *Z1 = malloc(sizeof(mat3) * 4 * V), *Z2 = malloc(sizeof(mat3) * 4 * V);
    memcpy(W, U, sizeof(double) * n);
    memcpy(c, chi, sizeof(double) * f * nrhs);
    for (int k = 0; k < nsteps; ++k) {
        /* W0 */
        for (int j = 0; j < nrhs; ++j) {
            laplacian(L, W, th, c + f * j, d0 + f * j);
            axpby(f, 1.0, c + f * j, 0.25 * eps, d0 + f * j, l1 + f * j);
        }
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) Z0[4 * x + mu] = scale3(flow_generator(L, W, x, mu), eps);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu)
                store_link(W, x, mu, mul(expm3(scale3(Z0[4 * x + mu], 0.25)), link_at(W, x, mu)));
        /* W1 */
        for (int j = 0; j < nrhs; ++j) {
            laplacian(L, W, th, l1 + f * j, tmp);
            axpby(f, 1.0, c + f * j, 8.0 / 9.0 * eps, tmp, l2 + f * j);
            axpby(f, 1.0, l2 + f * j, -2.0 / 9.0 * eps, d0 + f * j, l2 + f * j);
        }
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) Z1[4 * x + mu] = scale3(flow_generator(L, W, x, mu), eps);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) {
                mat3 X = add(scale3(Z1[4 * x + mu], 8.0 / 9.0), scale3(Z0[4 * x + mu], -17.0 / 36.0));
                store_link(W, x, mu, mul(expm3(X), link_at(W, x, mu)));
            }
        /* W2 */
        for (int j = 0; j < nrhs; ++j) {
            laplacian(L, W, th, l2 + f * j, tmp);
            axpby(f, 1.0, l1 + f * j, 0.75 * eps, tmp, c + f * j);
        }
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) Z2[4 * x + mu] = scale3(flow_generator(L, W, x, mu), eps);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) {
                mat3 X = add(add(scale3(Z2[4 * x + mu], 0.75), scale3(Z1[4 * x + mu], -8.0 / 9.0)),
                             scale3(Z0[4 * x + mu], 17.0 / 36.0));
                store_link(W, x, mu, mul(expm3(X), link_at(W, x, mu)));
            }
    }
    memcpy(Uout, W, sizeof(double) * n);
    memcpy(chiout, c, sizeof(double) * f * nrhs);
    free(W);
    free(c);
    free(d0);
    free(l1);
    free(l2);
    free(tmp);
    free(Z0);
    free(Z1);
    free(Z2);
}

/* The gauge stages W1, W2 of one Wilson-flow step from W0 (those of
 * oracle_wilson_flow). */
static void flow_stage_fields(const int L[4], const double *W0, double eps, double *W1, double *W2)
{
    const long V = volume_of(L);
    mat3 *Z0 = malloc(sizeof(mat3) * 4 * V), *Z1 = malloc(sizeof(mat3) * 4 * V);
    memcpy(W1, W0, sizeof(double) * 72 * V);
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) Z0[4 * x + mu] = scale3(flow_generator(L, W0, x, mu), eps);
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu)
            store_link(W1, x, mu, mul(expm3(scale3(Z0[4 * x + mu], 0.25)), link_at(W0, x, mu)));
    memcpy(W2, W1, sizeof(double) * 72 * V);
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) Z1[4 * x + mu] = scale3(flow_generator(L, W1, x, mu), eps);
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            mat3 X = add(scale3(Z1[4 * x + mu], 8.0 / 9.0), scale3(Z0[4 * x + mu], -17.0 / 36.0));
            store_link(W2, x, mu, mul(expm3(X), link_at(W1, x, mu)));
        }
    free(Z0);
    free(Z1);
}

/* Adjoint flow of quark fields (Sec. 3.2: the correlators of flowed fields
 * need "the integration of the adjoint flow equations", backflowing the
 * fermion field through stored gauge fields).  Reading: the exact adjoint of
 * the discrete forward flow of oracle_fermion_flow.  One forward step is
 *   chi' = M chi,  M = (1 + a D0) + d D2 + d b D2 D1 (1 + a D0) - d c D2 D0
 * (a = eps/4, b = 8 eps/9, c = 2 eps/9, d = 3 eps/4; Di = Delta(Wi), each
 * Hermitian), so one backward step is
 *   eta <- M^dag eta = eta + z2 + z1 + D0 (a eta + a z1 - c z2),
 *   z2 = d D2 eta,  z1 = b D1 z2,
 * applied for the steps in reverse order.  Each step's gauge stages are
 * rebuilt from the field at the step's start, itself obtained by flowing the
 * start field forward (the plain form of the checkpointing the paper
 * describes).  U: the gauge field at flow time 0 (not changed); eta: nrhs
 * fields at t = nsteps eps; etaout (may alias eta): the fields at 0. */
void oracle_fermion_backflow(const int *L, const double *U, const double *theta, double eps, int nsteps,
                             const double *eta, int nrhs, double *etaout)
{
    const long V = volume_of(L), n = 72 * V, f = 24 * V;
    const double a = 0.25 * eps, b = 8.0 / 9.0 * eps, c = 2.0 / 9.0 * eps, d = 0.75 * eps;
    cplx th[4];
    for (int mu = 0; mu < 4; ++mu) th[mu] = theta[2 * mu] + I * theta[2 * mu + 1];
    double *W0 = malloc(sizeof(double) * n), *W1 = malloc(sizeof(double) * n), *W2 = malloc(sizeof(double) * n);
    double *e = malloc(sizeof(double) * f * nrhs), *z1 = malloc(sizeof(double) * f), *z2 = malloc(sizeof(double) * f);
    double *w = malloc(sizeof(double) * f), *t0 = malloc(sizeof(double) * f);
    memcpy(e, eta, sizeof(double) * f * nrhs);
    for (int k = nsteps - 1; k >= 0; --k) {
        oracle_wilson_flow(L, U, eps, k, W0);  /* the field at the start of step k */
        flow_stage_fields(L, W0, eps, W1, W2);
        for (int j = 0; j < nrhs; ++j) {
            double *ej = e + f * j;
            laplacian(L, W2, th, ej, t0);
            axpby(f, d, t0, 0.0, t0, z2);          /* z2 = d D2 eta */
            laplacian(L, W1, th, z2, t0);
            axpby(f, b, t0, 0.0, t0, z1);          /* z1 = b D1 z2 */
            for (long q = 0; q < f; ++q) w[q] = a * ej[q] + a * z1[q] - c * z2[q];
            laplacian(L, W0, th, w, t0);           /* D0 (a eta + a z1 - c z2) */
            for (long q = 0; q < f; ++q) ej[q] = ej[q] + z2[q] + z1[q] + t0[q];
        }
    }
    memcpy(etaout, e, sizeof(double) * f * nrhs);
    free(W0);
    free(W1);
    free(W2);
    free(e);
    free(z1);
    free(z2);
    free(w);
    free(t0);
}

/* ------------------------------------------------------------------ */
/* Quenched Hybrid Monte Carlo (Sec. 3.1, HMC! with leapfrog)           */
/* ------------------------------------------------------------------ */

/* The Wilson gauge action with beta = 2N / g0^2 (N = 3), c0 = 1:
 *   S = (beta / 3) sum_x sum_{mu<nu} Re tr (1 - U_p(x)). */
static double wilson_action(const int L[4], const double *U, double beta)
{
    const long V = volume_of(L);
    double s = 0.0;
    for (long x = 0; x < V; ++x)
        for (int p = 0; p < 6; ++p) s += 3.0 - creal(trace3(plaquette_at(L, U, x, PLANE[p][0], PLANE[p][1])));
    return beta / 3.0 * s;
}

/* Momentum of a link from its 8 real coordinates: P = sum_a pi_a i lambda_a / 2 */
static mat3 momentum_of(const double *pi)
{
    mat3 P;
    memset(&P, 0, sizeof P);
    const double r3 = 1.0 / sqrt(3.0);
    P.m[0][1] += 0.5 * I * pi[0];
    P.m[1][0] += 0.5 * I * pi[0];
    P.m[0][1] += 0.5 * pi[1];
    P.m[1][0] -= 0.5 * pi[1];
    P.m[0][0] += 0.5 * I * pi[2];
    P.m[1][1] -= 0.5 * I * pi[2];
    P.m[0][2] += 0.5 * I * pi[3];
    P.m[2][0] += 0.5 * I * pi[3];
    P.m[0][2] += 0.5 * pi[4];
    P.m[2][0] -= 0.5 * pi[4];
    P.m[1][2] += 0.5 * I * pi[5];
    P.m[2][1] += 0.5 * I * pi[5];
    P.m[1][2] += 0.5 * pi[6];
    P.m[2][1] -= 0.5 * pi[6];
    P.m[0][0] += 0.5 * I * r3 * pi[7];
    P.m[1][1] += 0.5 * I * r3 * pi[7];
    P.m[2][2] -= I * r3 * pi[7];
    return P;
}

/* The HMC force F = -d S (Lie derivative, generators i lambda_a / 2): the
 * Wilson action is beta / 6 times the action of the flow generator, so
 * F = (beta / 6) Z with Z of flow_generator. */
static mat3 hmc_force(const int L[4], const double *U, long x, int mu, double beta)
{
    return scale3(flow_generator(L, U, x, mu), beta / 6.0);
}

/* One trajectory of the quenched HMC (HMC! of Sec. 3.1) with the leapfrog
 * integrator of nsteps steps of size eps:
 *   P += eps/2 F(U);  [U = exp(eps P) U;  P += eps F(U)] x (nsteps - 1);
 *   U = exp(eps P) U;  P += eps/2 F(U),
 * H = -sum tr P^2 + S(U).  mom: the initial momenta as 8 reals per link
 * [site][mu][a] (drawn by the caller); u: a uniform number in (0, 1): the
 * trajectory is accepted when u < exp(-dH).  Uout receives the accepted
 * field (the final one, or U when rejected); returns accepted (0 / 1). */
int oracle_hmc(const int *L, const double *U, double beta, double eps, int nsteps, const double *mom, double u,
               double *Uout, double *dH)
{
    const long V = volume_of(L), n = 72 * V;
    double *W = malloc(sizeof(double) * n);
    mat3 *P = malloc(sizeof(mat3) * 4 * V);
    memcpy(W, U, sizeof(double) * n);
    double K0 = 0.0;
    for (long k = 0; k < 4 * V; ++k) {
        P[k] = momentum_of(mom + 8 * k);
        K0 -= creal(trace3(mul(P[k], P[k])));
    }
    const double H0 = K0 + wilson_action(L, W, beta);
    for (int s = 0; s <= nsteps; ++s) {
        /* momentum: half step at both ends, full steps between */
        const double h = (s == 0 || s == nsteps) ? 0.5 * eps : eps;
        mat3 *F = malloc(sizeof(mat3) * 4 * V);
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu) F[4 * x + mu] = hmc_force(L, W, x, mu, beta);
        for (long k = 0; k < 4 * V; ++k) P[k] = add(P[k], scale3(F[k], h));
        free(F);
        if (s == nsteps) break;
        for (long x = 0; x < V; ++x)
            for (int mu = 0; mu < 4; ++mu)
                store_link(W, x, mu, mul(expm3(scale3(P[4 * x + mu], eps)), link_at(W, x, mu)));
    }
    double K1 = 0.0;
    for (long k = 0; k < 4 * V; ++k) K1 -= creal(trace3(mul(P[k], P[k])));
    *dH = K1 + wilson_action(L, W, beta) - H0;
    const int acc = u < exp(-*dH);
    memcpy(Uout, acc ? W : U, sizeof(double) * n);
    free(W);
    free(P);
    return acc;
}

/* The Wilson action and the force at one link (for the pins) */
double oracle_wilson_action(const int *L, const double *U, double beta) { return wilson_action(L, U, beta); }

void oracle_hmc_force(const int *L, const double *U, double beta, long x, int mu, double *F)
{
    mat3 f = hmc_force(L, U, x, mu, beta);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            F[2 * (3 * a + b)] = creal(f.m[a][b]);
            F[2 * (3 * a + b) + 1] = cimag(f.m[a][b]);
        }
}

/* ------------------------------------------------------------------ */
/* Point-source propagator and pion correlator (Sec. 3.3, propagator!) */
/* ------------------------------------------------------------------ */

/* C(t) = sum_{x vec} sum_{j, alpha, a} |S_j(x vec, t)_{alpha a}|^2 from the 12
 * columns S_j = D^{-1} eta_j, j = 3 spin + colour, prop[j][site][12] complex.
 * t is counted from the source time slice src_t (mod T). */
void oracle_pion_contract(const int *L, const double *prop, int src_t, double *corr)
{
    long V = volume_of(L), V3 = (long)L[0] * L[1] * L[2];
    for (int t = 0; t < L[3]; ++t) corr[t] = 0;
    for (int j = 0; j < 12; ++j)
        for (long s = 0; s < V; ++s) {
            int t = (int)(s / V3);
            int tr = ((t - src_t) % L[3] + L[3]) % L[3];
            const double *q = prop + 24 * (V * j + s);
            double acc = 0;
            for (int k = 0; k < 24; ++k) acc += q[k] * q[k];
            corr[tr] += acc;
        }
}

/* Meson two-point functions for arbitrary spin matrices (the contractions
 * Sec. 3.3 leaves to the user: "any contraction" of the propagator), read as
 * the connected correlator of O_G = psibar G psi with its conjugate at the
 * source, using the gamma5-hermiticity S(x0, x) = g5 S(x, x0)^dag g5:
 *     C_G(t) = - sum_xvec tr[ (G x 1) S(x) (Gbar x 1) g5 S(x)^dag g5 ],
 *     Gbar = g_t G^dag g_t,  x = (xvec, src_t + t mod T),
 * S(x) the 12 x 12 matrix S(x)[3 spin + colour][j] = prop[j][x][...].  For
 * G = g5 this is the pion contraction above.  Written out as plain 12 x 12
 * matrix products per site.  gammas: ng 4x4 complex row-major; corr: ng x T
 * complex (re, im), t from the source slice. */
void oracle_meson_contract(const int *L, const double *prop, int src_t, const double *gammas, int ng,
                           double *corr)
{
    init_gamma();
    const long V = volume_of(L), V3 = (long)L[0] * L[1] * L[2];
    const int T = L[3];
    for (long k = 0; k < 2L * ng * T; ++k) corr[k] = 0;
    static cplx S[12][12], R[12][12], A[12][12], B[12][12], Gs[4][4], Gb[4][4], tmp[4][4];
    for (long s = 0; s < V; ++s) {
        const int t = (int)(s / V3);
        const int tr = ((t - src_t) % T + T) % T;
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) {
                const double *q = prop + 24 * (V * j + s) + 2 * i;
                S[i][j] = q[0] + I * q[1];
            }
        /* R = g5 S^dag g5 (g5 = G[4] acts on the spin index) */
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) R[i][j] = G[4][i / 3][i / 3] * conj(S[j][i]) * G[4][j / 3][j / 3];
        for (int g = 0; g < ng; ++g) {
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b)
                    Gs[a][b] = gammas[2 * (16 * g + 4 * a + b)] + I * gammas[2 * (16 * g + 4 * a + b) + 1];
            /* Gbar = g_t G^dag g_t */
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) {
                    cplx c = 0;
                    for (int l = 0; l < 4; ++l) c += G[3][a][l] * conj(Gs[b][l]);
                    tmp[a][b] = c;
                }
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) {
                    cplx c = 0;
                    for (int l = 0; l < 4; ++l) c += tmp[a][l] * G[3][l][b];
                    Gb[a][b] = c;
                }
            /* A = (G x 1) S, B = (Gbar x 1) R, value = -tr(A B) */
            for (int i = 0; i < 12; ++i)
                for (int j = 0; j < 12; ++j) {
                    cplx ca = 0, cb = 0;
                    for (int l = 0; l < 4; ++l) {
                        ca += Gs[i / 3][l] * S[3 * l + i % 3][j];
                        cb += Gb[i / 3][l] * R[3 * l + i % 3][j];
                    }
                    A[i][j] = ca;
                    B[i][j] = cb;
                }
            cplx v = 0;
            for (int i = 0; i < 12; ++i)
                for (int k = 0; k < 12; ++k) v += A[i][k] * B[k][i];
            corr[2 * (g * T + tr)] -= creal(v);
            corr[2 * (g * T + tr) + 1] -= cimag(v);
        }
    }
}

/* Solves the 12 point sources at src = (x, y, z, t) and contracts them.
 * prop (may be NULL) receives the 12 columns [j][site][12] complex; iters and
 * resid (may be NULL) receive per-column counts and true residuals.  Returns
 * the number of columns that did not converge. */
int oracle_pion(const int *L, const double *U, double kappa, double csw, const double *theta,
                const int *src, double tol, int maxiter, double *corr, double *prop, int *iters,
                double *resid)
{
    long V = volume_of(L), n = 24 * V;
    double *S = prop ? prop : malloc(sizeof(double) * 12 * n);
    double *eta = calloc((size_t)n, sizeof(double));
    long s0 = index_of(L, src);
    int failed = 0;
    for (int j = 0; j < 12; ++j) {
        memset(eta, 0, sizeof(double) * n);
        eta[24 * s0 + 2 * j] = 1.0;
        double *x = S + (long)j * n;
        memset(x, 0, sizeof(double) * n);
        int it;
        double res;
        failed += oracle_cgnr(L, U, kappa, csw, theta, eta, x, tol, maxiter, &it, &res);
        if (iters) iters[j] = it;
        if (resid) resid[j] = res;
    }
    oracle_pion_contract(L, S, src[3], corr);
    free(eta);
    if (!prop) free(S);
    return failed;
}
