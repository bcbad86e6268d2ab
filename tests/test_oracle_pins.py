"""Pins for the FP64 oracle: checks against what the mathematics fixes.

None of these re-types an oracle formula.  They test it against:
  * the Clifford algebra and the chiral-basis convention (gamma matrices);
  * the closed-form free-field (unit-link) Wilson operator and propagator in
    momentum space, including twisted / antiperiodic boundary phases;
  * gamma5-hermiticity and the adjoint identity on rough fields with clover;
  * gauge covariance under a random SU(3) transformation;
  * the clover term: zero at unit links, and the closed form on a constant
    abelian field strength in each of the six planes (orientation, 1/8
    normalisation, traceless projection);
  * dense LU inversion at 2^4 and 4^4 (the solver), kappa = 0 (D = 1);
  * translation invariance of the pion correlator (source-relative t).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))

# Chiral basis, built here from the Pauli matrices (the convention the library
# documents): g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, -1], [-1, 0]].
_S = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]
_Z = np.zeros((2, 2))
_I2 = np.eye(2)
BASIS = [np.block([[_Z, -1j * s], [1j * s, _Z]]) for s in _S] + [np.block([[_Z, -_I2], [-_I2, _Z]])]
G5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(complex)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def g5(psi):
    return np.einsum("ab,...bc->...ac", G5, psi)


# --------------------------------------------------------------------------
# gamma matrices
# --------------------------------------------------------------------------

def test_gamma_clifford_algebra_and_basis():
    g = [oracle.gamma(mu) for mu in range(4)]
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * (mu == nu) * np.eye(4), atol=1e-15)
    gamma5 = oracle.gamma(4)
    assert np.allclose(gamma5, g[3] @ g[0] @ g[1] @ g[2], atol=1e-15)
    assert np.allclose(gamma5, G5, atol=1e-15)
    for mu in range(4):
        assert np.allclose(g[mu], BASIS[mu], atol=0), mu


# --------------------------------------------------------------------------
# free field: closed forms in momentum space
# --------------------------------------------------------------------------

def _momenta(dims, theta):
    """Allowed momenta p_mu = (2 pi n + phi_mu) / L_mu with theta_mu = exp(i phi_mu)."""
    ps = []
    for mu, L in enumerate(dims):
        phi = np.angle(theta[mu])
        ps.append((2 * np.pi * np.arange(L) + phi) / L)
    return ps


def _free_dirac_p(kappa, p):
    """D(p) = 1 - 2 kappa sum cos p + 2 i kappa sum g_mu sin p (4x4 spin matrix)."""
    m = (1 - 2 * kappa * sum(np.cos(pm) for pm in p)) * np.eye(4, dtype=complex)
    for mu in range(4):
        m = m + 2j * kappa * np.sin(p[mu]) * BASIS[mu]
    return m


def _coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x, y, z, t


@pytest.mark.parametrize("theta", [(1, 1, 1, -1), (np.exp(0.7j), np.exp(-1.1j), 1, np.exp(2.3j))])
def test_free_dirac_on_plane_waves(theta):
    dims = (4, 2, 6, 4)
    kappa = 0.13
    U = inputs.unit_gauge_field(dims)
    ps = _momenta(dims, theta)
    x, y, z, t = _coords(dims)
    rng = np.random.default_rng(5)
    for n in [(0, 0, 0, 0), (1, 1, 2, 3), (3, 0, 5, 1)]:
        p = [ps[mu][n[mu]] for mu in range(4)]
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = phase[..., None, None] * u
        want = phase[..., None, None] * (_free_dirac_p(kappa, p) @ u)
        got = oracle.dirac(dims, U, kappa, 1.3, psi, theta=theta)
        assert rel(got, want) < 1e-14


def _free_propagator_x(dims, kappa, theta):
    """S(x, 0) = V^-1 sum_p exp(i p x) S(p), S(p) = (A - 2 i kappa sum g sin p)/(A^2 + 4 kappa^2 sum sin^2).

    Returns shape (T, Z, Y, X, 4, 4) (spin matrix; colour is the identity).
    """
    ps = _momenta(dims, theta)
    x, y, z, t = _coords(dims)
    V = np.prod(dims)
    S = np.zeros(x.shape + (4, 4), dtype=complex)
    P = np.meshgrid(*ps, indexing="ij")
    P = [a.ravel() for a in P]
    for k in range(len(P[0])):
        p = [P[mu][k] for mu in range(4)]
        A = 1 - 2 * kappa * sum(np.cos(pm) for pm in p)
        den = A * A + 4 * kappa ** 2 * sum(np.sin(pm) ** 2 for pm in p)
        num = A * np.eye(4, dtype=complex)
        for mu in range(4):
            num = num - 2j * kappa * np.sin(p[mu]) * BASIS[mu]
        ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        S += ph[..., None, None] * (num / den)
    return S / V


def test_free_propagator_closed_form_dense_and_cg():
    dims = (2, 4, 2, 6)
    kappa = 0.124
    theta = (1, np.exp(0.4j), 1, -1)
    U = inputs.unit_gauge_field(dims)
    S = _free_propagator_x(dims, kappa, theta)
    # column (spin 1, colour 2) of the solver
    eta = inputs.point_source(dims, (0, 0, 0, 0), 1, 2)
    x, it, res, ok = oracle.cgnr(dims, U, kappa, 0.0, eta, theta=theta, tol=1e-13)
    assert ok and res <= 1e-13
    want = np.zeros_like(x)
    want[..., :, 2] = S[..., :, 1]
    assert rel(x, want) < 1e-11
    # dense inverse of the operator matrix agrees with the closed form everywhere
    D = oracle.dirac_matrix(dims, U, kappa, 0.0, theta=theta)
    Dinv = np.linalg.inv(D)
    col = Dinv[:, 3 * 1 + 2].reshape(x.shape)
    assert rel(col, want) < 1e-12


def test_free_pion_correlator_closed_form():
    dims = (4, 4, 4, 8)
    kappa = 0.12
    U = inputs.unit_gauge_field(dims)
    S = _free_propagator_x(dims, kappa, (1, 1, 1, -1))
    # C(t) = sum_xvec tr[S S^dag] with colour identity (factor 3)
    want = 3 * np.einsum("tzyxab,tzyxab->t", S, S.conj()).real
    corr, _, iters, res, failed = oracle.pion(dims, U, kappa, 1.0, (0, 0, 0, 0), tol=1e-13)
    assert failed == 0 and np.all(res <= 1e-13)
    assert rel(corr, want) < 1e-11
    # time-reflection symmetry of the free correlator: C(t) = C(T - t)
    assert np.allclose(corr[1:], corr[1:][::-1], rtol=1e-10)


# --------------------------------------------------------------------------
# twisted mass (DiracParam mu): D(mu) = D + 2 i kappa mu g5
# --------------------------------------------------------------------------

def test_twisted_mass_free_plane_waves_and_propagator():
    """Free field: D(mu)(p) = A + 2 i kappa sum g sin p + i M g5 with M = 2 kappa mu,
    and since g5 anticommutes with every g_mu its inverse is
    (A - 2 i kappa sum g sin p - i M g5) / (A^2 + 4 kappa^2 sum sin^2 p + M^2)."""
    dims = (2, 4, 2, 6)
    kappa, mu = 0.124, 0.35
    M = 2 * kappa * mu
    theta = (1, np.exp(0.4j), 1, -1)
    U = inputs.unit_gauge_field(dims)
    ps = _momenta(dims, theta)
    x, y, z, t = _coords(dims)
    rng = np.random.default_rng(8)
    for n in [(0, 0, 0, 0), (1, 3, 1, 4)]:
        p = [ps[m][n[m]] for m in range(4)]
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = phase[..., None, None] * u
        want = phase[..., None, None] * ((_free_dirac_p(kappa, p) + 1j * M * G5) @ u)
        assert rel(oracle.dirac_tm(dims, U, kappa, 1.1, mu, psi, theta=theta), want) < 1e-14
    # propagator column (spin 2, colour 0) against the momentum sum
    V = np.prod(dims)
    P = [a.ravel() for a in np.meshgrid(*ps, indexing="ij")]
    S = np.zeros(x.shape + (4, 4), dtype=complex)
    for k in range(len(P[0])):
        p = [P[m][k] for m in range(4)]
        A = 1 - 2 * kappa * sum(np.cos(pm) for pm in p)
        den = A * A + 4 * kappa ** 2 * sum(np.sin(pm) ** 2 for pm in p) + M * M
        num = A * np.eye(4, dtype=complex) - 1j * M * G5
        for m in range(4):
            num = num - 2j * kappa * np.sin(p[m]) * BASIS[m]
        S += np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None, None] * (num / den)
    S /= V
    eta = inputs.point_source(dims, (0, 0, 0, 0), 2, 0)
    sol, it, res, ok = oracle.cgnr_tm(dims, U, kappa, 0.0, mu, eta, theta=theta, tol=1e-13)
    assert ok and res <= 1e-13
    want = np.zeros_like(sol)
    want[..., :, 0] = S[..., :, 2]
    assert rel(sol, want) < 1e-11


def test_twisted_mass_identities_on_rough_fields():
    """With clover on a rough field: mu = 0 is the Wilson-clover D; the
    adjoint identity; g5 D(mu) g5 = D(-mu)^dag; and, because D = g5 D^dag g5,
    the cross terms cancel in |D(mu) x|^2 = |D x|^2 + (2 kappa mu)^2 |x|^2."""
    dims, U = _rough()
    k, c = ROUGH["kappa"], ROUGH["csw"]
    mu = 0.27
    th = (1, np.exp(0.3j), 1, -1)
    a = inputs.spinor_field(dims, seed=31)
    b = inputs.spinor_field(dims, seed=32)
    assert np.array_equal(oracle.dirac_tm(dims, U, k, c, 0.0, a, theta=th), oracle.dirac(dims, U, k, c, a, theta=th))
    Da = oracle.dirac_tm(dims, U, k, c, mu, a, theta=th)
    lhs = vdot(b, Da)
    rhs = vdot(oracle.dirac_tm(dims, U, k, c, mu, b, theta=th, dagger=True), a)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    assert rel(g5(oracle.dirac_tm(dims, U, k, c, mu, g5(a), theta=th)),
               oracle.dirac_tm(dims, U, k, c, -mu, a, theta=th, dagger=True)) < 1e-14
    n_mu = np.vdot(Da, Da).real
    n_0 = np.vdot(*(2 * [oracle.dirac(dims, U, k, c, a, theta=th)])).real
    assert abs(n_mu - (n_0 + (2 * k * mu) ** 2 * np.vdot(a, a).real)) <= 1e-13 * n_mu


# --------------------------------------------------------------------------
# rough fields: hermiticity, adjoint, covariance
# --------------------------------------------------------------------------

ROUGH = dict(dims=(4, 2, 4, 6), eps=0.5, kappa=0.137, csw=1.7)


def _rough():
    d = ROUGH["dims"]
    return d, inputs.gauge_field(d, ROUGH["eps"], seed=11)


def test_gamma5_hermiticity_with_clover():
    dims, U = _rough()
    a = inputs.spinor_field(dims, seed=3)
    b = inputs.spinor_field(dims, seed=4)
    th = (1, np.exp(0.3j), 1, -1)
    lhs = vdot(a, oracle.dirac(dims, U, ROUGH["kappa"], ROUGH["csw"], b, theta=th))
    rhs = vdot(g5(oracle.dirac(dims, U, ROUGH["kappa"], ROUGH["csw"], g5(a), theta=th)), b)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)


def test_adjoint_identity():
    dims, U = _rough()
    a = inputs.spinor_field(dims, seed=5)
    b = inputs.spinor_field(dims, seed=6)
    th = (np.exp(0.2j), 1, np.exp(-0.9j), -1)
    k, c = ROUGH["kappa"], ROUGH["csw"]
    lhs = vdot(a, oracle.dirac(dims, U, k, c, b, theta=th))
    rhs = vdot(oracle.dirac(dims, U, k, c, a, theta=th, dagger=True), b)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    # and the dagger equals gamma5 D gamma5 on the same field
    assert rel(oracle.dirac(dims, U, k, c, a, theta=th, dagger=True),
               g5(oracle.dirac(dims, U, k, c, g5(a), theta=th))) < 1e-14


def _transform(U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag (periodic shifts)."""
    out = np.empty_like(U)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    for mu in range(4):
        gshift = np.roll(g, -1, axis=axis[mu])
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gshift, -1, -2))
    return out


def test_gauge_covariance():
    dims, U = _rough()
    g = inputs.gauge_transform(dims, seed=9)
    psi = inputs.spinor_field(dims, seed=10)
    k, c = ROUGH["kappa"], ROUGH["csw"]
    Ug = _transform(U, g)
    lhs = oracle.dirac(dims, Ug, k, c, np.einsum("...ab,...sb->...sa", g, psi))
    rhs = np.einsum("...ab,...sb->...sa", g, oracle.dirac(dims, U, k, c, psi))
    assert rel(lhs, rhs) < 1e-14
    # F transforms covariantly too
    F = oracle.field_strength(dims, U)
    Fg = oracle.field_strength(dims, Ug)
    gd = np.conj(np.swapaxes(g, -1, -2))
    assert rel(Fg, g[..., None, :, :] @ F @ gd[..., None, :, :]) < 1e-13


# --------------------------------------------------------------------------
# clover term
# --------------------------------------------------------------------------

def test_clover_vanishes_at_unit_links():
    dims = (4, 4, 2, 4)
    U = inputs.unit_gauge_field(dims)
    psi = inputs.spinor_field(dims, seed=1)
    assert np.abs(oracle.field_strength(dims, U)).max() == 0
    assert rel(oracle.dirac(dims, U, 0.13, 1.9, psi), oracle.dirac(dims, U, 0.13, 0.0, psi)) == 0


def _abelian_field(dims, mu, nu, T, n, on_nu=True):
    """Constant field strength in the (mu, nu) plane.

    on_nu: U_nu(x) = exp(i phi x_mu T) (F_{mu nu} = +phi T); otherwise
    U_mu(x) = exp(i phi x_nu T) (F_{mu nu} = -phi T).  phi = 2 pi n / L makes
    every plaquette, including the wrapped ones, equal to exp(+-i phi T).
    """
    U = inputs.unit_gauge_field(dims).copy()
    x = _coords(dims)
    if on_nu:
        phi = 2 * np.pi * n / dims[mu]
        arg = phi * x[mu]
        U[..., nu, :, :] = 0
        for a in range(3):
            U[..., nu, a, a] = np.exp(1j * arg * T[a])
    else:
        phi = 2 * np.pi * n / dims[nu]
        arg = phi * x[nu]
        U[..., mu, :, :] = 0
        for a in range(3):
            U[..., mu, a, a] = np.exp(1j * arg * T[a])
    return U, phi


PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


@pytest.mark.parametrize("plane", range(6))
@pytest.mark.parametrize("on_nu", [True, False])
def test_clover_constant_abelian_field(plane, on_nu):
    """D(csw) - D(0) = i kappa csw sigma_{mu nu} (x) F with F = i sin(phi) (T - tr T/3)."""
    mu, nu = PLANES[plane]
    dims = (4, 6, 4, 8)
    kappa, csw = 0.125, 1.3
    for T in [(1.0, -1.0, 0.0), (1.0, 0.0, 0.0)]:  # traceless and not: pins the projection
        U, phi = _abelian_field(dims, mu, nu, T, n=1, on_nu=on_nu)
        sgn = 1.0 if on_nu else -1.0
        Fcol = 1j * sgn * np.sin(phi) * (np.diag(T) - np.trace(np.diag(T)) / 3 * np.eye(3))
        sig = 0.5j * (BASIS[mu] @ BASIS[nu] - BASIS[nu] @ BASIS[mu])
        psi = inputs.spinor_field(dims, seed=2)
        got = oracle.dirac(dims, U, kappa, csw, psi) - oracle.dirac(dims, U, kappa, 0.0, psi)
        want = 1j * kappa * csw * np.einsum("ab,cd,...bd->...ac", sig, Fcol, psi)
        assert rel(got, want) < 1e-13, (plane, T)
        # only that plane is populated in the stored field
        F = oracle.field_strength(dims, U)
        for q in range(6):
            if q == plane:
                assert np.allclose(F[..., q, :, :], Fcol, atol=1e-14)
            else:
                assert np.abs(F[..., q, :, :]).max() < 1e-14


def test_clover_site_term_is_hermitian():
    dims, U = _rough()
    F = oracle.field_strength(dims, U)
    # F is anti-Hermitian and traceless, so i sigma (x) F is Hermitian
    assert np.abs(F + np.conj(np.swapaxes(F, -1, -2))).max() < 1e-15
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-15


# --------------------------------------------------------------------------
# solver: dense inversion, kappa = 0
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims,eps,kappa,csw", [((2, 2, 2, 2), 0.4, 0.13, 1.5), ((4, 4, 4, 4), 0.2, 0.12, 1.0)])
def test_cgnr_matches_dense_inverse(dims, eps, kappa, csw):
    U = inputs.gauge_field(dims, eps, seed=1)
    b = inputs.spinor_field(dims, seed=2)
    D = oracle.dirac_matrix(dims, U, kappa, csw)
    xd = np.linalg.solve(D, b.ravel()).reshape(b.shape)
    x, it, res, ok = oracle.cgnr(dims, U, kappa, csw, b, tol=1e-13)
    assert ok and res <= 1e-13
    assert rel(x, xd) < 1e-11
    # the dense matrix of D^dag is the conjugate transpose of that of D
    if dims == (2, 2, 2, 2):
        Dd = oracle.dirac_matrix(dims, U, kappa, csw, dagger=True)
        assert np.abs(Dd - D.conj().T).max() < 1e-15


def test_kappa_zero_is_identity():
    dims, U = _rough()
    b = inputs.spinor_field(dims, seed=7)
    assert rel(oracle.dirac(dims, U, 0.0, 1.5, b), b) == 0
    x, it, res, ok = oracle.cgnr(dims, U, 0.0, 1.5, b)
    assert ok and rel(x, b) < 1e-15


# --------------------------------------------------------------------------
# pion correlator
# --------------------------------------------------------------------------

def test_pion_translation_invariance_and_positivity():
    dims = (4, 4, 4, 6)
    kappa, csw = 0.12, 1.0
    U = inputs.gauge_field(dims, 0.3, seed=21)
    c0, *_ = oracle.pion(dims, U, kappa, csw, (0, 0, 0, 0), tol=1e-12)
    # shift the whole configuration by (1, 2, 3, 2) and the source with it;
    # time shifts move across the antiperiodic boundary, which changes the
    # propagator by a sign on some slices but leaves |S|^2 unchanged
    shift = (1, 2, 3, 2)
    Us = np.roll(U, shift=(shift[3], shift[2], shift[1], shift[0]), axis=(0, 1, 2, 3))
    c1, *_ = oracle.pion(dims, Us, kappa, csw, shift, tol=1e-12)
    assert np.all(c0 > 0)
    assert rel(c1, c0) < 1e-10


def test_pion_contract_sums_all_columns():
    dims = (2, 2, 2, 4)
    rng = np.random.default_rng(0)
    prop = rng.normal(size=(12, 4, 2, 2, 2, 4, 3)) + 1j * rng.normal(size=(12, 4, 2, 2, 2, 4, 3))
    corr = oracle.pion_contract(dims, prop, src_t=1)
    # Parseval: the total over t is the squared Frobenius norm of the whole propagator
    assert abs(corr.sum() - np.sum(np.abs(prop) ** 2)) < 1e-12 * corr.sum()
    # a propagator living on one time slice only lands at (t - src_t) mod T
    p1 = np.zeros_like(prop)
    p1[:, 0] = prop[:, 0]
    c1 = oracle.pion_contract(dims, p1, src_t=1)
    assert np.count_nonzero(c1) == 1 and c1[3] > 0


def clifford16():
    """The 16 products 1, g_mu, g_mu g_nu (mu<nu), g_mu g_nu g_rho (mu<nu<rho),
    g5 of the chiral basis built in this file; orthonormal: tr(A B^dag) = 4 delta."""
    g = BASIS
    out = [np.eye(4, dtype=complex)] + list(g)
    out += [g[m] @ g[n] for m in range(4) for n in range(m + 1, 4)]
    out += [g[m] @ g[n] @ g[r] for m in range(4) for n in range(m + 1, 4) for r in range(n + 1, 4)]
    out.append(G5)
    return np.array(out)


def _random_prop(dims, seed):
    rng = np.random.default_rng(seed)
    shape = (12, dims[3], dims[2], dims[1], dims[0], 4, 3)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_meson_gamma5_channel_is_the_pion():
    """For G = g5, Gbar = g_t g5 g_t = -g5 and the trace collapses to sum |S|^2
    for any 12-column array: the meson contraction must equal the (separately
    pinned) pion contraction and be real."""
    dims = (2, 4, 2, 6)
    prop = _random_prop(dims, 3)
    c = oracle.meson_contract(dims, prop, 2, [G5])
    p = oracle.pion_contract(dims, prop, 2)
    assert rel(c[0].real, p) < 1e-13
    assert np.max(np.abs(c[0].imag)) < 1e-13 * np.max(p)


def test_meson_free_field_symmetries():
    """Free field on a cubic lattice: every channel is real and symmetric under
    t -> T - t (time reflection with antiperiodic time), and channels related
    by a spatial rotation are equal (x, y, z permuted)."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = inputs.unit_gauge_field(dims)
    _, prop, _, _, failed = oracle.pion(dims, U, kappa, 1.0, (0, 0, 0, 0), tol=1e-13, want_prop=True)
    assert failed == 0
    basis = clifford16()
    c = oracle.meson_contract(dims, prop, 0, basis)
    scale = np.max(np.abs(c))
    assert np.max(np.abs(c.imag)) < 1e-14 * scale
    assert np.max(np.abs(c[:, 1:] - c[:, 1:][:, ::-1])) < 1e-13 * scale
    # clifford16 order: 1, gx, gy, gz, gt, gxgy, gxgz, gxgt, gygz, gygt, gzgt,
    # gxgygz, gxgygt, gxgzgt, gygzgt, g5
    for group in ([1, 2, 3], [5, 6, 8], [7, 9, 10], [12, 13, 14]):
        for g in group[1:]:
            assert np.max(np.abs(c[g] - c[group[0]])) < 1e-13 * scale, (group, g)


def test_meson_fierz_completeness():
    """Completeness of the Clifford basis, sum_A (G_A)_ab (G_A^dag)_cd =
    4 delta_ad delta_bc, turns the sum over all 16 channels into
    -4 sum_xvec tr_c[ tr_s(S g_t) tr_s(g_t g5 S^dag g5) ], computed here with
    einsum on the propagator directly.  Any transposed, conjugated or
    misordered factor in the contraction breaks it."""
    basis = clifford16()
    gram = np.einsum("aij,bij->ab", basis, basis.conj())
    assert np.allclose(gram, 4 * np.eye(16), atol=1e-14)
    dims = (2, 2, 4, 4)
    src_t = 3
    prop = _random_prop(dims, 5)
    c = oracle.meson_contract(dims, prop, src_t, basis)
    gt = BASIS[3]
    g5d = np.diag(G5).real
    # S[t, site, alpha, a, beta, b] = prop[3 beta + b][t, site][alpha, a]
    S = prop.reshape(4, 3, dims[3], -1, 4, 3).transpose(2, 3, 4, 5, 0, 1)
    M = np.einsum("tsAaBb,BA->tsab", S, gt)                      # tr_s(S g_t)
    Tm = np.einsum("A,tsBbAa,B->tsAaBb", g5d, S.conj(), g5d)     # g5 S^dag g5
    N = np.einsum("AB,tsBaAb->tsab", gt, Tm)                      # tr_s(g_t T)
    rhs_t = -4 * np.einsum("tsab,tsba->t", M, N)
    rhs = np.array([rhs_t[(src_t + t) % dims[3]] for t in range(dims[3])])
    assert rel(c.sum(axis=0), rhs) < 1e-13


# --------------------------------------------------------------------------
# the input generator (shared by both sides)
# --------------------------------------------------------------------------

def test_noise_source_generator():
    dims = (8, 8, 8, 6)
    for kind in ("gauss", "z2"):
        eta = inputs.noise_source(dims, 4, seed=3, kind=kind)
        assert np.count_nonzero(np.delete(eta, 4, axis=0)) == 0
        m2 = np.mean(np.abs(eta[4]) ** 2)
        assert abs(m2 - 1.0) < 0.03, (kind, m2)
        assert abs(np.mean(eta[4])) < 0.03
        assert np.array_equal(eta, inputs.noise_source(dims, 4, seed=3, kind=kind))
    z2 = inputs.noise_source(dims, 4, seed=3, kind="z2")[4]
    assert np.allclose(np.abs(z2), 1.0, atol=1e-15)


def test_splitmix64_reference_outputs():
    vals = [int(l) for l in open(os.path.join(HERE, "golden", "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    got = [int(v) for v in inputs.splitmix64(1234567, 0, 5)]
    assert got == vals


def test_gauge_generator_su3_and_mean_plaquette():
    dims = (8, 8, 8, 8)
    eps = 0.4
    U = inputs.gauge_field(dims, eps, seed=3)
    m = U.reshape(-1, 3, 3)
    assert np.abs(m @ np.conj(np.swapaxes(m, 1, 2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(m) - 1).max() < 1e-14
    # i.i.d. adjoint-invariant links: E[Re tr P / 3] = u^4 with u = E[Re tr U / 3]
    u = np.mean(np.trace(m, axis1=1, axis2=2).real) / 3
    Ux, Uy = U[..., 0, :, :], U[..., 1, :, :]
    P = Ux @ np.roll(Uy, -1, axis=3) @ np.conj(np.swapaxes(np.roll(Ux, -1, axis=2), -1, -2)) \
        @ np.conj(np.swapaxes(Uy, -1, -2))
    plaq = np.mean(np.trace(P, axis1=-2, axis2=-1).real) / 3
    assert abs(plaq - u ** 4) < 0.01
    # second-order expansion of the mean link: u = 1 - 2 eps^2 / 3 + O(eps^4)
    assert abs(u - (1 - 2 * eps ** 2 / 3)) < 0.02


# --------------------------------------------------------------------------
# the per-site operator used on lattices too large for a full application
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims,eps,kappa,csw,theta", [
    ((4, 4, 4, 4), 0.5, 0.13, 1.7, (np.exp(0.4j), np.exp(-1.3j), np.exp(2.1j), -np.exp(0.6j))),
    ((4, 6, 2, 10), 0.6, 0.125, 1.5, (np.exp(-0.8j), 1, np.exp(1.7j), -1)),
    ((2, 2, 4, 2), 0.4, 0.14, 2.0, (1, np.exp(0.9j), 1, np.exp(-2.5j))),
    ((6, 4, 4, 8), 0.4, 0.132, 0.0, (1, 1, 1, -1)),
])
def test_dirac_sites_equals_full_operator(dims, eps, kappa, csw, theta):
    """oracle.dirac_sites rebuilds the clover term per site; at every site of
    rough fields with twisted phases in all four directions, extents of 2 and
    ragged extents it must equal the full-lattice operator, and
    g5 D(g5 psi) at the sites must equal the full D^dag (the use the parity
    tests make of it for the adjoint)."""
    U = inputs.gauge_field(dims, eps, seed=21)
    psi = inputs.spinor_field(dims, seed=22)
    V = int(np.prod(dims))
    sites = np.arange(V)
    full = oracle.dirac(dims, U, kappa, csw, psi, theta=theta).reshape(V, 4, 3)
    got = oracle.dirac_sites(dims, U, kappa, csw, psi, sites, theta=theta)
    assert np.max(np.abs(got - full)) <= 1e-14 * np.max(np.abs(full))
    # a shuffled subset returns the same rows in the requested order
    pick = np.random.default_rng(3).permutation(V)[: V // 3]
    assert np.array_equal(oracle.dirac_sites(dims, U, kappa, csw, psi, pick, theta=theta), got[pick])
    dag = oracle.dirac(dims, U, kappa, csw, psi, theta=theta, dagger=True).reshape(V, 4, 3)
    g5d = np.einsum("ab,kbc->kac", G5, oracle.dirac_sites(dims, U, kappa, csw, g5(psi), sites, theta=theta))
    assert np.max(np.abs(g5d - dag)) <= 1e-14 * np.max(np.abs(dag))


# --------------------------------------------------------------------------
# open boundary conditions in time and the boundary-to-bulk correlators
# --------------------------------------------------------------------------

def _time_matrix(T, kappa, cF, p):
    """(4T x 4T) matrix of the free open-boundary operator on e^{i p.x} f(x_t)
    spinors (colour trivial), from the momentum-space form: site term
    1 - kappa sum_k (2 cos p_k - 2 i g_k sin p_k) + 2 kappa (cF - 1) on x_t in
    {0, T-1}; time hops -kappa (1 - g_t) to t+1 and -kappa (1 + g_t) to t-1, no wrap."""
    g = BASIS
    I4 = np.eye(4)
    site = I4 * 1.0 + 0j
    for k in range(3):
        site = site - kappa * (2 * np.cos(p[k]) * I4 - 2j * np.sin(p[k]) * g[k])
    M = np.zeros((4 * T, 4 * T), complex)
    for t in range(T):
        M[4 * t:4 * t + 4, 4 * t:4 * t + 4] = site + (2 * kappa * (cF - 1) * I4 if t in (0, T - 1) else 0)
        if t + 1 < T:
            M[4 * t:4 * t + 4, 4 * (t + 1):4 * t + 8] = -kappa * (I4 - g[3])
        if t - 1 >= 0:
            M[4 * t:4 * t + 4, 4 * (t - 1):4 * t] = -kappa * (I4 + g[3])
    return M


def test_open_free_field_plane_waves_in_space():
    """Unit links, twisted spatial phases: e^{i p.x} f(x_t) with p_k =
    (arg theta_k + 2 pi n_k) / L_k is mapped to e^{i p.x} (M_p f)(x_t)."""
    dims = (4, 6, 2, 7)
    kappa, cF = 0.13, 1.37
    theta = (np.exp(0.4j), np.exp(-1.1j), 1.0, np.exp(0.9j))  # theta_t plays no part
    U = inputs.unit_gauge_field(dims)
    rng = np.random.default_rng(5)
    x, y, z = np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), np.arange(dims[2]), indexing="ij")
    for n in [(0, 0, 0), (1, 2, 1), (3, 5, 0)]:
        p = [(np.angle(theta[k]) + 2 * np.pi * n[k]) / dims[k] for k in range(3)]
        f = rng.normal(size=(dims[3], 4)) + 1j * rng.normal(size=(dims[3], 4))
        wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z)).transpose(2, 1, 0)  # [z, y, x]
        col = rng.normal(size=3) + 1j * rng.normal(size=3)
        psi = np.einsum("zyx,ts,c->tzyxsc", wave, f, col)
        Mf = (_time_matrix(dims[3], kappa, cF, p) @ f.reshape(-1)).reshape(dims[3], 4)
        want = np.einsum("zyx,ts,c->tzyxsc", wave, Mf, col)
        for csw in (0.0, 1.9):  # the clover term vanishes at unit links, also at the boundary
            got = oracle.dirac_open(dims, U, kappa, csw, cF, psi, theta=theta)
            assert rel(got, want) < 1e-14


def test_open_boundary_to_bulk_free_field():
    """f_P, f_A at unit links: the wall sources have zero spatial momentum,
    so H_j(x) = h_j(x_t) with M_0 h_j = delta_{t,0} P+ e_j, and the sums over
    xvec give L^3 times the slice values."""
    dims = (4, 4, 2, 6)
    kappa, cF = 0.12, 0.8
    T, L3 = dims[3], dims[0] * dims[1] * dims[2]
    U = inputs.unit_gauge_field(dims)
    fP, fA, H, iters, res, failed = oracle.boundary_corr(dims, U, kappa, 1.0, cF, tol=1e-13)
    assert failed == 0
    M = _time_matrix(T, kappa, cF, (0.0, 0.0, 0.0))
    Pp = 0.5 * (np.eye(4) + BASIS[3])
    wantP, wantA = np.zeros(T), np.zeros(T)
    for s in range(2):
        src = np.zeros(4 * T, complex)
        src[0:4] = Pp[:, s]
        h = np.linalg.solve(M, src).reshape(T, 4)
        for t in range(T):  # three colours, each the same spin vector
            wantP[t] += 3 * L3 * np.vdot(h[t], h[t]).real
            wantA[t] -= 3 * L3 * np.vdot(h[t], BASIS[3] @ h[t]).real
    assert np.allclose(fP, wantP, rtol=1e-11, atol=0)
    assert np.allclose(fA, wantA, rtol=1e-10, atol=1e-12 * np.max(np.abs(wantP)))


def _zero_boundary_links(dims, U):
    Uz = U.copy()
    Uz[dims[3] - 1, ..., 3, :, :] = 0
    return Uz


def test_open_operator_identities_on_rough_fields():
    """Rough field with clover: the open operator is the periodic operator of
    the field whose time links leaving the last slice are zero, plus
    2 kappa (cF - 1) on the first and last slice; gamma5-hermiticity, the
    adjoint identity and gauge covariance hold; interior slices see the
    periodic clover term."""
    dims = (4, 4, 2, 6)
    kappa, csw, cF = 0.125, 1.6, 1.3
    T = dims[3]
    U = inputs.gauge_field(dims, 0.5, seed=41)
    a = inputs.spinor_field(dims, seed=42)
    b = inputs.spinor_field(dims, seed=43)
    th = (np.exp(0.3j), 1, 1, np.exp(1.2j))
    D = lambda v, dag=False, UU=U: oracle.dirac_open(dims, UU, kappa, csw, cF, v, theta=th, dagger=dag)
    bmask = np.zeros(dims[::-1])[..., None, None]
    bmask[0] = bmask[T - 1] = 1.0
    per = oracle.dirac(dims, _zero_boundary_links(dims, U), kappa, csw, a, theta=th)
    assert rel(D(a), per + 2 * kappa * (cF - 1) * bmask * a) < 1e-14
    assert abs(vdot(a, D(b)) - vdot(g5(D(g5(a))), b)) <= 1e-14 * abs(vdot(a, D(b)))
    assert abs(vdot(a, D(b)) - vdot(D(a, True), b)) <= 1e-14 * abs(vdot(a, D(b)))
    g = inputs.gauge_transform(dims, seed=44)
    Ug = _transform(U, g)
    assert rel(D(np.einsum("...ab,...sb->...sa", g, a), UU=Ug), np.einsum("...ab,...sb->...sa", g, D(a))) < 1e-14
    # clover part away from the boundary slices equals the periodic one
    dc = D(a) - oracle.dirac_open(dims, U, kappa, 0.0, cF, a, theta=th)
    dp = oracle.dirac(dims, U, kappa, csw, a, theta=th) - oracle.dirac(dims, U, kappa, 0.0, a, theta=th)
    assert rel(dc[1:T - 1], dp[1:T - 1]) < 1e-13
    assert rel(dc[0], dp[0]) > 1e-3  # leaves through the missing links are gone


def test_open_cgnr_matches_dense_inverse():
    dims = (2, 2, 2, 4)
    kappa, csw, cF = 0.13, 1.4, 1.2
    U = inputs.gauge_field(dims, 0.4, seed=45)
    b = inputs.spinor_field(dims, seed=46)
    n = 12 * int(np.prod(dims))
    cols = np.eye(n, dtype=complex).reshape((n,) + tuple(dims[::-1]) + (4, 3))
    M = np.stack([oracle.dirac_open(dims, U, kappa, csw, cF, c).reshape(-1) for c in cols], axis=1)
    want = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    x, it, res, ok = oracle.cgnr_open(dims, U, kappa, csw, cF, b, tol=1e-13)
    assert ok and rel(x, want) < 1e-11


# --------------------------------------------------------------------------
# gauge observables and the Wilson flow
# --------------------------------------------------------------------------

def test_flow_and_observables_of_the_unit_field():
    dims = (4, 2, 4, 6)
    U = inputs.unit_gauge_field(dims)
    assert np.array_equal(oracle.wilson_flow(dims, U, 0.05, 3), U)
    plaq, Ep, Ec, Q = oracle.gauge_obs(dims, U)
    assert plaq == 1.0 and not Ep.any() and not Ec.any() and not Q.any()


def test_observables_two_constant_abelian_fluxes():
    """Constant commuting fluxes in the (x,y) and (z,t) planes: the plaquette,
    the plaquette and clover action densities and the clover charge have
    closed forms (F_xy = i sin(phi1) T1', F_zt = i sin(phi2) T2', T' traceless)."""
    dims = (4, 6, 4, 6)
    T1, T2 = (1.0, -1.0, 0.0), (1.0, 0.0, 0.0)
    U, phi1 = _abelian_field(dims, 0, 1, T1, n=1)
    U2, phi2 = _abelian_field(dims, 2, 3, T2, n=1)
    U[..., 3, :, :] = U2[..., 3, :, :]
    V3 = dims[0] * dims[1] * dims[2]
    t1 = np.diag(T1) - np.trace(np.diag(T1)) / 3 * np.eye(3)
    t2 = np.diag(T2) - np.trace(np.diag(T2)) / 3 * np.eye(3)
    rt1 = np.sum(np.cos(phi1 * np.array(T1)))  # Re tr exp(i phi T)
    rt2 = np.sum(np.cos(phi2 * np.array(T2)))
    plaq, Ep, Ec, Q = oracle.gauge_obs(dims, U)
    assert abs(plaq - ((rt1 + rt2) / 3 + 4) / 6) < 1e-15
    assert np.allclose(Ep, V3 * 2 * ((3 - rt1) + (3 - rt2)), rtol=1e-13, atol=0)
    wantE = V3 * (np.sin(phi1) ** 2 * np.trace(t1 @ t1) + np.sin(phi2) ** 2 * np.trace(t2 @ t2))
    assert np.allclose(Ec, wantE, rtol=1e-13, atol=0)
    wantQ = V3 * np.sin(phi1) * np.sin(phi2) * np.trace(t1 @ t2) / (4 * np.pi ** 2)
    assert np.allclose(Q, wantQ, rtol=1e-12, atol=0)


def _diag_field(dims, theta):
    """U_mu(x) = diag(e^{i theta_mu(x)}, e^{-i theta_mu(x)}, 1); theta[t, z, y, x, mu]."""
    U = np.zeros(tuple(dims[::-1]) + (4, 3, 3), complex)
    U[..., 0, 0] = np.exp(1j * theta)
    U[..., 1, 1] = np.exp(-1j * theta)
    U[..., 2, 2] = 1.0
    return U


def test_flow_normalisation_on_a_weak_abelian_wave():
    """A weak transverse abelian wave theta_mu(x) = a cos(p.x) (polarisation
    with p_mu = 0) decays under the flow as theta' = -phat^2 theta, phat^2 =
    sum 4 sin^2(p/2); each RK3 step multiplies it by the third-order Taylor
    polynomial of exp(-phat^2 eps)."""
    dims = (6, 4, 4, 8)
    x = _coords(dims)
    a, eps, n = 1e-5, 0.07, 5
    for mu_pol, p in [(1, (2 * np.pi / 6, 0, 0, 0)), (0, (0, 2 * np.pi / 4, 0, 2 * 2 * np.pi / 8))]:
        phase = sum(p[m] * x[m] for m in range(4))
        theta = np.zeros(tuple(dims[::-1]) + (4,))
        theta[..., mu_pol] = a * np.cos(phase)
        Uf = oracle.wilson_flow(dims, _diag_field(dims, theta), eps, n)
        lam = sum(4 * np.sin(q / 2) ** 2 for q in p) * eps
        g = (1 - lam + lam ** 2 / 2 - lam ** 3 / 6) ** n
        got = np.angle(Uf[..., 0, 0])
        assert np.max(np.abs(got - g * theta)) <= 1e-9 * a
        assert np.max(np.abs(np.angle(Uf[..., 1, 1]) + got)) <= 1e-15 + 1e-9 * a
        assert np.max(np.abs(Uf[..., 2, 2] - 1)) < 1e-14


def test_flow_is_third_order_covariant_unitary_and_lowers_the_action():
    dims = (4, 4, 2, 4)
    U = inputs.gauge_field(dims, 0.3, seed=61)
    t = 0.24
    ref = oracle.wilson_flow(dims, U, t / 192, 192)
    errs = [np.max(np.abs(oracle.wilson_flow(dims, U, t / n, n) - ref)) for n in (6, 12, 24)]
    for e1, e2 in zip(errs, errs[1:]):
        assert 7.0 < e1 / e2 < 11.0, errs  # ~2^3 per halving: third order (second order gives ~4)
    Uf = oracle.wilson_flow(dims, U, 0.02, 5)
    uu = np.einsum("...ba,...bc->...ac", Uf.conj(), Uf)
    assert np.max(np.abs(uu - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(Uf) - 1)) < 1e-13
    g = inputs.gauge_transform(dims, seed=62)
    gd = np.conj(np.swapaxes(g, -1, -2))
    flowed_g = oracle.wilson_flow(dims, _transform(U, g), 0.02, 5)
    assert np.max(np.abs(flowed_g - _transform(Uf, g))) < 1e-13
    S = [np.sum(oracle.gauge_obs(dims, oracle.wilson_flow(dims, U, 0.02, k))[1]) for k in range(0, 6)]
    assert all(b < a for a, b in zip(S, S[1:]))
    assert abs(np.sum(oracle.gauge_obs(dims, _transform(U, g))[1]) - S[0]) < 1e-12 * S[0]
    del gd


# --------------------------------------------------------------------------
# quenched HMC
# --------------------------------------------------------------------------

def _generators():
    return np.array([0.5j * lam for lam in inputs.gell_mann()])  # T^a = i lambda_a / 2, tr T^a T^b = -delta / 2


def _moms(dims, seed):
    n = 8 * 4 * int(np.prod(dims))
    return inputs.normals(seed, 0, n).reshape(tuple(dims[::-1]) + (4, 8))


def test_hmc_force_is_minus_the_lie_derivative_of_the_action():
    """F = -sum_a T^a d_a S with d_a S = d/dh S(exp(h T^a) U_link) at h = 0,
    by central differences of the action."""
    from scipy.linalg import expm
    dims, beta = (4, 2, 2, 4), 5.7
    U = inputs.gauge_field(dims, 0.5, seed=81)
    Tg = _generators()
    for site, mu in [(0, 0), (5, 3), (13, 1)]:
        t, r = divmod(site, dims[0] * dims[1] * dims[2])
        z, r = divmod(r, dims[0] * dims[1])
        y, x = divmod(r, dims[0])
        h = 1e-5
        d = []
        for a in range(8):
            vals = []
            for sg in (+1, -1):
                Up = U.copy()
                Up[t, z, y, x, mu] = expm(sg * h * Tg[a]) @ U[t, z, y, x, mu]
                vals.append(oracle.wilson_action(dims, Up, beta))
            d.append((vals[0] - vals[1]) / (2 * h))
        want = -np.einsum("a,aij->ij", np.array(d), Tg)
        got = oracle.hmc_force(dims, U, beta, site, mu)
        assert np.max(np.abs(got - want)) <= 1e-8 * np.max(np.abs(want)), (site, mu)


def test_hmc_leapfrog_energy_violation_is_second_order_and_covariant():
    dims, beta, tau = (4, 2, 2, 4), 5.7, 0.5
    U = inputs.gauge_field(dims, 0.4, seed=82)
    mom = _moms(dims, 83)
    dHs = [oracle.hmc(dims, U, beta, tau / n, n, mom, 0.5)[1] for n in (8, 16, 32)]
    for a, b in zip(dHs, dHs[1:]):
        assert 3.3 < abs(a) / abs(b) < 4.7, dHs
    # gauge covariance: (U^g, g P g^dag) evolves into (U'^g, ...) with the same dH
    g = inputs.gauge_transform(dims, seed=84)
    Tg = _generators()
    P = np.einsum("...a,aij->...ij", mom, Tg)
    gP = g[..., None, :, :] @ P @ np.conj(np.swapaxes(g, -1, -2))[..., None, :, :]
    mom_g = -2 * np.einsum("aij,...ji->...a", Tg, gP).real
    acc, dH, Uf = oracle.hmc(dims, U, beta, tau / 16, 16, mom, 1e-300)
    acc_g, dH_g, Uf_g = oracle.hmc(dims, _transform(U, g), beta, tau / 16, 16, mom_g, 1e-300)
    assert acc and acc_g
    assert abs(dH - dH_g) < 1e-11
    assert np.max(np.abs(Uf_g - _transform(Uf, g))) < 1e-12


def test_hmc_trivial_cases_and_metropolis():
    dims, beta = (2, 2, 2, 2), 6.0
    U1 = inputs.unit_gauge_field(dims)
    acc, dH, Uf = oracle.hmc(dims, U1, beta, 0.1, 5, np.zeros(tuple(dims[::-1]) + (4, 8)), 0.5)
    assert acc and dH == 0.0 and np.array_equal(Uf, U1)
    U = inputs.gauge_field(dims, 0.4, seed=85)
    mom = _moms(dims, 86)
    _, dH, Uf = oracle.hmc(dims, U, beta, 0.2, 4, mom, 1e-300)
    p = np.exp(-dH)
    acc_lo, _, U_lo = oracle.hmc(dims, U, beta, 0.2, 4, mom, 0.999999 * min(p, 1.0))
    assert acc_lo and np.array_equal(U_lo, Uf)
    if p < 1.0:
        acc_hi, _, U_hi = oracle.hmc(dims, U, beta, 0.2, 4, mom, 1.000001 * p)
        assert not acc_hi and np.array_equal(U_hi, U)


# --------------------------------------------------------------------------
# fermion gradient flow (covariant Laplacian, RK3 with the gauge stages)
# --------------------------------------------------------------------------

def _laplace_p(p):
    """Eigenvalue of the free covariant Laplacian on a plane wave: -sum 4 sin^2(p/2)."""
    return -sum(4 * np.sin(pm / 2) ** 2 for pm in p)


@pytest.mark.parametrize("theta", [(1, 1, 1, -1), (np.exp(0.7j), np.exp(-1.1j), 1, np.exp(2.3j))])
def test_laplacian_free_plane_waves_and_rk3_step_factor(theta):
    dims = (4, 2, 6, 4)
    U = inputs.unit_gauge_field(dims)
    ps = _momenta(dims, theta)
    x, y, z, t = _coords(dims)
    rng = np.random.default_rng(7)
    eps, n = 0.05, 4
    for nn in [(0, 0, 0, 0), (1, 1, 2, 3), (3, 0, 5, 1)]:
        p = [ps[mu][nn[mu]] for mu in range(4)]
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = phase[..., None, None] * u
        lam = _laplace_p(p)
        assert rel(oracle.laplacian(dims, U, psi, theta=theta), lam * psi) < 1e-13
        # unit links stay unit under the Wilson flow, so each step multiplies the
        # plane wave by the RK3 polynomial of h = eps lam
        h = eps * lam
        Uf, cf = oracle.fermion_flow(dims, U, psi, eps, n, theta=theta)
        assert np.max(np.abs(Uf - U)) == 0.0
        assert rel(cf, (1 + h + h * h / 2 + h ** 3 / 6) ** n * psi) < 1e-13


def test_laplacian_is_hermitian_negative_and_covariant():
    dims, U = _rough()
    th = (np.exp(0.4j), 1, np.exp(-0.8j), -1)
    a = inputs.spinor_field(dims, seed=21)
    b = inputs.spinor_field(dims, seed=22)
    la, lb = oracle.laplacian(dims, U, a, theta=th), oracle.laplacian(dims, U, b, theta=th)
    assert abs(vdot(a, lb) - vdot(la, b)) <= 1e-14 * abs(vdot(a, lb))
    assert vdot(a, la).real < 0 and abs(vdot(a, la).imag) <= 1e-13 * abs(vdot(a, la))
    g = inputs.gauge_transform(dims, seed=23)
    ga = np.einsum("...ab,...sb->...sa", g, a)
    lhs = oracle.laplacian(dims, _transform(U, g), ga, theta=th)
    assert rel(lhs, np.einsum("...ab,...sb->...sa", g, la)) < 1e-14
    # colour only: the same operator on every spin component
    a0 = a.copy()
    a0[..., 1:, :] = 0
    assert np.max(np.abs(oracle.laplacian(dims, U, a0, theta=th)[..., 1:, :])) == 0.0


def test_fermion_flow_third_order_gauge_part_covariance_linearity():
    dims = (4, 4, 2, 4)
    U = inputs.gauge_field(dims, 0.3, seed=63)
    chi = inputs.spinor_field(dims, seed=64, nrhs=2)
    th = (1, np.exp(0.5j), 1, -1)
    t = 0.24
    _, ref = oracle.fermion_flow(dims, U, chi, t / 192, 192, theta=th, nrhs=2)
    errs = [np.max(np.abs(oracle.fermion_flow(dims, U, chi, t / n, n, theta=th, nrhs=2)[1] - ref))
            for n in (6, 12, 24)]
    for e1, e2 in zip(errs, errs[1:]):
        assert 6.5 < e1 / e2 < 11.0, errs  # ~2^3 per halving: third order in the coupled system
    Uf, cf = oracle.fermion_flow(dims, U, chi, 0.02, 5, theta=th, nrhs=2)
    assert np.max(np.abs(Uf - oracle.wilson_flow(dims, U, 0.02, 5))) == 0.0  # no back-reaction
    # each field flows on its own and linearly
    _, c0 = oracle.fermion_flow(dims, U, chi[0], 0.02, 5, theta=th)
    _, cs = oracle.fermion_flow(dims, U, 2.0 * chi[0] - 3.0j * chi[1], 0.02, 5, theta=th)
    assert rel(cf[0], c0) < 1e-15
    assert rel(cs, 2.0 * cf[0] - 3.0j * cf[1]) < 1e-13
    # gauge covariance: flowing transformed fields gives the transformed flow
    g = inputs.gauge_transform(dims, seed=65)
    Ufg, cfg = oracle.fermion_flow(dims, _transform(U, g), np.einsum("...ab,...sb->...sa", g, chi), 0.02, 5,
                                   theta=th, nrhs=2)
    assert np.max(np.abs(Ufg - _transform(Uf, g))) < 1e-13
    assert rel(cfg, np.einsum("...ab,...sb->...sa", g, cf)) < 1e-13
    # the flow smooths: the norm decreases step by step
    norms = [np.linalg.norm(oracle.fermion_flow(dims, U, chi, 0.02, k, theta=th, nrhs=2)[1]) for k in range(4)]
    assert all(b < a for a, b in zip(norms, norms[1:]))


def test_fermion_backflow_is_the_adjoint_of_the_flow():
    dims = (4, 4, 2, 4)
    th = (1, np.exp(0.5j), np.exp(-0.2j), -1)
    U = inputs.gauge_field(dims, 0.3, seed=66)
    chi = inputs.spinor_field(dims, seed=67, nrhs=2)
    eta = inputs.spinor_field(dims, seed=68, nrhs=2)
    for eps, n in ((0.03, 4), (0.05, 2)):
        _, fc = oracle.fermion_flow(dims, U, chi, eps, n, theta=th, nrhs=2)
        be = oracle.fermion_backflow(dims, U, eta, eps, n, theta=th, nrhs=2)
        for j in range(2):
            lhs, rhs = vdot(eta[j], fc[j]), vdot(be[j], chi[j])
            assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    assert np.array_equal(oracle.fermion_backflow(dims, U, eta, 0.03, 0, theta=th, nrhs=2), eta)
    # covariance, and the free plane wave takes the forward step factor (h is real)
    g = inputs.gauge_transform(dims, seed=69)
    be = oracle.fermion_backflow(dims, U, eta[0], 0.03, 3, theta=th)
    bg = oracle.fermion_backflow(dims, _transform(U, g), np.einsum("...ab,...sb->...sa", g, eta[0]), 0.03, 3,
                                 theta=th)
    assert rel(bg, np.einsum("...ab,...sb->...sa", g, be)) < 1e-13
    ps = _momenta(dims, th)
    x, y, z, t = _coords(dims)
    p = [ps[mu][(1, 2, 1, 3)[mu]] for mu in range(4)]
    psi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None, None] * np.ones((4, 3))
    h = 0.05 * _laplace_p(p)
    got = oracle.fermion_backflow(dims, inputs.unit_gauge_field(dims), psi, 0.05, 3, theta=th)
    assert rel(got, (1 + h + h * h / 2 + h ** 3 / 6) ** 3 * psi) < 1e-13


# --------------------------------------------------------------------------
# Schroedinger-functional boundaries (slice 0 the boundary)
# --------------------------------------------------------------------------

def _sf_time_matrix(T, kappa, cF, p):
    """(4T x 4T) matrix of the free SF operator on e^{i p.x} f(x_t) spinors: the
    identity on x_t = 0; on 1 .. T-1 the site term of _time_matrix, 2 kappa (cF - 1)
    added on x_t = 1 and T - 1, time hops only between the slices 1 .. T-1."""
    M = _time_matrix(T, kappa, 1.0, p)
    I4 = np.eye(4)
    for t in (1, T - 1):
        M[4 * t:4 * t + 4, 4 * t:4 * t + 4] += 2 * kappa * (cF - 1) * I4
    M[0:4, :] = 0
    M[:, 0:4] = 0
    M[0:4, 0:4] = I4
    return M


def test_sf_free_field_plane_waves_in_space():
    dims = (4, 6, 2, 7)
    kappa, cF = 0.13, 1.37
    theta = (np.exp(0.4j), np.exp(-1.1j), 1.0, np.exp(0.9j))  # theta_t plays no part
    U = inputs.unit_gauge_field(dims)
    rng = np.random.default_rng(6)
    x, y, z = np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), np.arange(dims[2]), indexing="ij")
    for n in [(0, 0, 0), (1, 2, 1), (3, 5, 0)]:
        p = [(np.angle(theta[k]) + 2 * np.pi * n[k]) / dims[k] for k in range(3)]
        f = rng.normal(size=(dims[3], 4)) + 1j * rng.normal(size=(dims[3], 4))
        wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z)).transpose(2, 1, 0)
        col = rng.normal(size=3) + 1j * rng.normal(size=3)
        psi = np.einsum("zyx,ts,c->tzyxsc", wave, f, col)
        Mf = (_sf_time_matrix(dims[3], kappa, cF, p) @ f.reshape(-1)).reshape(dims[3], 4)
        want = np.einsum("zyx,ts,c->tzyxsc", wave, Mf, col)
        for csw in (0.0, 1.9):
            got = oracle.dirac_sf(dims, U, kappa, csw, cF, psi, theta=theta)
            assert rel(got, want) < 1e-14


def test_sf_boundary_to_bulk_free_field():
    """At unit links the sources U_t(0)^dag P+ e_j on slice 1 have zero spatial
    momentum: H_j(x) = h_j(x_t) with M h_j = delta_{t,1} P+ e_j."""
    dims = (4, 4, 2, 6)
    kappa, cF = 0.12, 0.8
    T, L3 = dims[3], dims[0] * dims[1] * dims[2]
    fP, fA, H, iters, res, failed = oracle.boundary_corr_sf(dims, inputs.unit_gauge_field(dims), kappa, 1.0, cF,
                                                            tol=1e-13)
    assert failed == 0
    M = _sf_time_matrix(T, kappa, cF, (0.0, 0.0, 0.0))
    Pp = 0.5 * (np.eye(4) + BASIS[3])
    wantP, wantA = np.zeros(T), np.zeros(T)
    for s in range(2):
        src = np.zeros(4 * T, complex)
        src[4:8] = Pp[:, s]
        h = np.linalg.solve(M, src).reshape(T, 4)
        for t in range(T):
            wantP[t] += 3 * L3 * np.vdot(h[t], h[t]).real
            wantA[t] -= 3 * L3 * np.vdot(h[t], BASIS[3] @ h[t]).real
    assert fP[0] == 0.0 and fA[0] == 0.0
    assert np.allclose(fP, wantP, rtol=1e-11, atol=0)
    assert np.allclose(fA, wantA, rtol=1e-10, atol=1e-12 * np.max(np.abs(wantP)))


def test_sf_operator_identities_on_rough_fields():
    """Rough field with clover: slice 0 is the identity and decouples; on 1 .. T-1
    the SF operator is the periodic operator applied to the field with its slice
    0 zeroed, plus 2 kappa (cF - 1) on the slices 1 and T-1, and the clover term
    there is the periodic one (built from every link); gamma5-hermiticity, the
    adjoint identity and gauge covariance hold."""
    dims = (4, 4, 2, 6)
    kappa, csw, cF = 0.125, 1.6, 1.3
    T = dims[3]
    U = inputs.gauge_field(dims, 0.5, seed=46)
    a = inputs.spinor_field(dims, seed=47)
    b = inputs.spinor_field(dims, seed=48)
    th = (np.exp(0.3j), 1, 1, np.exp(1.2j))
    D = lambda v, dag=False, UU=U: oracle.dirac_sf(dims, UU, kappa, csw, cF, v, theta=th, dagger=dag)
    Da = D(a)
    assert np.array_equal(Da[0], a[0])
    a0 = a.copy()
    a0[0] = 0
    per = oracle.dirac(dims, U, kappa, csw, a0, theta=th)
    bmask = np.zeros(dims[::-1])[..., None, None]
    bmask[1] = bmask[T - 1] = 1.0
    want = per + 2 * kappa * (cF - 1) * bmask * a0
    assert rel(Da[1:], want[1:]) < 1e-14
    assert rel(D(a0)[1:], Da[1:]) < 1e-15  # nothing on 1 .. T-1 reads the slice 0
    assert abs(vdot(a, D(b)) - vdot(g5(D(g5(a))), b)) <= 1e-14 * abs(vdot(a, D(b)))
    assert abs(vdot(a, D(b)) - vdot(D(a, True), b)) <= 1e-14 * abs(vdot(a, D(b)))
    g = inputs.gauge_transform(dims, seed=49)
    Ug = _transform(U, g)
    assert rel(D(np.einsum("...ab,...sb->...sa", g, a), UU=Ug), np.einsum("...ab,...sb->...sa", g, D(a))) < 1e-14


def test_sf_cgnr_matches_dense_inverse_and_vanishes_on_the_boundary():
    dims = (2, 2, 2, 4)
    kappa, csw, cF = 0.13, 1.4, 1.2
    U = inputs.gauge_field(dims, 0.4, seed=50)
    V = int(np.prod(dims))
    n = 12 * V
    M = np.zeros((n, n), complex)
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = 1
        M[:, k] = oracle.dirac_sf(dims, U, kappa, csw, cF, e.reshape(dims[::-1] + (4, 3))).reshape(-1)
    b = inputs.spinor_field(dims, seed=51)
    b[0] = 0  # the boundary carries no source
    x, it, res, ok = oracle.cgnr_sf(dims, U, kappa, csw, cF, b, tol=1e-13)
    assert ok
    xd = np.linalg.solve(M, b.reshape(-1)).reshape(x.shape)
    assert rel(x, xd) < 1e-11
    assert np.max(np.abs(x[0])) < 1e-14 * np.max(np.abs(x))


# --------------------------------------------------------------------------
# boundary-to-bulk correlators and the twisted-mass solve on rough fields
# --------------------------------------------------------------------------

def _dense(apply, dims):
    """The matrix of a linear spinor map, column by column."""
    n = 12 * int(np.prod(dims))
    M = np.zeros((n, n), complex)
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = 1
        M[:, k] = apply(e.reshape(dims[::-1] + (4, 3))).reshape(-1)
    return M


def _fP_fA(H):
    """f_P(t) = sum_j sum_xvec |H_j|^2, f_A(t) = -sum_j sum_xvec H_j^dag g_t H_j."""
    fP = np.einsum("jtzyxsc,jtzyxsc->t", np.conj(H), H).real
    fA = -np.einsum("jtzyxsc,sr,jtzyxrc->t", np.conj(H), BASIS[3], H).real
    return fP, fA


def _boundary_sources(dims, U, slice_t, link):
    """W_j, j = 3 s + c: (P+ e_s) times a colour vector on every site of one
    slice; the colour vector is e_c, or link(U_t(0, yvec)) e_c."""
    lx, ly, lz, lt = dims
    Pp = 0.5 * (np.eye(4) + BASIS[3])
    W = np.zeros((6, lt, lz, ly, lx, 4, 3), complex)
    for j in range(6):
        s, c = divmod(j, 3)
        col = np.zeros((lz, ly, lx, 3), complex)
        if link is None:
            col[..., c] = 1
        else:
            col[...] = link(U[0, ..., 3, :, :])[..., :, c]
        W[j, slice_t] = np.einsum("s,zyxa->zyxsa", Pp[:, s], col)
    return W


def _g_trivial_on_slice0(dims, seed):
    g = inputs.gauge_transform(dims, seed=seed)
    g[0] = np.eye(3)
    return g


@pytest.mark.parametrize("bc", ["open", "sf"])
def test_boundary_to_bulk_on_rough_fields(bc):
    """With clover on a rough field: every H_j is the solve of its source (a
    dense inverse), f_P and f_A follow from H, f_P > 0 on the dynamical
    slices, and f_P, f_A do not change under a gauge transformation that is
    the identity on slice 0 (the boundary). For SF that invariance holds only
    because the source carries U_t(0)^dag: the same source with U_t(0) in
    its place (a plausible slip, invisible at unit links) is shown to break it."""
    dims = (2, 2, 2, 4)
    kappa, csw, cF = 0.13, 1.4, 1.2
    th = (np.exp(0.4j), 1, np.exp(-0.7j), 1)
    U = inputs.gauge_field(dims, 0.45, seed=60)
    if bc == "open":
        corr = lambda UU: oracle.boundary_corr(dims, UU, kappa, csw, cF, theta=th, tol=1e-13, want_prop=True)
        Dop = lambda UU: (lambda v: oracle.dirac_open(dims, UU, kappa, csw, cF, v, theta=th))
        src = lambda UU, link=None: _boundary_sources(dims, UU, 0, None)
    else:
        corr = lambda UU: oracle.boundary_corr_sf(dims, UU, kappa, csw, cF, theta=th, tol=1e-13, want_prop=True)
        Dop = lambda UU: (lambda v: oracle.dirac_sf(dims, UU, kappa, csw, cF, v, theta=th))
        dag = lambda u: np.conj(np.swapaxes(u, -1, -2))
        src = lambda UU, link=dag: _boundary_sources(dims, UU, 1, link)
    fP, fA, H, iters, res, failed = corr(U)
    assert failed == 0 and np.all(res <= 1e-13)
    M = _dense(Dop(U), dims)
    W = src(U)
    Hd = np.linalg.solve(M, W.reshape(6, -1).T).T.reshape(W.shape)
    assert rel(H, Hd) < 1e-11
    wP, wA = _fP_fA(Hd)
    assert np.allclose(fP, wP, rtol=1e-11, atol=0)
    assert np.allclose(fA, wA, rtol=1e-10, atol=1e-12 * np.max(wP))
    first = 0 if bc == "open" else 1
    assert np.all(fP[first:] > 0)
    if bc == "sf":
        assert fP[0] == 0.0 and fA[0] == 0.0
    Ug = _transform(U, _g_trivial_on_slice0(dims, 61))
    gP, gA, *_ = corr(Ug)
    assert np.allclose(gP, fP, rtol=1e-10, atol=0)
    assert np.allclose(gA, fA, rtol=1e-9, atol=1e-11 * np.max(fP))
    if bc == "sf":
        def fP_of(UU, link):
            W = src(UU, link)
            Hs = np.linalg.solve(_dense(Dop(UU), dims), W.reshape(6, -1).T).T.reshape(W.shape)
            return _fP_fA(Hs)[0]
        plain = lambda u: u
        assert np.max(np.abs(fP_of(Ug, plain) - fP_of(U, plain))) > 1e-3 * np.max(fP)


def test_twisted_mass_cgnr_matches_dense_inverse():
    """D(mu) x = b on a rough field with clover and twisted boundary phases;
    the CGNR solution equals the dense inverse, and mu -> -mu gives the
    solve of the gamma5-sandwiched adjoint: D(-mu) = g5 D(mu)^dag g5."""
    dims = (2, 2, 2, 4)
    kappa, csw, mu = 0.13, 1.4, 0.21
    th = (np.exp(0.3j), 1, 1, np.exp(1.1j))
    U = inputs.gauge_field(dims, 0.4, seed=62)
    b = inputs.spinor_field(dims, seed=63)
    M = _dense(lambda v: oracle.dirac_tm(dims, U, kappa, csw, mu, v, theta=th), dims)
    x, it, res, ok = oracle.cgnr_tm(dims, U, kappa, csw, mu, b, theta=th, tol=1e-13)
    assert ok and res <= 1e-13
    assert rel(x, np.linalg.solve(M, b.reshape(-1)).reshape(x.shape)) < 1e-11
    y, it2, res2, ok2 = oracle.cgnr_tm(dims, U, kappa, csw, -mu, b, theta=th, tol=1e-13)
    g5mat = np.kron(np.eye(int(np.prod(dims))), np.kron(G5, np.eye(3)))
    Mm = g5mat @ np.conj(M.T) @ g5mat
    assert ok2 and rel(y, np.linalg.solve(Mm, b.reshape(-1)).reshape(y.shape)) < 1e-11
