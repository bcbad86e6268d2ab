"""FP64 CPU oracle for the Wilson-clover propagator path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  The arithmetic lives in
``oracle.c`` (plain C, FP64, single thread); this wrapper only compiles it and
marshals numpy arrays.  Every function documents the paper passage it follows
in ``oracle.c``.

Layouts (shared with the library's host ABI): gauge ``U[t,z,y,x,mu,3,3]``,
spinor ``psi[t,z,y,x,spin,colour]``, complex128; ``dims = (Lx, Ly, Lz, T)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

DEFAULT_THETA = (1.0, 1.0, 1.0, -1.0)


def build(force: bool = False) -> str:
    """Compiles oracle.c into _build/liboracle.so with gcc (no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fcx-limited-range", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.oracle_gamma.argtypes = [ctypes.c_int, dp]
        lib.oracle_field_strength.argtypes = [ip, dp, dp]
        lib.oracle_dirac.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp, ctypes.c_int]
        lib.oracle_dirac_many.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, ctypes.c_long, dp, dp,
                                          ctypes.c_int]
        lib.oracle_dirac_sites.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, dp,
                                           ctypes.c_long, lp, dp]
        lib.oracle_cgnr.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                    ctypes.c_double, ctypes.c_int, ip, dp]
        lib.oracle_cgnr.restype = ctypes.c_int
        lib.oracle_pion_contract.argtypes = [ip, dp, ctypes.c_int, dp]
        lib.oracle_meson_contract.argtypes = [ip, dp, ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_dirac_tm.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                        ctypes.c_int]
        lib.oracle_cgnr_tm.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                       ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double)]
        lib.oracle_pion.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.c_double, ctypes.c_int, dp, dp, ip, dp]
        lib.oracle_dirac_open.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                          ctypes.c_int]
        lib.oracle_cgnr_open.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                         ctypes.c_double, ctypes.c_int, ip, dp]
        lib.oracle_cgnr_open.restype = ctypes.c_int
        lib.oracle_boundary_corr.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                             ctypes.c_double, ctypes.c_int, dp, dp, dp, ip, dp]
        lib.oracle_boundary_corr.restype = ctypes.c_int
        lib.oracle_dirac_sf.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                        ctypes.c_int]
        lib.oracle_cgnr_sf.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                       ctypes.c_double, ctypes.c_int, ip, dp]
        lib.oracle_cgnr_sf.restype = ctypes.c_int
        lib.oracle_boundary_corr_sf.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                                ctypes.c_double, ctypes.c_int, dp, dp, dp, ip, dp]
        lib.oracle_boundary_corr_sf.restype = ctypes.c_int
        lib.oracle_gauge_obs.argtypes = [ip, dp, dp, dp, dp, dp]
        lib.oracle_wilson_flow.argtypes = [ip, dp, ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_laplacian.argtypes = [ip, dp, dp, dp, dp]
        lib.oracle_fermion_flow.argtypes = [ip, dp, dp, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.oracle_fermion_backflow.argtypes = [ip, dp, dp, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_hmc.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, ctypes.c_double, dp,
                                   dp]
        lib.oracle_hmc.restype = ctypes.c_int
        lib.oracle_wilson_action.argtypes = [ip, dp, ctypes.c_double]
        lib.oracle_wilson_action.restype = ctypes.c_double
        lib.oracle_hmc_force.argtypes = [ip, dp, ctypes.c_double, ctypes.c_long, ctypes.c_int, dp]
        lib.oracle_pion.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(dims):
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    assert d.shape == (4,)
    return d


def _theta(theta):
    th = np.asarray(theta, dtype=np.complex128)
    assert th.shape == (4,)
    return np.ascontiguousarray(th)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3 = x,y,z,t) or gamma5 (mu = 4) as a 4x4 complex matrix."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().oracle_gamma(mu, _dp(out))
    return out


def field_strength(dims, U) -> np.ndarray:
    """Clover field F_{mu nu}(x), shape (T,Z,Y,X,6,3,3), planes xy xz xt yz yt zt."""
    lx, ly, lz, lt = dims
    U = _c128(U)
    out = np.zeros((lt, lz, ly, lx, 6, 3, 3), dtype=np.complex128)
    d = _dims(dims)
    _load().oracle_field_strength(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), _dp(out))
    return out


def dirac(dims, U, kappa, csw, psi, theta=DEFAULT_THETA, dagger=False) -> np.ndarray:
    """Full-lattice D psi (or D^dag psi) in FP64."""
    U, psi, th, d = _c128(U), _c128(psi), _theta(theta), _dims(dims)
    out = np.zeros_like(psi)
    _load().oracle_dirac(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw,
                         _dp(th), _dp(psi), _dp(out), int(bool(dagger)))
    return out


def dirac_matrix(dims, U, kappa, csw, theta=DEFAULT_THETA, dagger=False) -> np.ndarray:
    """Dense matrix of D (or D^dag), shape (12V, 12V), built column by column."""
    U, th, d = _c128(U), _theta(theta), _dims(dims)
    n = 12 * int(np.prod(dims))
    eye = np.eye(n, dtype=np.complex128)
    out = np.zeros_like(eye)
    _load().oracle_dirac_many(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, _dp(th),
                              n, _dp(eye), _dp(out), int(bool(dagger)))
    return out.T.copy()


def dirac_sites(dims, U, kappa, csw, psi, sites, theta=DEFAULT_THETA) -> np.ndarray:
    """(D psi)(x) at the lexicographic site indices ``sites``, shape (n, 4, 3)."""
    U, psi, th, d = _c128(U), _c128(psi), _theta(theta), _dims(dims)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.zeros((len(s), 4, 3), dtype=np.complex128)
    _load().oracle_dirac_sites(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw,
                               _dp(th), _dp(psi), len(s), s.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                               _dp(out))
    return out


def cgnr(dims, U, kappa, csw, b, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000, x0=None):
    """Solves D x = b by CGNR to true relative residual ``tol``.

    Returns (x, iterations, true relative residual, converged).
    """
    U, b, th, d = _c128(U), _c128(b), _theta(theta), _dims(dims)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    it = ctypes.c_int(0)
    res = ctypes.c_double(0)
    st = _load().oracle_cgnr(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, _dp(th),
                             _dp(b), _dp(x), tol, maxiter, ctypes.byref(it), ctypes.byref(res))
    return x, it.value, res.value, st == 0


def dirac_tm(dims, U, kappa, csw, mu, psi, theta=DEFAULT_THETA, dagger=False) -> np.ndarray:
    """Twisted-mass D(mu) psi = D psi + 2 i kappa mu g5 psi (or its adjoint), FP64."""
    U, psi, th, d = _c128(U), _c128(psi), _theta(theta), _dims(dims)
    out = np.zeros_like(psi)
    _load().oracle_dirac_tm(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, mu,
                            _dp(th), _dp(psi), _dp(out), int(bool(dagger)))
    return out


def cgnr_tm(dims, U, kappa, csw, mu, b, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000):
    """Solves D(mu) x = b by CGNR; returns (x, iterations, true relative residual, converged)."""
    U, b, th, d = _c128(U), _c128(b), _theta(theta), _dims(dims)
    x = np.zeros_like(b)
    it = ctypes.c_int(0)
    res = ctypes.c_double(0)
    st = _load().oracle_cgnr_tm(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, mu, _dp(th),
                                _dp(b), _dp(x), tol, maxiter, ctypes.byref(it), ctypes.byref(res))
    return x, it.value, res.value, st == 0


def dirac_open(dims, U, kappa, csw, cF, psi, theta=DEFAULT_THETA, dagger=False) -> np.ndarray:
    """D (or D^dag) with open boundary conditions in time and boundary coefficient cF."""
    U, psi, th, d = _c128(U), _c128(psi), _theta(theta), _dims(dims)
    out = np.zeros_like(psi)
    _load().oracle_dirac_open(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, cF, _dp(th),
                              _dp(psi), _dp(out), int(bool(dagger)))
    return out


def cgnr_open(dims, U, kappa, csw, cF, b, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000):
    """Solves the open-boundary D x = b by CGNR; returns (x, iterations, true relative residual, converged)."""
    U, b, th, d = _c128(U), _c128(b), _theta(theta), _dims(dims)
    x = np.zeros_like(b)
    it = ctypes.c_int(0)
    res = ctypes.c_double(0)
    st = _load().oracle_cgnr_open(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, cF, _dp(th),
                                  _dp(b), _dp(x), tol, maxiter, ctypes.byref(it), ctypes.byref(res))
    return x, it.value, res.value, st == 0


def boundary_corr(dims, U, kappa, csw, cF, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000, want_prop=False):
    """Open-boundary f_P(x_t), f_A(x_t) from the six P+ wall sources on slice 0.

    Returns (fP, fA, H or None [6, T, Z, Y, X, 4, 3], iterations[6], residuals[6], failed_columns)."""
    lx, ly, lz, lt = dims
    U, th, d = _c128(U), _theta(theta), _dims(dims)
    fP, fA = np.zeros(lt), np.zeros(lt)
    H = np.zeros((6, lt, lz, ly, lx, 4, 3), dtype=np.complex128) if want_prop else None
    iters = np.zeros(6, dtype=np.int32)
    res = np.zeros(6)
    failed = _load().oracle_boundary_corr(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, cF,
                                          _dp(th), tol, maxiter, _dp(fP), _dp(fA),
                                          _dp(H) if H is not None else None,
                                          iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(res))
    return fP, fA, H, iters, res, failed


def dirac_sf(dims, U, kappa, csw, cF, psi, theta=DEFAULT_THETA, dagger=False) -> np.ndarray:
    """D (or D^dag) with Schroedinger-functional boundaries (slice 0 the boundary) and coefficient cF."""
    U, psi, th, d = _c128(U), _c128(psi), _theta(theta), _dims(dims)
    out = np.zeros_like(psi)
    _load().oracle_dirac_sf(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, cF, _dp(th),
                            _dp(psi), _dp(out), int(bool(dagger)))
    return out


def cgnr_sf(dims, U, kappa, csw, cF, b, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000):
    """Solves the SF D x = b by CGNR; returns (x, iterations, true relative residual, converged)."""
    U, b, th, d = _c128(U), _c128(b), _theta(theta), _dims(dims)
    x = np.zeros_like(b)
    it = ctypes.c_int(0)
    res = ctypes.c_double(0)
    st = _load().oracle_cgnr_sf(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, cF, _dp(th),
                                _dp(b), _dp(x), tol, maxiter, ctypes.byref(it), ctypes.byref(res))
    return x, it.value, res.value, st == 0


def boundary_corr_sf(dims, U, kappa, csw, cF, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000, want_prop=False):
    """SF f_P(x_t), f_A(x_t) from the six sources U_t(0)^dag P+ e_j on slice 1.

    Returns (fP, fA, H or None [6, T, Z, Y, X, 4, 3], iterations[6], residuals[6], failed_columns)."""
    lx, ly, lz, lt = dims
    U, th, d = _c128(U), _theta(theta), _dims(dims)
    fP, fA = np.zeros(lt), np.zeros(lt)
    H = np.zeros((6, lt, lz, ly, lx, 4, 3), dtype=np.complex128) if want_prop else None
    iters = np.zeros(6, dtype=np.int32)
    res = np.zeros(6)
    failed = _load().oracle_boundary_corr_sf(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw,
                                             cF, _dp(th), tol, maxiter, _dp(fP), _dp(fA),
                                             _dp(H) if H is not None else None,
                                             iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(res))
    return fP, fA, H, iters, res, failed


def gauge_obs(dims, U):
    """(plaquette average, Eplaq[T], Eclov[T], Q[T]): per-slice sums of the action density
    (plaquette and clover) and of the clover topological charge density."""
    U, d = _c128(U), _dims(dims)
    T = dims[3]
    plaq = ctypes.c_double(0)
    Ep, Ec, Q = np.zeros(T), np.zeros(T), np.zeros(T)
    _load().oracle_gauge_obs(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), ctypes.byref(plaq), _dp(Ep),
                             _dp(Ec), _dp(Q))
    return plaq.value, Ep, Ec, Q


def wilson_flow(dims, U, eps, nsteps) -> np.ndarray:
    """The gauge field after nsteps RK3 Wilson-flow steps of size eps."""
    U, d = _c128(U), _dims(dims)
    out = np.zeros_like(U)
    _load().oracle_wilson_flow(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), float(eps), int(nsteps),
                               _dp(out))
    return out


def laplacian(dims, U, psi, theta=DEFAULT_THETA) -> np.ndarray:
    """Covariant Laplacian (Delta psi)(x) = sum_mu [U~ psi(x+mu) + U~^dag psi(x-mu) - 2 psi(x)], colour only."""
    U, psi, th, d = _c128(U), _c128(psi), _theta(theta), _dims(dims)
    out = np.zeros_like(psi)
    _load().oracle_laplacian(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), _dp(th), _dp(psi), _dp(out))
    return out


def fermion_flow(dims, U, chi, eps, nsteps, theta=DEFAULT_THETA, nrhs=1):
    """Gauge and quark fields after nsteps RK3 steps of the coupled Wilson / fermion flow.
    chi: nrhs fields [nrhs, T, Z, Y, X, 4, 3] (or one field).  Returns (U_flowed, chi_flowed)."""
    U, chi, th, d = _c128(U), _c128(chi), _theta(theta), _dims(dims)
    assert chi.size == nrhs * 12 * int(np.prod(dims))
    Uo, co = np.zeros_like(U), np.zeros_like(chi)
    _load().oracle_fermion_flow(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), _dp(th), float(eps),
                                int(nsteps), _dp(chi), int(nrhs), _dp(Uo), _dp(co))
    return Uo, co


def fermion_backflow(dims, U, eta, eps, nsteps, theta=DEFAULT_THETA, nrhs=1):
    """Adjoint (back-)flow of nrhs quark fields from t = nsteps eps to 0 through the
    Wilson flow that starts at U (the exact adjoint of fermion_flow's discrete steps)."""
    U, eta, th, d = _c128(U), _c128(eta), _theta(theta), _dims(dims)
    assert eta.size == nrhs * 12 * int(np.prod(dims))
    out = np.zeros_like(eta)
    _load().oracle_fermion_backflow(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), _dp(th), float(eps),
                                    int(nsteps), _dp(eta), int(nrhs), _dp(out))
    return out


def hmc(dims, U, beta, eps, nsteps, mom, u):
    """One leapfrog HMC trajectory; mom: momenta [T, Z, Y, X, mu, 8] (coordinates on i lambda_a / 2),
    u: uniform in (0, 1).  Returns (accepted, dH, field after the trajectory or U if rejected)."""
    U, d = _c128(U), _dims(dims)
    m = np.ascontiguousarray(mom, dtype=np.float64)
    assert m.size == 8 * 4 * int(np.prod(dims))
    out = np.zeros_like(U)
    dH = ctypes.c_double(0)
    acc = _load().oracle_hmc(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), float(beta), float(eps),
                             int(nsteps), _dp(m), float(u), _dp(out), ctypes.byref(dH))
    return bool(acc), dH.value, out


def wilson_action(dims, U, beta) -> float:
    U, d = _c128(U), _dims(dims)
    return _load().oracle_wilson_action(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), float(beta))


def hmc_force(dims, U, beta, site, mu) -> np.ndarray:
    """The HMC force F = -dS at the link (lexicographic site, mu), 3x3 complex."""
    U, d = _c128(U), _dims(dims)
    out = np.zeros((3, 3), dtype=np.complex128)
    _load().oracle_hmc_force(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), float(beta), int(site), int(mu),
                             _dp(out))
    return out


def pion_contract(dims, prop, src_t) -> np.ndarray:
    """C(t) from 12 propagator columns prop[j, t, z, y, x, spin, colour]."""
    prop, d = _c128(prop), _dims(dims)
    out = np.zeros(dims[3])
    _load().oracle_pion_contract(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(prop), int(src_t),
                                 _dp(out))
    return out


def meson_contract(dims, prop, src_t, gammas) -> np.ndarray:
    """C_G(t) for each 4x4 spin matrix G in gammas[ng, 4, 4] from 12 propagator
    columns prop[j, t, z, y, x, spin, colour]; complex array [ng, T]."""
    prop, d = _c128(prop), _dims(dims)
    g = _c128(np.asarray(gammas, dtype=np.complex128).reshape(-1, 4, 4))
    out = np.zeros(2 * g.shape[0] * dims[3])
    _load().oracle_meson_contract(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(prop), int(src_t), _dp(g),
                                  int(g.shape[0]), _dp(out))
    return out.view(np.complex128).reshape(g.shape[0], dims[3])


def pion(dims, U, kappa, csw, src, theta=DEFAULT_THETA, tol=1e-13, maxiter=100000, want_prop=False):
    """Point-source propagator (12 columns) and pion C(t).

    Returns (corr, prop or None, iterations[12], residuals[12], failed_columns).
    """
    lx, ly, lz, lt = dims
    U, th, d = _c128(U), _theta(theta), _dims(dims)
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    corr = np.zeros(lt)
    prop = np.zeros((12, lt, lz, ly, lx, 4, 3), dtype=np.complex128) if want_prop else None
    iters = np.zeros(12, dtype=np.int32)
    res = np.zeros(12)
    failed = _load().oracle_pion(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(U), kappa, csw, _dp(th),
                                 s.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), tol, maxiter, _dp(corr),
                                 _dp(prop) if prop is not None else None,
                                 iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(res))
    return corr, prop, iters, res, failed
