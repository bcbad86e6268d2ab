"""Python binding of the C ABI in include/lqcd.h (ctypes; marshalling only).

The names follow the C calls without the ``lqcd_`` prefix.  Every step of
the computation runs in liblqcd.so; there is no Python or CPU fallback: if
the library is not built, importing works but every call raises
``LqcdError`` with the build instructions.

Fields are numpy ``complex128`` arrays in the host layout of lqcd.h
(``U[t,z,y,x,mu,3,3]``, ``psi[..., t,z,y,x,spin,colour]``) or CUDA tensors
(PyTorch, complex128 or float64 with the same number of reals), which are
passed as device pointers together with the tensor's current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBUSY, ETIMEOUT, ENOTFOUND, ENOTIMPL = 0, -1, -2, -3, -4, -5, -6, -7, -8
PREC_FP64, PREC_MIXED_FP32, PREC_MIXED_FP16 = 0, 1, 2
DAG, DEVICE_PTRS, GUESS = 1, 2, 4
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_MIXED_FP32, "fp16": PREC_MIXED_FP16}
STATUS_NAMES = {0: "LQCD_OK", -1: "LQCD_EINVAL", -2: "LQCD_ENOMEM", -3: "LQCD_ECUDA", -4: "LQCD_ENOCONV",
                -5: "LQCD_EBUSY", -6: "LQCD_ETIMEOUT", -7: "LQCD_ENOTFOUND", -8: "LQCD_ENOTIMPL"}
DEFAULT_THETA = (1.0, 1.0, 1.0, -1.0)


class LqcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class DiracParams(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("csw", ctypes.c_double), ("theta_re", ctypes.c_double * 4),
                ("theta_im", ctypes.c_double * 4), ("mu", ctypes.c_double), ("cF", ctypes.c_double),
                ("bc", ctypes.c_int)]


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("nrhs", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong), ("bytes", ctypes.c_double),
                ("timed_launches", ctypes.c_longlong), ("timed_ms", ctypes.c_double), ("timed_bytes", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters_inner", ctypes.c_int), ("iters_outer", ctypes.c_int), ("true_resid", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {"iters_inner": self.iters_inner, "iters_outer": self.iters_outer,
                "true_resid": self.true_resid, "status": self.status}


class PionJob(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_void_p), ("gauge_id", ctypes.c_int), ("dp", DiracParams), ("src", ctypes.c_int * 4),
                ("corr", ctypes.POINTER(ctypes.c_double)), ("info", SolveInfo * 12), ("status", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Loads liblqcd.so (raises LqcdError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise LqcdError(ECUDA, f"{_build.LIB} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_build.LIB)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.lqcd_last_error.restype = ctypes.c_char_p
    sig = {
        "lqcd_abi_version": [],
        "lqcd_lattice_create": [ip, ctypes.c_int, ctypes.POINTER(vp)],
        "lqcd_lattice_destroy": [vp],
        "lqcd_gauge_upload": [vp, vp, ip],
        "lqcd_gauge_free": [vp, ctypes.c_int],
        "lqcd_dirac_apply": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), vp, vp, ctypes.c_int, vp],
        "lqcd_schur_apply": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), ctypes.c_int, vp, vp, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, vp],
        "lqcd_cg_solve": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), ctypes.POINTER(SolverParams), vp, vp,
                          ctypes.c_int, ctypes.POINTER(SolveInfo), ctypes.c_int, vp],
        "lqcd_pion_corr": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), ctypes.POINTER(SolverParams), ip, vp, vp,
                           ctypes.POINTER(SolveInfo), ctypes.c_int, vp],
        "lqcd_pion_contract": [vp, vp, ctypes.c_int, vp, ctypes.c_int, vp],
        "lqcd_meson_contract": [vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp],
        "lqcd_pion_corr_batch": [ctypes.POINTER(PionJob), ctypes.c_int, ctypes.POINTER(SolverParams), ctypes.c_int, vp],
        "lqcd_pion_contract_noalloc": [ip, vp, ctypes.c_int, vp, vp],
        "lqcd_gauge_flow": [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp],
        "lqcd_fermion_flow": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), vp, ctypes.c_int, ctypes.c_double,
                              ctypes.c_int, ctypes.c_int, vp],
        "lqcd_fermion_backflow": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), vp, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, vp],
        "lqcd_gauge_observables": [vp, ctypes.c_int, dp, dp, dp, dp, vp],
        "lqcd_gauge_download": [vp, ctypes.c_int, vp, ctypes.c_int, vp],
        "lqcd_hmc_trajectory": [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp,
                                ctypes.c_double, dp, ip, vp],
        "lqcd_boundary_corr": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), ctypes.POINTER(SolverParams), vp, vp,
                               vp, ctypes.POINTER(SolveInfo), ctypes.c_int, vp],
        "lqcd_serve_create": [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)],
        "lqcd_serve_gauge": [vp, ip, vp, ip],
        "lqcd_serve_submit": [vp, ctypes.c_int, ctypes.POINTER(DiracParams), ctypes.POINTER(SolverParams), ip,
                              ctypes.POINTER(ctypes.c_uint64)],
        "lqcd_serve_poll": [vp, ctypes.c_uint64, dp, ctypes.POINTER(SolveInfo), dp, ctypes.c_int],
        "lqcd_serve_destroy": [vp],
        "lqcd_profile_reset": [ctypes.c_int],
        "lqcd_tune_report": [ctypes.c_char_p, ctypes.c_size_t],
        "lqcd_tune_export": [ctypes.c_char_p, ctypes.c_size_t],
        "lqcd_tune_import": [ctypes.c_char_p],
        "lqcd_profile_read": [ctypes.POINTER(KernelStat), ctypes.c_int, ip],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().lqcd_last_error().decode()


def _check(rc, allow=(OK,)):
    if rc not in allow:
        raise LqcdError(rc, last_error())
    return rc


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _host(a, dtype=np.complex128):
    if _is_cuda_tensor(a):
        raise TypeError("mixing device and host buffers in one call is not supported")
    return np.ascontiguousarray(a, dtype=dtype)


def _dev_ptr(t, nreal):
    """Device pointer of a contiguous CUDA tensor holding `nreal` doubles."""
    if not t.is_contiguous():
        raise ValueError("device tensors must be contiguous")
    if t.is_complex():
        n = t.numel() * 2
        ok = str(t.dtype) == "torch.complex128"
    else:
        n = t.numel()
        ok = str(t.dtype) == "torch.float64"
    if not ok:
        raise TypeError("device tensors must be complex128 or float64")
    if n != nreal:
        raise ValueError(f"device tensor has {n} reals, expected {nreal}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_of(t, stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch  # only reached for device tensors
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


BCS = {"periodic": 0, "open": 1, "sf": 2}


def dirac_params(kappa, csw, theta=DEFAULT_THETA, mu=0.0, cF=1.0, bc="periodic") -> DiracParams:
    """DiracParam (kappa instead of m0): theta phase factors, twisted mass mu, boundary
    coefficient cF and the time boundary ("periodic", "open" or "sf")."""
    th = np.asarray(theta, dtype=np.complex128)
    p = DiracParams()
    p.kappa, p.csw, p.mu, p.cF = float(kappa), float(csw), float(mu), float(cF)
    p.bc = BCS[bc] if isinstance(bc, str) else int(bc)
    for k in range(4):
        p.theta_re[k] = th[k].real
        p.theta_im[k] = th[k].imag
    return p


def solver_params(tol=1e-10, maxiter=10000, precision="fp64", inner_tol=0.0, nrhs=1) -> SolverParams:
    s = SolverParams()
    s.tol, s.maxiter, s.inner_tol, s.nrhs = float(tol), int(maxiter), float(inner_tol), int(nrhs)
    s.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return s


# ---------------------------------------------------------------------------
# the ABI
# ---------------------------------------------------------------------------

def abi_version() -> int:
    return load().lqcd_abi_version()


def lattice_create(dims, device=0):
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    h = ctypes.c_void_p()
    _check(load().lqcd_lattice_create(d, int(device), ctypes.byref(h)))
    return h


def lattice_destroy(lat):
    _check(load().lqcd_lattice_destroy(lat))


def gauge_upload(lat, U) -> int:
    u = _host(U)
    gid = ctypes.c_int(-1)
    _check(load().lqcd_gauge_upload(lat, u.ctypes.data_as(ctypes.c_void_p), ctypes.byref(gid)))
    return gid.value


def gauge_free(lat, gauge_id):
    _check(load().lqcd_gauge_free(lat, int(gauge_id)))


def dirac_apply(lat, gauge_id, params: DiracParams, psi, out=None, dagger=False, stream=None):
    """out = D psi (or D^dag psi); numpy in -> numpy out, CUDA tensor in -> tensor out."""
    flags = DAG if dagger else 0
    if _is_cuda_tensor(psi):
        if out is None:
            out = psi.new_empty(psi.shape)
        n = psi.numel() * (2 if psi.is_complex() else 1)
        rc = load().lqcd_dirac_apply(lat, int(gauge_id), ctypes.byref(params), _dev_ptr(psi, n), _dev_ptr(out, n),
                                     flags | DEVICE_PTRS, _stream_of(psi, stream))
        _check(rc)
        return out
    p = _host(psi)
    o = np.empty_like(p) if out is None else out
    rc = load().lqcd_dirac_apply(lat, int(gauge_id), ctypes.byref(params), p.ctypes.data_as(ctypes.c_void_p),
                                 o.ctypes.data_as(ctypes.c_void_p), flags, None)
    _check(rc)
    return o


def schur_apply(lat, gauge_id, params: DiracParams, psi, precision="fp64", nrhs=1, repeat=1, dagger=False,
                out=None, stream=None):
    """Even-odd preconditioned operator Dhat (or Dhat^dag) on the even sites of psi, in `precision`."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    flags = DAG if dagger else 0
    if _is_cuda_tensor(psi):
        out = psi.new_empty(psi.shape) if out is None else out
        n = psi.numel() * (2 if psi.is_complex() else 1)
        _check(load().lqcd_schur_apply(lat, int(gauge_id), ctypes.byref(params), prec, _dev_ptr(psi, n),
                                       _dev_ptr(out, n), int(nrhs), int(repeat), flags | DEVICE_PTRS,
                                       _stream_of(psi, stream)))
        return out
    p = _host(psi)
    o = np.empty_like(p) if out is None else out
    _check(load().lqcd_schur_apply(lat, int(gauge_id), ctypes.byref(params), prec, p.ctypes.data_as(ctypes.c_void_p),
                                   o.ctypes.data_as(ctypes.c_void_p), int(nrhs), int(repeat), flags, None))
    return o


def cg_solve(lat, gauge_id, params: DiracParams, solver: SolverParams, b, nrhs=1, x=None, stream=None,
             guess=False):
    """Solves D x_j = b_j.  Returns (x, [info dicts], status).

    ``guess=True``: ``x`` (required then) holds the initial guess and receives
    the solution (``LQCD_GUESS``); otherwise the solve starts from zero."""
    info = (SolveInfo * nrhs)()
    if guess and x is None:
        raise ValueError("guess=True needs x (the initial guess)")
    flags = GUESS if guess else 0
    if _is_cuda_tensor(b):
        if x is None:
            x = b.new_empty(b.shape)
        n = b.numel() * (2 if b.is_complex() else 1)
        rc = load().lqcd_cg_solve(lat, int(gauge_id), ctypes.byref(params), ctypes.byref(solver), _dev_ptr(b, n),
                                  _dev_ptr(x, n), int(nrhs), info, DEVICE_PTRS | flags, _stream_of(b, stream))
    else:
        bb = _host(b)
        if x is None:
            x = np.empty_like(bb)
        elif not (isinstance(x, np.ndarray) and x.dtype == bb.dtype and x.shape == bb.shape
                  and x.flags.c_contiguous):
            raise ValueError("x must be a C-contiguous array of b's dtype and shape")
        rc = load().lqcd_cg_solve(lat, int(gauge_id), ctypes.byref(params), ctypes.byref(solver),
                                  bb.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p), int(nrhs),
                                  info, flags, None)
    _check(rc, allow=(OK, ENOCONV))
    return x, [i.as_dict() for i in info], rc


def pion_corr(lat, gauge_id, params: DiracParams, solver: SolverParams, src, dims=None, want_prop=False,
              device_out=None, stream=None):
    """12-column point-source propagator + pion C(t).

    Host mode (default): returns (corr ndarray, prop ndarray or None, infos, status); ``dims`` is needed
    for the output shapes.  Device mode: ``device_out = (corr_tensor, prop_tensor_or_None)``.
    """
    s = (ctypes.c_int * 4)(*[int(v) for v in src])
    info = (SolveInfo * 12)()
    if device_out is not None:
        corr_t, prop_t = device_out
        rc = load().lqcd_pion_corr(lat, int(gauge_id), ctypes.byref(params), ctypes.byref(solver), s,
                                   ctypes.c_void_p(corr_t.data_ptr()),
                                   ctypes.c_void_p(prop_t.data_ptr()) if prop_t is not None else None, info,
                                   DEVICE_PTRS, _stream_of(corr_t, stream))
        _check(rc, allow=(OK, ENOCONV))
        return corr_t, prop_t, [i.as_dict() for i in info], rc
    lx, ly, lz, lt = dims
    corr = np.zeros(lt)
    prop = np.zeros((12, lt, lz, ly, lx, 4, 3), dtype=np.complex128) if want_prop else None
    rc = load().lqcd_pion_corr(lat, int(gauge_id), ctypes.byref(params), ctypes.byref(solver), s,
                               corr.ctypes.data_as(ctypes.c_void_p),
                               prop.ctypes.data_as(ctypes.c_void_p) if prop is not None else None, info, 0, None)
    _check(rc, allow=(OK, ENOCONV))
    return corr, prop, [i.as_dict() for i in info], rc


def gauge_flow(lat, gauge_id, eps, nsteps, stream=None):
    """Wilson flow (RK3) of the resident field, in place: t = nsteps * eps."""
    _check(load().lqcd_gauge_flow(lat, int(gauge_id), float(eps), int(nsteps), stream))


def fermion_flow(lat, gauge_id, params: DiracParams, psi, eps, nsteps, nrhs=1, stream=None):
    """Flows the resident links (as gauge_flow) and nrhs quark fields alongside
    (lqcd_fermion_flow).  A CUDA tensor is flowed in place and returned; a
    host array is copied, and the flowed copy is returned."""
    if _is_cuda_tensor(psi):
        n = psi.numel() * (2 if psi.is_complex() else 1)
        _check(load().lqcd_fermion_flow(lat, int(gauge_id), ctypes.byref(params), _dev_ptr(psi, n), int(nrhs),
                                        float(eps), int(nsteps), DEVICE_PTRS, _stream_of(psi, stream)))
        return psi
    p = np.array(_host(psi), copy=True)
    if p.size != nrhs * 12 * int(np.prod(p.shape[-6:-2])):
        raise ValueError("psi must hold nrhs full-lattice quark fields")
    _check(load().lqcd_fermion_flow(lat, int(gauge_id), ctypes.byref(params), p.ctypes.data_as(ctypes.c_void_p),
                                    int(nrhs), float(eps), int(nsteps), 0, None))
    return p


def fermion_backflow(lat, gauge_id, params: DiracParams, eta, eps, nsteps, nrhs=1, nsave=4, stream=None):
    """Adjoint flow of nrhs quark fields from t = nsteps eps to 0 (lqcd_fermion_backflow); the
    resident links stay at t = 0.  A CUDA tensor is changed in place; a host array is copied."""
    if _is_cuda_tensor(eta):
        n = eta.numel() * (2 if eta.is_complex() else 1)
        _check(load().lqcd_fermion_backflow(lat, int(gauge_id), ctypes.byref(params), _dev_ptr(eta, n), int(nrhs),
                                            float(eps), int(nsteps), int(nsave), DEVICE_PTRS, _stream_of(eta, stream)))
        return eta
    p = np.array(_host(eta), copy=True)
    if p.size != nrhs * 12 * int(np.prod(p.shape[-6:-2])):
        raise ValueError("eta must hold nrhs full-lattice quark fields")
    _check(load().lqcd_fermion_backflow(lat, int(gauge_id), ctypes.byref(params), p.ctypes.data_as(ctypes.c_void_p),
                                        int(nrhs), float(eps), int(nsteps), int(nsave), 0, None))
    return p


def gauge_observables(lat, gauge_id, T):
    """(plaquette average, Eplaq[T], Eclov[T], Q[T]) per-slice sums."""
    plaq = ctypes.c_double(0)
    Ep, Ec, Q = np.zeros(T), np.zeros(T), np.zeros(T)
    dpp = ctypes.POINTER(ctypes.c_double)
    _check(load().lqcd_gauge_observables(lat, int(gauge_id), ctypes.byref(plaq), Ep.ctypes.data_as(dpp),
                                         Ec.ctypes.data_as(dpp), Q.ctypes.data_as(dpp), None))
    return plaq.value, Ep, Ec, Q


def hmc_trajectory(lat, gauge_id, beta, eps, nsteps, mom, u):
    """One leapfrog HMC trajectory of the resident field; mom [T, Z, Y, X, 4, 8] (coordinates on
    i lambda_a / 2), u uniform in (0, 1).  Returns (accepted, dH)."""
    m = np.ascontiguousarray(mom, dtype=np.float64)
    dH = ctypes.c_double(0)
    acc = ctypes.c_int(0)
    _check(load().lqcd_hmc_trajectory(lat, int(gauge_id), float(beta), float(eps), int(nsteps),
                                      m.ctypes.data_as(ctypes.c_void_p), float(u), ctypes.byref(dH),
                                      ctypes.byref(acc), None))
    return bool(acc.value), dH.value


def gauge_download(lat, gauge_id, dims):
    """The resident FP64 links, host layout U[t, z, y, x, mu, 3, 3]."""
    lx, ly, lz, lt = dims
    U = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    _check(load().lqcd_gauge_download(lat, int(gauge_id), U.ctypes.data_as(ctypes.c_void_p), 0, None))
    return U


def boundary_corr(lat, gauge_id, params: DiracParams, solver: SolverParams, dims, want_prop=False):
    """Boundary-to-bulk f_P, f_A (host arrays) from the six P+ wall sources on slice 0
    (on slice 1, carried in by U_t(0)^dag, for bc="sf").

    Returns (fP, fA, H or None [6, T, Z, Y, X, 4, 3], infos, status)."""
    lx, ly, lz, lt = dims
    fP, fA = np.zeros(lt), np.zeros(lt)
    H = np.zeros((6, lt, lz, ly, lx, 4, 3), dtype=np.complex128) if want_prop else None
    info = (SolveInfo * 6)()
    rc = load().lqcd_boundary_corr(lat, int(gauge_id), ctypes.byref(params), ctypes.byref(solver),
                                   fP.ctypes.data_as(ctypes.c_void_p), fA.ctypes.data_as(ctypes.c_void_p),
                                   H.ctypes.data_as(ctypes.c_void_p) if H is not None else None, info, 0, None)
    _check(rc, allow=(OK, ENOCONV))
    return fP, fA, H, [i.as_dict() for i in info], rc


def pion_corr_batch(jobs, solver: SolverParams, chunk=0):
    """Batched propagators: jobs = [(lat, gauge_id, DiracParams, src, T), ...].

    Returns (list of corr arrays, list of per-job info lists, list of statuses, rc)."""
    arr = (PionJob * len(jobs))()
    corrs = []
    for k, (lat, gid, dp, src, T) in enumerate(jobs):
        c = np.zeros(int(T))
        corrs.append(c)
        arr[k].lat = lat
        arr[k].gauge_id = int(gid)
        arr[k].dp = dp
        for m in range(4):
            arr[k].src[m] = int(src[m])
        arr[k].corr = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = load().lqcd_pion_corr_batch(arr, len(jobs), ctypes.byref(solver), int(chunk), None)
    _check(rc, allow=(OK, ENOCONV))
    return corrs, [[i.as_dict() for i in a.info] for a in arr], [a.status for a in arr], rc


def pion_contract(lat, prop, src_t, T=None, corr=None, stream=None):
    """C(t) from 12 host-layout propagator columns (numpy or CUDA tensor)."""
    if _is_cuda_tensor(prop):
        n = prop.numel() * (2 if prop.is_complex() else 1)
        if corr is None:
            raise ValueError("device mode needs a float64 CUDA tensor `corr` of length T")
        _check(load().lqcd_pion_contract(lat, _dev_ptr(prop, n), int(src_t), ctypes.c_void_p(corr.data_ptr()),
                                         DEVICE_PTRS, _stream_of(prop, stream)))
        return corr
    p = _host(prop)
    T = p.shape[1] if T is None else T
    c = np.zeros(T)
    _check(load().lqcd_pion_contract(lat, p.ctypes.data_as(ctypes.c_void_p), int(src_t),
                                     c.ctypes.data_as(ctypes.c_void_p), 0, None))
    return c


def meson_contract(lat, prop, src_t, gammas, T=None, corr=None, stream=None):
    """C_G(t) for each 4x4 spin matrix G in gammas[ng, 4, 4] from 12 host-layout
    propagator columns (numpy or CUDA tensor); complex [ng, T].  With a CUDA
    `prop`, `corr` must be a complex128 (or float64 [ng, T, 2]) CUDA tensor."""
    g = np.ascontiguousarray(np.asarray(gammas, dtype=np.complex128).reshape(-1, 4, 4))
    gp = g.ctypes.data_as(ctypes.c_void_p)
    if _is_cuda_tensor(prop):
        n = prop.numel() * (2 if prop.is_complex() else 1)
        if corr is None:
            raise ValueError("device mode needs a CUDA tensor `corr` of ng * T complex values")
        _check(load().lqcd_meson_contract(lat, _dev_ptr(prop, n), int(src_t), gp, int(g.shape[0]),
                                          ctypes.c_void_p(corr.data_ptr()), DEVICE_PTRS, _stream_of(prop, stream)))
        return corr
    p = _host(prop)
    T = p.shape[1] if T is None else T
    c = np.zeros((g.shape[0], T), dtype=np.complex128)
    _check(load().lqcd_meson_contract(lat, p.ctypes.data_as(ctypes.c_void_p), int(src_t), gp, int(g.shape[0]),
                                      c.ctypes.data_as(ctypes.c_void_p), 0, None))
    return c


def pion_contract_noalloc(dims, prop, src_t, corr, stream=None):
    """C(t) into the float64 CUDA tensor `corr` from a CUDA tensor `prop`, allocating nothing.

    For callers that cannot allocate device memory (see lqcd.h).  The work is
    queued on the stream; synchronize before reading `corr`.
    """
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    n = prop.numel() * (2 if prop.is_complex() else 1)
    if corr.numel() != int(dims[3]) or str(corr.dtype) != "torch.float64" or not corr.is_cuda:
        raise ValueError("corr must be a float64 CUDA tensor of length T")
    _check(load().lqcd_pion_contract_noalloc(d, _dev_ptr(prop, 12 * 24 * int(np.prod(dims))), int(src_t),
                                             ctypes.c_void_p(corr.data_ptr()), _stream_of(prop, stream)))
    return corr


# ---------------------------------------------------------------------------
# launch accounting
# ---------------------------------------------------------------------------

def profile_reset(timing=False):
    _check(load().lqcd_profile_reset(1 if timing else 0))


def profile_read() -> dict:
    """{kernel name: {launches, bytes, timed_launches, timed_ms, timed_bytes}}."""
    n = ctypes.c_int(0)
    _check(load().lqcd_profile_read(None, 0, ctypes.byref(n)))
    buf = (KernelStat * max(1, n.value))()
    _check(load().lqcd_profile_read(buf, n.value, ctypes.byref(n)))
    return {buf[i].name.decode(): {"launches": buf[i].launches, "bytes": buf[i].bytes,
                                   "timed_launches": buf[i].timed_launches, "timed_ms": buf[i].timed_ms,
                                   "timed_bytes": buf[i].timed_bytes} for i in range(n.value)}


def tune_export() -> str:
    """The autotuner's decisions as text for tune_import (lqcd_tune_export)."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().lqcd_tune_export(buf, len(buf)))
    return buf.value.decode()


def tune_import(text: str) -> None:
    """Loads decisions written by tune_export (lqcd_tune_import)."""
    _check(load().lqcd_tune_import(text.encode()))


def tune_report() -> list:
    """Autotuning decisions taken so far (list of dicts)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().lqcd_tune_report(buf, len(buf)))
    return json.loads(buf.value.decode())


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

def serve_create(device=0, hbm_budget_bytes=0, max_slots=4):
    h = ctypes.c_void_p()
    _check(load().lqcd_serve_create(int(device), int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
    return h


def serve_gauge(srv, dims, U) -> int:
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    u = _host(U)
    gid = ctypes.c_int(-1)
    _check(load().lqcd_serve_gauge(srv, d, u.ctypes.data_as(ctypes.c_void_p), ctypes.byref(gid)))
    return gid.value


def serve_submit(srv, gauge_id, params: DiracParams, solver: SolverParams, src) -> int:
    s = (ctypes.c_int * 4)(*[int(v) for v in src])
    t = ctypes.c_uint64(0)
    _check(load().lqcd_serve_submit(srv, int(gauge_id), ctypes.byref(params), ctypes.byref(solver), s,
                                    ctypes.byref(t)))
    return t.value


def serve_poll(srv, ticket, T, timeout_ms=0):
    """Returns (status, corr, infos, timestamps); status may be EBUSY / ETIMEOUT (then the rest is None)."""
    corr = np.zeros(T)
    info = (SolveInfo * 12)()
    ts = (ctypes.c_double * 4)()
    rc = load().lqcd_serve_poll(srv, ctypes.c_uint64(ticket), corr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                info, ts, int(timeout_ms))
    if rc in (EBUSY, ETIMEOUT):
        return rc, None, None, None
    _check(rc, allow=(OK, ENOCONV))
    return rc, corr, [i.as_dict() for i in info], list(ts)


def serve_destroy(srv):
    _check(load().lqcd_serve_destroy(srv))
