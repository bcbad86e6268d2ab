"""GPU twisted mass (DiracParam's mu, Sec. 3.3) against the FP64 oracle.

Reading: in the kappa normalisation the site term gains 2 i kappa mu g5
(the paper's D_w gains i mu g5 and D = 2 kappa D_w); D(mu)^dag = g5 D(-mu) g5.
The oracle's D(mu) and CGNR on it are pinned by the free-field closed forms
and identities in test_oracle_pins.py.  Gates as for mu = 0: FP64 D within
1e-13 relative L2, solves with true residual <= 1e-10 (by the oracle's
D(mu)) and error <= 1e-8 against the oracle's 1e-13 solution, C(t) within
1e-8 per slice.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS, KAPPA, CSW, EPS = (6, 4, 4, 8), 0.13, 1.5, 0.4
THETA = (np.exp(0.3j), 1, np.exp(-0.7j), -1)


@pytest.fixture(scope="module")
def lq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_16994_gb300 import lqcd
    return lqcd


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def parity_mask(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2 == 0)[..., None, None]


@pytest.mark.parametrize("mu", [0.05, -0.2])
@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_tm_matches_oracle(lq, mu, dagger):
    U = inputs.gauge_field(DIMS, EPS, seed=31)
    psi = inputs.spinor_field(DIMS, seed=32)
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        got = lq.dirac_apply(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, mu=mu), psi, dagger=dagger)
    finally:
        lq.lattice_destroy(lat)
    want = oracle.dirac_tm(DIMS, U, KAPPA, CSW, mu, psi, theta=THETA, dagger=dagger)
    assert rel(got, want) <= 1e-13


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 4e-3)])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_tm_low_precision_against_fp64(lq, prec, tol, dagger):
    """The even-odd operator with mu in FP32/FP16 storage against FP64 (the
    FP64 one is checked through the solves below)."""
    U = inputs.gauge_field(DIMS, EPS, seed=33)
    x = inputs.spinor_field(DIMS, seed=34, nrhs=3) * parity_mask(DIMS)
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(KAPPA, CSW, THETA, mu=0.1)
        ref = lq.schur_apply(lat, gid, dp, x, precision="fp64", nrhs=3, dagger=dagger)
        got = lq.schur_apply(lat, gid, dp, x, precision=prec, nrhs=3, dagger=dagger)
        plain = lq.schur_apply(lat, gid, lq.dirac_params(KAPPA, CSW, THETA), x, precision="fp64", nrhs=3,
                               dagger=dagger)
    finally:
        lq.lattice_destroy(lat)
    for j in range(3):
        assert rel(got[j], ref[j]) <= tol
        assert rel(plain[j], ref[j]) > 1e-3  # the twist does change the operator


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_solve_tm_matches_oracle(lq, prec):
    mu = 0.04
    U = inputs.gauge_field(DIMS, EPS, seed=35)
    b = inputs.spinor_field(DIMS, seed=36, nrhs=2)
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, mu=mu),
                                  lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), b, nrhs=2)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    for j in range(2):
        assert info[j]["true_resid"] <= 1e-10
        r = b[j] - oracle.dirac_tm(DIMS, U, KAPPA, CSW, mu, x[j], theta=THETA)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[j])
        xo, it, res, ok = oracle.cgnr_tm(DIMS, U, KAPPA, CSW, mu, b[j], theta=THETA, tol=1e-13)
        assert ok
        assert rel(x[j], xo) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_pion_tm_against_oracle_propagator(lq, prec):
    """C(t) at mu != 0 against the oracle's contraction of the oracle's
    12 twisted-mass columns."""
    dims, kappa, csw, mu, src = (4, 4, 4, 8), 0.125, 1.2, 0.03, (1, 2, 3, 5)
    U = inputs.gauge_field(dims, 0.3, seed=37)
    cols = []
    for j in range(12):
        eta = inputs.point_source(dims, src, j // 3, j % 3)
        xo, it, res, ok = oracle.cgnr_tm(dims, U, kappa, csw, mu, eta, tol=1e-13)
        assert ok
        cols.append(xo)
    ref = oracle.pion_contract(dims, np.stack(cols), src[3])
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr, prop, info, rc = lq.pion_corr(lat, gid, lq.dirac_params(kappa, csw, mu=mu),
                                            lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), src,
                                            dims=dims, want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert np.all(np.abs(corr - ref) <= 1e-8 * ref)
    for j in range(12):
        assert rel(prop[j], cols[j]) <= 1e-8


def test_served_twisted_request_equals_alone(lq):
    """A request with mu != 0 through the serving loop gives the C(t) of the
    same request solved alone (and admission charges its extra inverse)."""
    dims, kappa, csw, src = (4, 4, 4, 8), 0.125, 1.2, (0, 1, 2, 3)
    U = inputs.gauge_field(dims, 0.3, seed=38)
    sp = lq.solver_params(tol=1e-10, maxiter=5000, precision="fp16")
    srv = lq.serve_create(device=0, hbm_budget_bytes=0, max_slots=2)
    try:
        g = lq.serve_gauge(srv, dims, U)
        tickets = [lq.serve_submit(srv, g, lq.dirac_params(kappa, csw, mu=mu), sp, src) for mu in (0.03, 0.0)]
        served = [lq.serve_poll(srv, t, dims[3], timeout_ms=-1) for t in tickets]
    finally:
        lq.serve_destroy(srv)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        for (rc, corr, infos, ts), mu in zip(served, (0.03, 0.0)):
            assert rc == lq.OK, infos
            alone, _, _, rc2 = lq.pion_corr(lat, gid, lq.dirac_params(kappa, csw, mu=mu), sp, src, dims=dims)
            assert rc2 == lq.OK
            assert np.all(np.abs(corr - alone) <= 1e-8 * alone)
        assert np.max(np.abs(served[0][1] - served[1][1]) / served[1][1]) > 1e-4  # mu matters
    finally:
        lq.lattice_destroy(lat)
