"""GPU Schroedinger-functional boundaries and the SF f_P / f_A.

Reading (Sec. 2.1 BC_SF_*, Sec. 3.3 cF and the SF boundary-to-bulk
propagators): the slice 0 is the boundary at x_t = 0 and x_t = T, the
operator is the identity there and no hop reaches it, the clover term on
1 .. T-1 uses every link, the slices 1 and T-1 get 2 kappa (cF - 1), and f_P,
f_A come from the sources U_t(0, yvec)^dag P+ e_j on the slice 1.  The
oracle's operator and correlators are pinned in test_oracle_pins.py.
Gates: FP64 D within 1e-13, solves with true residual <= 1e-10 and error
<= 1e-8 in every precision, f_P and f_A within 1e-8 (f_A on the scale of
f_P), and the unsupported combinations rejected.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS, KAPPA, CSW, CF, EPS = (6, 4, 4, 8), 0.128, 1.6, 1.25, 0.4
THETA = (np.exp(0.3j), 1, np.exp(-0.7j), 1)


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


@pytest.mark.parametrize("dagger", [False, True])
def test_sf_dirac_matches_oracle(lq, dagger):
    U = inputs.gauge_field(DIMS, EPS, seed=61)
    psi = inputs.spinor_field(DIMS, seed=62)
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        got = lq.dirac_apply(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, cF=CF, bc="sf"), psi, dagger=dagger)
        opn = lq.dirac_apply(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, cF=CF, bc="open"), psi, dagger=dagger)
    finally:
        lq.lattice_destroy(lat)
    want = oracle.dirac_sf(DIMS, U, KAPPA, CSW, CF, psi, theta=THETA, dagger=dagger)
    assert rel(got, want) <= 1e-13
    assert np.array_equal(got[0], psi[0])  # the boundary slice is the identity
    assert rel(opn, got) > 1e-3


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_sf_solve_matches_oracle(lq, prec):
    U = inputs.gauge_field(DIMS, EPS, seed=63)
    b = inputs.spinor_field(DIMS, seed=64, nrhs=2)
    b[:, 0] = 0  # no source on the boundary
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, cF=CF, bc="sf"),
                                  lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), b, nrhs=2)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    for j in range(2):
        r = b[j] - oracle.dirac_sf(DIMS, U, KAPPA, CSW, CF, x[j], theta=THETA)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[j])
        xo, it, res, ok = oracle.cgnr_sf(DIMS, U, KAPPA, CSW, CF, b[j], theta=THETA, tol=1e-13)
        assert ok
        assert rel(x[j], xo) <= 1e-8
        assert np.max(np.abs(x[j][0])) <= 1e-12 * np.max(np.abs(x[j]))


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_sf_boundary_correlators_match_oracle(lq, prec):
    dims = (4, 4, 4, 10)
    U = inputs.gauge_field(dims, 0.3, seed=65)
    fPo, fAo, Ho, iters, res, failed = oracle.boundary_corr_sf(dims, U, 0.125, 1.3, 1.1, tol=1e-13, want_prop=True)
    assert failed == 0
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        fP, fA, H, info, rc = lq.boundary_corr(lat, gid, lq.dirac_params(0.125, 1.3, cF=1.1, bc="sf"),
                                               lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), dims,
                                               want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert fP[0] == 0.0 and fA[0] == 0.0
    assert np.all(np.abs(fP[1:] - fPo[1:]) <= 1e-8 * fPo[1:])
    assert np.all(np.abs(fA - fAo) <= 1e-8 * np.max(fPo))
    for j in range(6):
        assert rel(H[j], Ho[j]) <= 1e-8


def test_sf_rejections(lq):
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.3, seed=66)
    psi = inputs.spinor_field(dims, seed=67)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        with pytest.raises(lq.LqcdError) as e:
            lq.dirac_apply(lat, gid, lq.dirac_params(0.12, 1.0, mu=0.1, bc="sf"), psi)
        assert e.value.code == lq.EINVAL
    finally:
        lq.lattice_destroy(lat)
    srv = lq.serve_create(device=0, hbm_budget_bytes=0, max_slots=1)
    try:
        g = lq.serve_gauge(srv, dims, U)
        with pytest.raises(lq.LqcdError) as e:
            lq.serve_submit(srv, g, lq.dirac_params(0.12, 1.0, bc="sf"), lq.solver_params(precision="fp16"),
                            (0, 0, 0, 1))
        assert e.value.code == lq.EINVAL
    finally:
        lq.serve_destroy(srv)
