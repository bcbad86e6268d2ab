"""GPU open boundary conditions in time and boundary-to-bulk f_P / f_A.

Reading (Sec. 2.1 BC_OPEN, Sec. 3.3 cF and the boundary-to-bulk
propagators): the time links leaving the last slice are absent, so hops and
clover leaves across the time boundary vanish; the first and last slices get
2 kappa (cF - 1); f_P and f_A come from the six P+ wall sources on slice 0.
The oracle's operator and correlators are pinned in test_oracle_pins.py (free
field against the momentum-space time matrix, rough-field identities, dense
inverse).  Gates: FP64 D within 1e-13, solves with true residual <= 1e-10 and
error <= 1e-8, f_P and f_A within 1e-8 (f_A on the scale of f_P).
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
@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_open_dirac_matches_oracle(lq, dagger, mu):
    U = inputs.gauge_field(DIMS, EPS, seed=51)
    psi = inputs.spinor_field(DIMS, seed=52)
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        got = lq.dirac_apply(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, mu=mu, cF=CF, bc="open"), psi,
                             dagger=dagger)
        per = lq.dirac_apply(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, mu=mu), psi, dagger=dagger)
    finally:
        lq.lattice_destroy(lat)
    if mu == 0.0:
        want = oracle.dirac_open(DIMS, U, KAPPA, CSW, CF, psi, theta=THETA, dagger=dagger)
        assert rel(got, want) <= 1e-13
    else:  # the twist adds 2 i kappa mu g5 (its adjoint -) to the open operator as to the periodic one
        sg = (-1 if dagger else 1) * 2j * KAPPA * mu * np.array([1, 1, -1, -1])[:, None]
        want = oracle.dirac_open(DIMS, U, KAPPA, CSW, CF, psi, theta=THETA, dagger=dagger) + sg * psi
        assert rel(got, want) <= 1e-13
    assert rel(per, got) > 1e-3  # the boundary does change the operator


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_open_solve_matches_oracle(lq, prec):
    U = inputs.gauge_field(DIMS, EPS, seed=53)
    b = inputs.spinor_field(DIMS, seed=54, nrhs=2)
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(KAPPA, CSW, THETA, cF=CF, bc="open"),
                                  lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), b, nrhs=2)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    for j in range(2):
        r = b[j] - oracle.dirac_open(DIMS, U, KAPPA, CSW, CF, x[j], theta=THETA)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[j])
        xo, it, res, ok = oracle.cgnr_open(DIMS, U, KAPPA, CSW, CF, b[j], theta=THETA, tol=1e-13)
        assert ok
        assert rel(x[j], xo) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_boundary_to_bulk_correlators_match_oracle(lq, prec):
    dims = (4, 4, 4, 10)
    U = inputs.gauge_field(dims, 0.3, seed=55)
    fPo, fAo, Ho, iters, res, failed = oracle.boundary_corr(dims, U, 0.125, 1.3, 1.1, tol=1e-13, want_prop=True)
    assert failed == 0
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        fP, fA, H, info, rc = lq.boundary_corr(lat, gid, lq.dirac_params(0.125, 1.3, cF=1.1, bc="open"),
                                               lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), dims,
                                               want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert all(i["true_resid"] <= 1e-10 for i in info)
    assert np.all(np.abs(fP - fPo) <= 1e-8 * fPo)
    assert np.all(np.abs(fA - fAo) <= 1e-8 * fPo)
    for j in range(6):
        assert rel(H[j], Ho[j]) <= 1e-8
