"""GPU: lqcd_cg_solve started from an initial guess (LQCD_GUESS).

The solve of Sec. 3.3 (CG!) works on a given field; a caller resumes a solve
from a saved x_0 or warm-starts it from a nearby solution.  Gates as in the
other solver tests: true relative residual <= 1e-10 by the FP64 oracle's own
D, solution error <= 1e-8 against the oracle's 1e-13 solution; and a good
guess must cost fewer inner iterations than the zero start.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS, KAPPA, CSW, EPS = (6, 4, 4, 8), 0.13, 1.5, 0.4
THETA = (1, np.exp(0.4j), 1, -1)


@pytest.fixture(scope="module")
def lq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_16994_gb300 import lqcd
    return lqcd


@pytest.fixture(scope="module")
def problem():
    U = inputs.gauge_field(DIMS, EPS, seed=2)
    b = inputs.spinor_field(DIMS, seed=3, nrhs=2)
    xo = np.stack([oracle.cgnr(DIMS, U, KAPPA, CSW, b[j], theta=THETA, tol=1e-13)[0] for j in range(2)])
    return U, b, xo


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def true_resid(U, x, b):
    return np.linalg.norm(b - oracle.dirac(DIMS, U, KAPPA, CSW, x, theta=THETA)) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("device_ptrs", [False, True])
def test_perturbed_oracle_solution_as_guess(lq, problem, prec, device_ptrs):
    """x_0 = oracle solution + a seeded perturbation of relative size 1e-4:
    converges to the gates in fewer inner iterations than the zero start."""
    import torch
    U, b, xo = problem
    noise = inputs.spinor_field(DIMS, seed=7, nrhs=2)
    x0 = xo + 1e-4 * noise * (np.linalg.norm(xo) / np.linalg.norm(noise))
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(KAPPA, CSW, THETA)
        sp = lq.solver_params(tol=1e-10, maxiter=5000, precision=prec)
        _, info0, rc0 = lq.cg_solve(lat, gid, dp, sp, b, nrhs=2)
        assert rc0 == lq.OK, info0
        if device_ptrs:
            xg = torch.from_numpy(x0.copy()).cuda()
            x, info, rc = lq.cg_solve(lat, gid, dp, sp, torch.from_numpy(b).cuda(), nrhs=2, x=xg, guess=True)
            x = x.cpu().numpy()
        else:
            x, info, rc = lq.cg_solve(lat, gid, dp, sp, b, nrhs=2, x=x0.copy(), guess=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    for j in range(2):
        assert info[j]["true_resid"] <= 1e-10
        assert true_resid(U, x[j], b[j]) <= 1e-10
        assert rel(x[j], xo[j]) <= 1e-8
        assert info[j]["iters_inner"] < info0[j]["iters_inner"], (info[j], info0[j])


def test_exact_guess_returns_without_iterating(lq, problem):
    """A guess that already meets tol is accepted by the first FP64 residual."""
    U, b, xo = problem
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(KAPPA, CSW, THETA),
                                  lq.solver_params(tol=1e-10, maxiter=5000, precision="fp16"), b, nrhs=2,
                                  x=xo.copy(), guess=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    for j in range(2):
        assert info[j]["iters_inner"] == 0, info[j]
        assert true_resid(U, x[j], b[j]) <= 1e-10
        assert rel(x[j], xo[j]) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_resume_after_iteration_cap(lq, problem, prec):
    """A solve stopped by maxiter (LQCD_ENOCONV, x filled) resumes from its
    own x and reaches the gates; without LQCD_GUESS the same call would
    start over from zero."""
    U, b, xo = problem
    lat = lq.lattice_create(DIMS)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(KAPPA, CSW, THETA)
        _, info_full, rc = lq.cg_solve(lat, gid, dp, lq.solver_params(tol=1e-10, maxiter=5000, precision=prec),
                                       b, nrhs=2)
        assert rc == lq.OK
        cap = max(info_full[0]["iters_inner"] // 3, 1)
        x1, info1, rc1 = lq.cg_solve(lat, gid, dp, lq.solver_params(tol=1e-10, maxiter=cap, precision=prec),
                                     b, nrhs=2)
        assert rc1 == lq.ENOCONV, info1
        assert all(i["true_resid"] > 1e-10 for i in info1)
        x2, info2, rc2 = lq.cg_solve(lat, gid, dp, lq.solver_params(tol=1e-10, maxiter=5000, precision=prec),
                                     b, nrhs=2, x=x1.copy(), guess=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc2 == lq.OK, info2
    for j in range(2):
        assert true_resid(U, x2[j], b[j]) <= 1e-10
        assert rel(x2[j], xo[j]) <= 1e-8
        assert info2[j]["iters_inner"] < info_full[j]["iters_inner"], (info2[j], info_full[j])
