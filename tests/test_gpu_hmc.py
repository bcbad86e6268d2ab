"""GPU quenched HMC trajectory (Sec. 3.1, HMC! with leapfrog) against the oracle.

The oracle's trajectory is pinned in test_oracle_pins.py (the force is minus
the Lie derivative of the action, second-order energy violation, gauge
covariance, Metropolis).  Same momenta and uniform number on both sides:
the decision must agree, dH within 1e-9 and the links within 1e-11; a
rejected trajectory restores the links exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_16994_gb300 import lqcd
    return lqcd


def _moms(dims, seed):
    return inputs.normals(seed, 0, 32 * int(np.prod(dims))).reshape(tuple(dims[::-1]) + (4, 8))


@pytest.mark.parametrize("eps,nsteps", [(0.05, 10), (0.1, 3)])
def test_hmc_trajectory_matches_oracle(lq, eps, nsteps):
    dims, beta = (4, 4, 2, 6), 5.8
    U = inputs.gauge_field(dims, 0.4, seed=91)
    mom = _moms(dims, 92)
    u = 0.3
    acc_o, dH_o, U_o = oracle.hmc(dims, U, beta, eps, nsteps, mom, u)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        acc, dH = lq.hmc_trajectory(lat, gid, beta, eps, nsteps, mom, u)
        Ug = lq.gauge_download(lat, gid, dims)
    finally:
        lq.lattice_destroy(lat)
    assert abs(dH - dH_o) <= 1e-9, (dH, dH_o)
    assert acc == acc_o
    assert np.max(np.abs(Ug - U_o)) <= 1e-11


@pytest.mark.parametrize("u", [0.5, 0.05])
def test_metropolis_decision_and_restore(lq, u):
    # dH = 2.46 on this field: u = 0.5 > exp(-dH) rejects, u = 0.05 accepts
    dims, beta, eps, nsteps = (4, 4, 2, 4), 6.0, 0.1, 2
    U = inputs.gauge_field(dims, 0.3, seed=93)
    mom = _moms(dims, 94)
    acc_o, dH_o, U_o = oracle.hmc(dims, U, beta, eps, nsteps, mom, u)
    assert 1.0 < dH_o < 5.0
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        acc, dH = lq.hmc_trajectory(lat, gid, beta, eps, nsteps, mom, u)
        Ug = lq.gauge_download(lat, gid, dims)
    finally:
        lq.lattice_destroy(lat)
    assert abs(dH - dH_o) <= 1e-9 * max(1.0, abs(dH_o))
    assert acc == acc_o == (u < np.exp(-dH_o))
    if acc:
        assert np.max(np.abs(Ug - U_o)) <= 1e-11
    else:
        assert np.array_equal(Ug, U)
