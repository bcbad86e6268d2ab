"""GPU Wilson flow and gauge observables (Sec. 3.2) against the FP64 oracle.

The oracle's flow (RK3 in Luescher's normalisation) and observables are
pinned in test_oracle_pins.py (weak abelian wave, third-order convergence,
covariance, closed forms on constant abelian fluxes).  Gates: flowed links
within 1e-12, observables within 1e-12 relative, and a propagator solved on
the flowed field (FP16 and FP64) matching the oracle's on the oracle-flowed
field within 1e-8 (the flow rebuilds the reduced-precision links and drops
the clover fields of the old links).
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


def test_flow_and_observables_match_oracle(lq):
    dims = (4, 6, 4, 6)
    U = inputs.gauge_field(dims, 0.35, seed=71)
    eps, n = 0.02, 8
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        assert np.max(np.abs(lq.gauge_download(lat, gid, dims) - U)) == 0.0
        obs0 = lq.gauge_observables(lat, gid, dims[3])
        lq.gauge_flow(lat, gid, eps, n)
        Uf = lq.gauge_download(lat, gid, dims)
        obs1 = lq.gauge_observables(lat, gid, dims[3])
        with pytest.raises(lq.LqcdError) as e:
            lq.gauge_flow(lat, gid, 0.0, 1)
        assert e.value.code == lq.EINVAL
    finally:
        lq.lattice_destroy(lat)
    Uo = oracle.wilson_flow(dims, U, eps, n)
    assert np.max(np.abs(Uf - Uo)) <= 1e-12
    for got, field in ((obs0, U), (obs1, Uo)):
        want = oracle.gauge_obs(dims, field)
        assert abs(got[0] - want[0]) <= 1e-13
        for k in (1, 2):
            assert np.allclose(got[k], want[k], rtol=1e-12, atol=0)
        assert np.allclose(got[3], want[3], rtol=0, atol=1e-12 * np.max(want[2]))
    assert np.sum(obs1[1]) < np.sum(obs0[1])  # the flow smooths


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_propagator_on_the_flowed_field(lq, prec):
    dims, kappa, csw, src = (4, 4, 4, 6), 0.125, 1.2, (0, 1, 2, 3)
    U = inputs.gauge_field(dims, 0.4, seed=72)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(kappa, csw)
        sp = lq.solver_params(tol=1e-10, maxiter=5000, precision=prec)
        before, _, _, rc0 = lq.pion_corr(lat, gid, dp, sp, src, dims=dims)  # caches the clover of U
        lq.gauge_flow(lat, gid, 0.05, 4)
        corr, prop, info, rc = lq.pion_corr(lat, gid, dp, sp, src, dims=dims, want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc0 == lq.OK and rc == lq.OK, info
    Uo = oracle.wilson_flow(dims, U, 0.05, 4)
    ref, prop_ref, *_ = oracle.pion(dims, Uo, kappa, csw, src, tol=1e-13, want_prop=True)
    assert np.all(np.abs(corr - ref) <= 1e-8 * ref)
    assert np.linalg.norm(prop - prop_ref) <= 1e-8 * np.linalg.norm(prop_ref)
    assert np.max(np.abs(before - ref) / ref) > 1e-4  # the flowed field gives a different propagator
