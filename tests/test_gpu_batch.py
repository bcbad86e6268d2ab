"""GPU tests of lqcd_pion_corr_batch: propagators on uneven lattices solved
together in one CUDA graph per chunk of iterations.

Each job's C(t) must equal the same propagator solved alone with
lqcd_pion_corr and the FP64 oracle within 1e-8 relative, every column's true
residual <= 1e-10 (FP64, full lattice), for the mixed precisions.
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


@pytest.mark.parametrize("prec,chunk", [("fp16", 4), ("fp32", 8), ("fp64", 3)])
def test_batch_matches_alone_and_oracle(lq, prec, chunk):
    sizes = {"a": ((4, 4, 4, 4), 0.3, 1), "b": ((6, 6, 6, 8), 0.3, 2), "c": ((8, 4, 6, 6), 0.2, 3)}
    U = {k: inputs.gauge_field(d, e, seed=s) for k, (d, e, s) in sizes.items()}
    lats = {k: lq.lattice_create(sizes[k][0]) for k in sizes}
    try:
        gid = {k: lq.gauge_upload(lats[k], U[k]) for k in sizes}
        plan = [("a", 0.120, 1.0, (0, 0, 0, 0)), ("b", 0.125, 1.5, (1, 2, 3, 5)), ("c", 0.118, 1.3, (3, 1, 2, 4)),
                ("b", 0.129, 1.5, (0, 0, 0, 0)), ("a", 0.110, 1.7, (2, 3, 1, 1)), ("c", 0.121, 0.0, (7, 3, 5, 5))]
        jobs = [(lats[k], gid[k], lq.dirac_params(kap, c), src, sizes[k][0][3]) for k, kap, c, src in plan]
        sp = lq.solver_params(tol=1e-10, maxiter=5000, precision=prec)
        corrs, infos, statuses, rc = lq.pion_corr_batch(jobs, sp, chunk=chunk)
        assert rc == lq.OK and all(s == lq.OK for s in statuses)
        for (k, kap, c, src), corr, info in zip(plan, corrs, infos):
            dims = sizes[k][0]
            assert all(i["true_resid"] <= 1e-10 for i in info)
            ref, *_ = oracle.pion(dims, U[k], kap, c, src, tol=1e-13)
            assert np.all(np.abs(corr - ref) <= 1e-8 * np.abs(ref)), (k, kap)
            alone, _, _, rc2 = lq.pion_corr(lats[k], gid[k], lq.dirac_params(kap, c), sp, src, dims=dims)
            assert rc2 == lq.OK
            assert np.all(np.abs(corr - alone) <= 1e-8 * np.abs(alone))
    finally:
        for l in lats.values():
            lq.lattice_destroy(l)


def test_batch_rejects_bad_jobs(lq):
    dims = (4, 4, 4, 4)
    lat = lq.lattice_create(dims)
    try:
        g = lq.gauge_upload(lat, inputs.gauge_field(dims, 0.2, seed=1))
        with pytest.raises(lq.LqcdError) as e:
            lq.pion_corr_batch([(lat, g, lq.dirac_params(0.12, 1.0), (4, 0, 0, 0), 4)], lq.solver_params())
        assert e.value.code == lq.EINVAL
        with pytest.raises(lq.LqcdError) as e:
            lq.pion_corr_batch([(lat, 7, lq.dirac_params(0.12, 1.0), (0, 0, 0, 0), 4)], lq.solver_params())
        assert e.value.code == lq.EINVAL
    finally:
        lq.lattice_destroy(lat)
