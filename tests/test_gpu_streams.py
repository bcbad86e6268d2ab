"""Small solves on a caller's stream.

Below 2^20 site-RHS the solver replays graph-captured chunks of iterations:
on the legacy default stream it runs them on a stream of its own, on a
caller's stream it captures that stream directly.  Both must give the same
bits, and the call must be ordered on the caller's stream (the result is
ready after a synchronize of that stream alone).
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


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_user_stream_equals_default_stream(lq, prec):
    import torch
    dims, kappa, csw = (6, 4, 4, 8), 0.13, 1.5
    U = inputs.gauge_field(dims, 0.4, seed=111)
    b = inputs.spinor_field(dims, seed=112, nrhs=3)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(kappa, csw)
        sp = lq.solver_params(tol=1e-10, maxiter=5000, precision=prec)
        bt = torch.from_numpy(b).cuda()
        x0, info0, rc0 = lq.cg_solve(lat, gid, dp, sp, bt, nrhs=3)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            bs = bt.clone()
            xs = torch.empty_like(bs)
        s.synchronize()
        x1, info1, rc1 = lq.cg_solve(lat, gid, dp, sp, bs, nrhs=3, x=xs, stream=s)
        s.synchronize()
        got = xs.cpu().numpy()
    finally:
        lq.lattice_destroy(lat)
    assert rc0 == lq.OK and rc1 == lq.OK, (info0, info1)
    assert np.array_equal(got, x0.cpu().numpy())
    r = b[1] - oracle.dirac(dims, U, kappa, csw, got[1])
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[1])
