"""Incremental residual updates of the mixed solvers against the oracle.

Between FP64 residual recomputations (the anchors) a mixed solver moves the
FP64 residual by the FP32 image of the correction, rhat <- rhat - scale
Dhat e, while |rhat| >= 1e-4 |anchor| and >= 3 tol |b|; the updates that can
finish and the final true residual stay FP64.  Batches of at least 2^20
site-RHS poll every iteration and take these updates.  Gates: true residual
<= 1e-10 by the oracle's D, solution within 1e-8 of the FP64 solver's, both
FP32 and FP16 inner formats, and fewer FP64 hopping launches than FP32 ones
(the incremental updates did run and replaced FP64 recomputations).
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def system(lq):
    import torch
    dims, kappa, csw, nrhs = (16, 16, 16, 32), 0.128, 1.5, 16  # 65536 x 16 = 2^20 site-RHS
    U = inputs.gauge_field(dims, 0.4, seed=85)
    b = inputs.spinor_field(dims, seed=86, nrhs=nrhs)
    lat = lq.lattice_create(dims)
    gid = lq.gauge_upload(lat, U)
    dp = lq.dirac_params(kappa, csw)
    bt = torch.from_numpy(b).cuda()
    x64, info64, rc64 = lq.cg_solve(lat, gid, dp, lq.solver_params(tol=1e-10, maxiter=20000, precision="fp64"),
                                    bt, nrhs=nrhs)
    assert rc64 == lq.OK, info64
    yield dict(dims=dims, kappa=kappa, csw=csw, nrhs=nrhs, U=U, b=b, bt=bt, lat=lat, gid=gid, dp=dp,
               x64=x64.cpu().numpy())
    lq.lattice_destroy(lat)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_incremental_updates_meet_the_gates(lq, system, prec):
    s = system
    lq.profile_reset(timing=False)
    x, info, rc = lq.cg_solve(s["lat"], s["gid"], s["dp"],
                              lq.solver_params(tol=1e-10, maxiter=20000, precision=prec), s["bt"], nrhs=s["nrhs"])
    prof = lq.profile_read()
    assert rc == lq.OK, info
    assert all(i["true_resid"] <= 1e-10 for i in info)
    f32 = prof.get("hop_f32_selfclov", {}).get("launches", 0)
    f64 = prof.get("hop_f64_selfclov", {}).get("launches", 0)
    if prec == "fp16":  # the FP32 launches of an FP16 solve are the incremental updates
        assert f32 > 0 and f64 < f32, (f32, f64)
    x = x.cpu().numpy()
    for j in (0, s["nrhs"] // 2, s["nrhs"] - 1):
        r = s["b"][j] - oracle.dirac(s["dims"], s["U"], s["kappa"], s["csw"], x[j])
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(s["b"][j])
        assert rel(x[j], s["x64"][j]) <= 1e-8
