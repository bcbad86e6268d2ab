"""GPU propagators against oracle-solved golden files (tests/golden/).

The golden files hold the 12-column point-source propagator of a seeded
configuration as solved by the FP64 CPU oracle (unpreconditioned CGNR to a
true residual of 1e-13, written by tests/golden/make_pion_golden.py): C(t),
C(t) per column, |x_j|^2 and every component of every column at sampled
sites.  lqcd_pion_corr must match them in every precision, with the gates of
the solver tests: C(t) within 1e-8 relative per time slice, the propagator
within 1e-8 relative (per column, against its largest sampled value), and a
true residual <= 1e-10 (C(t) per column within 1e-8 of the slice's C(t)).

Configurations: 4^4 (eps 0.2, kappa 0.120, csw 1.0) and 16^3 x 32 (eps 0.4,
kappa 0.130, csw 1.5), seed 1, source at the origin.
"""
import json
import os

import numpy as np
import pytest

from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = {"4c4": "pion_4c4_seed1.json", "16c32": "pion_16c32_seed1.json"}


@pytest.fixture(scope="module")
def lq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_16994_gb300 import lqcd
    return lqcd


def load(name):
    with open(os.path.join(HERE, "golden", GOLDEN[name])) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["4c4", "16c32"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_pion_propagator_matches_oracle_golden(lq, name, prec):
    import torch
    doc = load(name)
    c = doc["config"]
    dims = tuple(c["dims"])
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, c["eps"], seed=c["seed"], workers=None)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr = torch.zeros(dims[3], dtype=torch.float64, device="cuda")
        prop = torch.zeros(12 * V * 12, dtype=torch.complex128, device="cuda")
        _, _, infos, rc = lq.pion_corr(lat, gid, lq.dirac_params(c["kappa"], c["csw"], tuple(c["theta"])),
                                       lq.solver_params(tol=1e-10, maxiter=20000, precision=prec), tuple(c["src"]),
                                       device_out=(corr, prop))
        torch.cuda.synchronize()
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, infos
    assert all(i["true_resid"] <= 1e-10 for i in infos)
    ref = np.asarray(doc["corr"])
    got = corr.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-8 * ref), np.max(np.abs(got - ref) / ref)
    S = prop.cpu().numpy().reshape(12, dims[3], dims[2], dims[1], dims[0], 12)
    src_t = c["src"][3]
    per_t = np.roll(np.sum(np.abs(S) ** 2, axis=(2, 3, 4, 5)), -src_t, axis=1)
    colref = np.asarray(doc["corr_col"])
    # per column, on the scale of the slice's C(t) (single columns can be far smaller)
    assert np.all(np.abs(per_t - colref) <= 1e-8 * ref[None, :]), np.max(np.abs(per_t - colref) / ref[None, :])
    assert np.all(np.abs(np.sum(np.abs(S) ** 2, axis=(1, 2, 3, 4, 5)) - doc["x_norm2"])
                  <= 2e-8 * np.asarray(doc["x_norm2"]))
    vals = np.asarray(doc["samples"]["values"])
    want = vals[..., 0] + 1j * vals[..., 1]  # [column][site][component]
    for j in range(12):
        g = np.array([S[j, s[3], s[2], s[1], s[0]] for s in doc["samples"]["sites"]])
        assert np.max(np.abs(g - want[j])) <= 1e-8 * np.max(np.abs(want[j])), (j, np.max(np.abs(g - want[j])))
