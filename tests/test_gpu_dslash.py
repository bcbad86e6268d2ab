"""GPU parity of the FP64 Wilson-clover operator against the oracle.

Gate: relative L2 error <= 1e-13 (FP64 Dslash).  Sizes span several 128-site
tiles with ragged tails, the degenerate L = 2 extent (x+mu and x-mu are the
same site), twisted complex boundary phases, the dagger, host and device
pointers, and sampled sites of the 32^3 x 64 lattice.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13


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


CASES = [
    ((2, 2, 2, 2), 0.4, 0.13, 1.5, (1, 1, 1, -1)),
    ((4, 4, 4, 4), 0.2, 0.12, 1.0, (1, 1, 1, -1)),
    ((6, 4, 4, 8), 0.4, 0.132, 1.7, (1, 1, 1, -1)),          # Vh = 384: 3 tiles
    ((4, 6, 2, 10), 0.4, 0.13, 1.5, (np.exp(0.3j), 1, np.exp(-1.2j), -1)),  # Vh = 240: ragged
    ((8, 8, 8, 8), 0.3, 0.125, 1.3, (1, 1, 1, -1)),          # Vh = 2048
    ((10, 6, 4, 6), 0.5, 0.137, 2.0, (1, np.exp(2.0j), 1, np.exp(0.5j))),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_fp64_host_pointers(lq, case, dagger):
    dims, eps, kappa, csw, theta = case
    U = inputs.gauge_field(dims, eps, seed=7)
    psi = inputs.spinor_field(dims, seed=8)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        got = lq.dirac_apply(lat, gid, lq.dirac_params(kappa, csw, theta), psi, dagger=dagger)
    finally:
        lq.lattice_destroy(lat)
    want = oracle.dirac(dims, U, kappa, csw, psi, theta=theta, dagger=dagger)
    assert rel(got, want) <= TOL


def test_dslash_fp64_device_pointers_and_cache(lq):
    import torch
    dims = (6, 4, 4, 8)
    U = inputs.gauge_field(dims, 0.4, seed=3)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        for kappa, csw in [(0.13, 1.5), (0.12, 1.0), (0.13, 1.5)]:  # clover cache hit on the third
            psi = inputs.spinor_field(dims, seed=int(kappa * 1000))
            got = lq.dirac_apply(lat, gid, lq.dirac_params(kappa, csw), torch.from_numpy(psi).cuda())
            assert rel(got.cpu().numpy(), oracle.dirac(dims, U, kappa, csw, psi)) <= TOL
        # a second resident field on the same lattice
        U2 = inputs.gauge_field(dims, 0.3, seed=4)
        gid2 = lq.gauge_upload(lat, U2)
        psi = inputs.spinor_field(dims, seed=5)
        got = lq.dirac_apply(lat, gid2, lq.dirac_params(0.13, 1.5), psi)
        assert rel(got, oracle.dirac(dims, U2, 0.13, 1.5, psi)) <= TOL
        lq.gauge_free(lat, gid2)
        with pytest.raises(lq.LqcdError):
            lq.dirac_apply(lat, gid2, lq.dirac_params(0.13, 1.5), psi)
    finally:
        lq.lattice_destroy(lat)


def test_dslash_free_field_is_clover_free(lq):
    dims = (4, 4, 4, 6)
    U = inputs.unit_gauge_field(dims)
    psi = inputs.spinor_field(dims, seed=1)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        a = lq.dirac_apply(lat, gid, lq.dirac_params(0.13, 1.9), psi)
        b = lq.dirac_apply(lat, gid, lq.dirac_params(0.13, 0.0), psi)
    finally:
        lq.lattice_destroy(lat)
    assert rel(a, b) <= 1e-15


def test_dslash_fp64_full_size_sampled(lq):
    """32^3 x 64 (the benchmark lattice): sampled sites against the oracle."""
    import torch
    dims = (32, 32, 32, 64)
    kappa, csw = 0.132, 1.7
    U = inputs.gauge_field(dims, 0.4, seed=1, workers=None)
    psi = inputs.spinor_field(dims, seed=2)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        for dag in (False, True):
            got = lq.dirac_apply(lat, gid, lq.dirac_params(kappa, csw), torch.from_numpy(psi).cuda(),
                                 dagger=dag).cpu().numpy()
            V = inputs.volume(dims)
            rng = np.random.default_rng(0)
            corners = [0, V - 1, 31, 32 * 31, 32 * 32 * 31, 32 ** 3 * 63]
            sites = np.unique(np.concatenate([corners, rng.integers(0, V, 400)]))
            if not dag:
                want = oracle.dirac_sites(dims, U, kappa, csw, psi, sites)
            else:
                # D^dag = g5 D g5
                g5 = np.array([1, 1, -1, -1])[:, None]
                want = g5 * oracle.dirac_sites(dims, U, kappa, csw, g5 * psi, sites)
            flat = got.reshape(V, 4, 3)[sites]
            assert rel(flat, want) <= TOL
    finally:
        lq.lattice_destroy(lat)
