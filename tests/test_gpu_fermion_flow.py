"""GPU fermion gradient flow (Sec. 3.2) against the FP64 oracle.

The oracle's flow (covariant Laplacian, third-order scheme on the gauge RK3
stages) is pinned in test_oracle_pins.py.  Gates: flowed links within 1e-12
of the oracle's, flowed quark fields within 1e-12 relative (every element on
the scale of the largest), a free plane wave multiplied by the RK3 step
polynomial exactly as the closed form says, the host and device paths equal,
and bad arguments rejected.
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


def test_fermion_flow_matches_oracle(lq):
    import torch
    dims, eps, n, nrhs = (4, 6, 4, 6), 0.02, 5, 2
    th = (1, np.exp(0.5j), np.exp(-0.3j), -1)
    U = inputs.gauge_field(dims, 0.35, seed=101)
    chi = inputs.spinor_field(dims, seed=102, nrhs=nrhs)
    Uo, co = oracle.fermion_flow(dims, U, chi, eps, n, theta=th, nrhs=nrhs)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dev = torch.from_numpy(chi.copy()).cuda()
        lq.fermion_flow(lat, gid, lq.dirac_params(0.13, 1.2, th), dev, eps, n, nrhs=nrhs)
        got = dev.cpu().numpy()
        Ug = lq.gauge_download(lat, gid, dims)
        gid2 = lq.gauge_upload(lat, U)
        host = lq.fermion_flow(lat, gid2, lq.dirac_params(0.13, 1.2, th), chi, eps, n, nrhs=nrhs)
        with pytest.raises(lq.LqcdError) as e:
            lq.fermion_flow(lat, gid, lq.dirac_params(0.13, 1.2, th, bc="open"), chi, eps, 1, nrhs=nrhs)
        assert e.value.code == lq.EINVAL
        with pytest.raises(lq.LqcdError) as e:
            lq.fermion_flow(lat, gid, lq.dirac_params(0.13, 1.2, th), chi, 0.0, 1, nrhs=nrhs)
        assert e.value.code == lq.EINVAL
    finally:
        lq.lattice_destroy(lat)
    assert np.max(np.abs(Ug - Uo)) <= 1e-12
    assert np.max(np.abs(got - co)) <= 1e-12 * np.max(np.abs(co))
    assert np.linalg.norm(got - co) <= 1e-12 * np.linalg.norm(co)
    assert np.array_equal(host, got)


def test_free_plane_wave_step_factor(lq):
    dims, eps, n = (4, 2, 6, 4), 0.05, 4
    th = (np.exp(0.7j), np.exp(-1.1j), 1, np.exp(2.3j))
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    nn = (1, 1, 2, 3)
    p = [(2 * np.pi * nn[mu] + np.angle(th[mu])) / dims[mu] for mu in range(4)]
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = np.random.default_rng(9).normal(size=(4, 3)) + 0j
    psi = phase[..., None, None] * u
    h = -eps * sum(4 * np.sin(pm / 2) ** 2 for pm in p)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, inputs.unit_gauge_field(dims))
        got = lq.fermion_flow(lat, gid, lq.dirac_params(0.1, 0.0, th), psi, eps, n)
    finally:
        lq.lattice_destroy(lat)
    want = (1 + h + h * h / 2 + h ** 3 / 6) ** n * psi
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("nsave", [1, 2, 5])
def test_backflow_matches_oracle_and_is_the_adjoint(lq, nsave):
    import torch
    dims, eps, n, nrhs = (4, 6, 4, 6), 0.03, 5, 2
    th = (np.exp(0.2j), 1, np.exp(-0.6j), -1)
    U = inputs.gauge_field(dims, 0.35, seed=103)
    eta = inputs.spinor_field(dims, seed=104, nrhs=nrhs)
    chi = inputs.spinor_field(dims, seed=105, nrhs=nrhs)
    want = oracle.fermion_backflow(dims, U, eta, eps, n, theta=th, nrhs=nrhs)
    dp = lq.dirac_params(0.13, 1.2, th)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dev = torch.from_numpy(eta.copy()).cuda()
        lq.fermion_backflow(lat, gid, dp, dev, eps, n, nrhs=nrhs, nsave=nsave)
        got = dev.cpu().numpy()
        assert np.array_equal(lq.gauge_download(lat, gid, dims), U)  # the links stay at t = 0
        fwd = lq.fermion_flow(lat, gid, dp, chi, eps, n, nrhs=nrhs)
        with pytest.raises(lq.LqcdError) as e:
            lq.fermion_backflow(lat, gid, dp, eta, eps, n, nrhs=nrhs, nsave=0)
        assert e.value.code == lq.EINVAL
    finally:
        lq.lattice_destroy(lat)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    for j in range(nrhs):  # <eta, F chi> = <B eta, chi> with both flows on the GPU
        lhs, rhs = np.vdot(eta[j], fwd[j]), np.vdot(got[j], chi[j])
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_backflow_checkpointing_gives_the_same_bits(lq):
    dims, eps, n = (4, 4, 4, 4), 0.02, 7
    U = inputs.gauge_field(dims, 0.3, seed=106)
    eta = inputs.spinor_field(dims, seed=107)
    dp = lq.dirac_params(0.13, 1.2)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        outs = [lq.fermion_backflow(lat, gid, dp, eta, eps, n, nsave=k) for k in (1, 3, 7, 9)]
        zero = lq.fermion_backflow(lat, gid, dp, eta, eps, 0)
    finally:
        lq.lattice_destroy(lat)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert np.array_equal(zero, eta)
