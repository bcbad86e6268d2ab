"""GPU parity of the even-odd preconditioned operator Dhat in every storage format.

FP64: checked against the oracle through the Schur identity: if w = Dhat x_e
then D^-1 (w on the even sites, 0 on the odd) has x_e on its even sites.
FP32 and FP16 storage: against the GPU FP64 operator, relative L2 <= 2e-6
(FP32) and <= 4e-3 (FP16 mantissa 2^-11 with per-site scale), including a
field spanning ~40 decades (a decaying propagator-like profile whose tail
is FP32-denormal), which must stay finite.
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


def parity_mask(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2 == 0)[..., None, None]


G5 = np.array([1, 1, -1, -1])[:, None]


@pytest.mark.parametrize("dagger", [False, True])
def test_schur_fp64_identity_with_oracle(lq, dagger):
    dims, kappa, csw = (6, 4, 4, 8), 0.13, 1.6
    theta = (1, np.exp(0.7j), 1, -1)
    U = inputs.gauge_field(dims, 0.4, seed=12)
    ev = parity_mask(dims)
    x = inputs.spinor_field(dims, seed=13) * ev
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        w = lq.schur_apply(lat, gid, lq.dirac_params(kappa, csw, theta), x, precision="fp64", dagger=dagger)
    finally:
        lq.lattice_destroy(lat)
    assert np.all(w[~np.broadcast_to(ev, w.shape)] == 0)
    b = G5 * w if dagger else w  # Dhat^dag = g5 Dhat g5
    chi, it, res, ok = oracle.cgnr(dims, U, kappa, csw, b, theta=theta, tol=1e-13)
    assert ok
    got = G5 * chi if dagger else chi
    assert rel(got * ev, x) <= 1e-10


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (16, 16, 16, 32)])
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 4e-3)])
def test_schur_low_precision_against_fp64(lq, dims, prec, tol):
    import torch
    kappa, csw = 0.132, 1.7
    U = inputs.gauge_field(dims, 0.4, seed=3, workers=None)
    ev = parity_mask(dims)
    x = inputs.spinor_field(dims, seed=4, nrhs=2) * ev
    # second field: decaying profile exp(-3 |t - T/2|) -> tail ~ 1e-42 (FP32 denormal)
    lt = dims[3]
    prof = np.exp(-3.0 * np.abs(np.arange(lt) - lt // 2))[:, None, None, None, None, None]
    x[1] = x[1] * prof
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(kappa, csw)
        xt = torch.from_numpy(x).cuda()
        for dag in (False, True):
            ref = lq.schur_apply(lat, gid, dp, xt, precision="fp64", nrhs=2, dagger=dag).cpu().numpy()
            got = lq.schur_apply(lat, gid, dp, xt, precision=prec, nrhs=2, dagger=dag).cpu().numpy()
            assert np.all(np.isfinite(got))
            for j in range(2):
                assert rel(got[j], ref[j]) <= tol, (j, rel(got[j], ref[j]))
            # batched equals single
            one = lq.schur_apply(lat, gid, dp, xt[1].contiguous(), precision=prec, dagger=dag).cpu().numpy()
            assert np.array_equal(one, got[1])
    finally:
        lq.lattice_destroy(lat)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 4e-3)])
def test_every_kernel_shape_agrees(lq, prec, tol, monkeypatch):
    """Forces each hopping-kernel shape the autotuner can pick (two right-hand
    sides per thread in packed FP32x2 lanes, plain, with 2/3 directions of
    words staged in shared memory, or with links and clover prepared once per
    32-site tile in shared memory, 1-3 per thread in scalar arithmetic, or
    one per thread with 2/4/8 directions of loads issued ahead, times groups
    per block and the super-tile block order) and checks it against FP64.
    In FP16 storage every shape computes the same per-lane arithmetic, so all
    shapes must give identical bits."""
    import torch
    dims, kappa, csw = (6, 4, 4, 10), 0.13, 1.6
    U = inputs.gauge_field(dims, 0.4, seed=21)
    ev = parity_mask(dims)
    nrhs = 5  # odd: exercises a half-empty last pair / group
    x = inputs.spinor_field(dims, seed=22, nrhs=nrhs) * ev
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(kappa, csw, (1, np.exp(0.3j), 1, -1))
        xt = torch.from_numpy(x).cuda()
        outs = {}
        for dag in (False, True):
            ref = lq.schur_apply(lat, gid, dp, xt, precision="fp64", nrhs=nrhs, dagger=dag).cpu().numpy()
            for nr, gpb, swz in [(0, 1, 1), (0, 3, 1), (0, 1, 8), (1, 1, 1), (1, 5, 1), (1, 1, 8), (2, 1, 1), (2, 3, 1),
                                 (3, 1, 32), (-2, 1, 1), (-4, 5, 1), (-8, 1, 8), (12, 1, 1), (12, 3, 1), (13, 2, 8),
                                 (20, 1, 1), (20, 3, 1), (21, 2, 1)]:
                monkeypatch.setenv("LQCD_HOP_NR", str(nr))
                monkeypatch.setenv("LQCD_HOP_GPB", str(gpb))
                monkeypatch.setenv("LQCD_HOP_SWZ", str(swz))
                got = lq.schur_apply(lat, gid, dp, xt, precision=prec, nrhs=nrhs, dagger=dag).cpu().numpy()
                for j in range(nrhs):
                    assert rel(got[j], ref[j]) <= tol, (nr, gpb, j)
                outs[(dag, nr, gpb, swz)] = got
            base = outs[(dag, 1, 1, 1)]
            for k, v in outs.items():
                if k[0] == dag:
                    if prec == "fp16":
                        assert np.array_equal(v, base), k
                    else:
                        assert rel(v, base) <= 50 * 2e-7, k
    finally:
        lq.lattice_destroy(lat)
