"""GPU parity of the even-odd preconditioned solver and the pion correlator.

Gates (every precision, the mixed ones included): true relative residual
|b - D x| / |b| <= 1e-10, computed by the FP64 oracle's own D on the returned
x; relative solution error <= 1e-8 against the oracle's solution (solved to
1e-13); pion C(t) <= 1e-8 relative per time slice.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp32", "fp16"]


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


def true_resid(dims, U, kappa, csw, x, b, theta=oracle.DEFAULT_THETA):
    return np.linalg.norm(b - oracle.dirac(dims, U, kappa, csw, x, theta=theta)) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", PRECS)
def test_point_source_solve_4x4(lq, prec):
    """4^4, eps = 0.2, kappa = 0.120, csw = 1.0, source (0,0,0,0) spin 0 colour 0, tol 1e-10."""
    dims, kappa, csw = (4, 4, 4, 4), 0.120, 1.0
    U = inputs.gauge_field(dims, 0.2, seed=1)
    b = inputs.point_source(dims, (0, 0, 0, 0), 0, 0)
    xo, it, res, ok = oracle.cgnr(dims, U, kappa, csw, b, tol=1e-13)
    assert ok
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(kappa, csw),
                                  lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), b)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert info[0]["true_resid"] <= 1e-10
    assert true_resid(dims, U, kappa, csw, x, b) <= 1e-10
    assert rel(x, xo) <= 1e-8


@pytest.mark.parametrize("dims", [(6, 4, 4, 8), (6, 6, 2, 6)])
def test_fp16_solve_identical_for_every_kernel_shape(lq, monkeypatch, dims):
    """Every FP16 hopping-kernel shape computes the same per-lane arithmetic,
    and the norms go through the same per-tile partial sums, so a whole
    mixed-precision solve (with the norm-computing kernel variants) must give
    the same bits whichever shape runs.  Three RHS on ragged lattices (6x6x2x6:
    216 sites per parity, a partly filled 32-site tile and an empty one)."""
    import torch
    kappa, csw = 0.13, 1.5
    theta = (1, np.exp(0.4j), 1, -1)
    U = inputs.gauge_field(dims, 0.4, seed=2)
    b = inputs.spinor_field(dims, seed=3, nrhs=3)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(kappa, csw, theta)
        sp = lq.solver_params(tol=1e-10, maxiter=5000, precision="fp16")
        sols = {}
        for nr, gpb in [(1, 1), (0, 1), (0, 2), (12, 1), (12, 2), (13, 1), (-4, 1), (2, 1), (20, 1), (20, 2), (21, 2)]:
            monkeypatch.setenv("LQCD_HOP_NR", str(nr))
            monkeypatch.setenv("LQCD_HOP_GPB", str(gpb))
            x, info, rc = lq.cg_solve(lat, gid, dp, sp, torch.from_numpy(b).cuda(), nrhs=3)
            assert rc == lq.OK, (nr, gpb, info)
            sols[(nr, gpb)] = x.cpu().numpy()
    finally:
        lq.lattice_destroy(lat)
    base = sols[(1, 1)]
    for j in range(3):
        assert true_resid(dims, U, kappa, csw, base[j], b[j], theta) <= 1e-10
    for k, v in sols.items():
        assert np.array_equal(v, base), k


@pytest.mark.parametrize("prec", PRECS)
def test_multi_rhs_batch_matches_single(lq, prec):
    """Three random right-hand sides in one batch, each also solved alone (ragged 6x4x4x8)."""
    import torch
    dims, kappa, csw = (6, 4, 4, 8), 0.13, 1.5
    theta = (1, np.exp(0.4j), 1, -1)
    U = inputs.gauge_field(dims, 0.4, seed=2)
    b = inputs.spinor_field(dims, seed=3, nrhs=3)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(kappa, csw, theta)
        sp = lq.solver_params(tol=1e-10, maxiter=5000, precision=prec)
        xb, infob, rc = lq.cg_solve(lat, gid, dp, sp, torch.from_numpy(b).cuda(), nrhs=3)
        assert rc == lq.OK
        xb = xb.cpu().numpy()
        for j in range(3):
            xs, infos, rc = lq.cg_solve(lat, gid, dp, sp, b[j])
            assert rc == lq.OK
            assert true_resid(dims, U, kappa, csw, xb[j], b[j], theta) <= 1e-10
            assert true_resid(dims, U, kappa, csw, xs, b[j], theta) <= 1e-10
            assert rel(xb[j], xs) <= 1e-8
            xo, *_ = oracle.cgnr(dims, U, kappa, csw, b[j], theta=theta, tol=1e-13)
            assert rel(xb[j], xo) <= 1e-8
    finally:
        lq.lattice_destroy(lat)


@pytest.mark.parametrize("prec", PRECS)
def test_pion_correlator_against_oracle(lq, prec):
    dims, kappa, csw = (6, 6, 6, 8), 0.125, 1.3
    src = (1, 2, 3, 5)
    U = inputs.gauge_field(dims, 0.3, seed=5)
    ref, prop_ref, *_ = oracle.pion(dims, U, kappa, csw, src, tol=1e-13, want_prop=True)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr, prop, info, rc = lq.pion_corr(lat, gid, lq.dirac_params(kappa, csw),
                                            lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), src,
                                            dims=dims, want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert np.all(np.abs(corr - ref) <= 1e-8 * np.abs(ref))
    for j in range(12):
        eta = inputs.point_source(dims, src, j // 3, j % 3)
        assert true_resid(dims, U, kappa, csw, prop[j], eta) <= 1e-10
        assert rel(prop[j], prop_ref[j]) <= 1e-8


def test_pion_contract_host_and_device(lq):
    import torch
    dims = (4, 6, 4, 6)
    rng = np.random.default_rng(1)
    prop = rng.normal(size=(12, 6, 4, 6, 4, 4, 3)) + 1j * rng.normal(size=(12, 6, 4, 6, 4, 4, 3))
    lat = lq.lattice_create(dims)
    try:
        for src_t in (0, 4):
            want = oracle.pion_contract(dims, prop, src_t)
            got = lq.pion_contract(lat, prop, src_t)
            assert np.allclose(got, want, rtol=1e-13, atol=0)
            c = torch.zeros(6, dtype=torch.float64, device="cuda")
            lq.pion_contract(lat, torch.from_numpy(prop).cuda(), src_t, corr=c)
            assert np.allclose(c.cpu().numpy(), want, rtol=1e-13, atol=0)
    finally:
        lq.lattice_destroy(lat)


def test_free_field_pion_closed_form_via_oracle(lq):
    dims = (4, 4, 4, 8)
    U = inputs.unit_gauge_field(dims)
    ref, *_ = oracle.pion(dims, U, 0.12, 1.0, (0, 0, 0, 0), tol=1e-13)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr, _, info, rc = lq.pion_corr(lat, gid, lq.dirac_params(0.12, 1.0),
                                         lq.solver_params(tol=1e-10, precision="fp16"), (0, 0, 0, 0), dims=dims)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK
    assert np.all(np.abs(corr - ref) <= 1e-8 * ref)


def test_maxiter_gives_enoconv(lq):
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.4, seed=9)
    b = inputs.spinor_field(dims, seed=10)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        for prec in PRECS:
            x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(0.13, 1.5),
                                      lq.solver_params(tol=1e-10, maxiter=1, precision=prec), b)
            assert rc == lq.ENOCONV
            assert info[0]["status"] == lq.ENOCONV and info[0]["iters_inner"] <= 2
        # the lattice is still usable afterwards
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(0.13, 1.5), lq.solver_params(tol=1e-10), b)
        assert rc == lq.OK
    finally:
        lq.lattice_destroy(lat)


def test_zero_source_and_bad_arguments(lq):
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.2, seed=1)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(0.12, 1.0), lq.solver_params(), np.zeros((4, 4, 4, 4, 4, 3)))
        assert rc == lq.OK and np.all(x == 0) and info[0]["iters_inner"] == 0
        with pytest.raises(lq.LqcdError) as e:
            lq.pion_corr(lat, gid, lq.dirac_params(0.12, 1.0), lq.solver_params(), (4, 0, 0, 0), dims=dims)
        assert e.value.code == lq.EINVAL
        with pytest.raises(lq.LqcdError) as e:
            lq.cg_solve(lat, gid, lq.dirac_params(0.12, 1.0, mu=float("nan")), lq.solver_params(),
                        np.zeros((4, 4, 4, 4, 4, 3)))
        assert e.value.code == lq.EINVAL
        with pytest.raises(lq.LqcdError) as e:
            lq.cg_solve(lat, 99, lq.dirac_params(0.12, 1.0), lq.solver_params(), np.zeros((4, 4, 4, 4, 4, 3)))
        assert e.value.code == lq.EINVAL
    finally:
        lq.lattice_destroy(lat)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_propagator_16x32_full_size(lq, prec):
    """16^3 x 32, eps = 0.4, kappa = 0.130, csw = 1.5: the 12-column propagator and C(t).

    The oracle cannot solve this size in test time, so the properties are:
    every column's true residual (oracle D on the full lattice) <= 1e-10, and
    C(t) equal to the oracle's contraction of the returned columns.
    """
    dims, kappa, csw = (16, 16, 16, 32), 0.130, 1.5
    U = inputs.gauge_field(dims, 0.4, seed=1, workers=None)
    src = (0, 0, 0, 0)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr, prop, info, rc = lq.pion_corr(lat, gid, lq.dirac_params(kappa, csw),
                                            lq.solver_params(tol=1e-10, maxiter=20000, precision=prec), src,
                                            dims=dims, want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert np.allclose(corr, oracle.pion_contract(dims, prop, src[3]), rtol=1e-12, atol=0)
    for j in (0, 5, 11):
        eta = inputs.point_source(dims, src, j // 3, j % 3)
        assert true_resid(dims, U, kappa, csw, prop[j], eta) <= 1e-10


def test_propagator_32x64_bench_configuration(lq):
    """32^3 x 64, eps 0.4, kappa 0.132, csw 1.7, FP16 storage, 12 RHS, tol
    1e-10: the benchmark's propagator, in the call the benchmark times.

    Checked at this size: C(t) equals the oracle's contraction of the returned
    columns, and for three columns the residual eta - D S_j at sampled sites
    (the source, its 8 neighbours, two corners and 300 random sites), with
    the oracle's D, is at most 1e-10 per site: |eta| = 1, so a true residual
    <= 1e-10 bounds every site.
    """
    dims, kappa, csw = (32, 32, 32, 64), 0.132, 1.7
    U = inputs.gauge_field(dims, 0.4, seed=1, workers=None)
    src = (0, 0, 0, 0)
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr, prop, info, rc = lq.pion_corr(lat, gid, lq.dirac_params(kappa, csw),
                                            lq.solver_params(tol=1e-10, maxiter=20000, precision="fp16"), src,
                                            dims=dims, want_prop=True)
    finally:
        lq.lattice_destroy(lat)
    assert rc == lq.OK, info
    assert max(i["true_resid"] for i in info) <= 1e-10
    assert np.allclose(corr, oracle.pion_contract(dims, prop, src[3]), rtol=1e-12, atol=0)
    V = inputs.volume(dims)
    # source at the origin; lexicographic index x + 32 (y + 32 (z + 32 t))
    near = [0, 1, 31, 32, 32 * 31, 32 * 32, 32 * 32 * 31, 32 ** 3, 32 ** 3 * 63, V - 1]
    rng = np.random.default_rng(1)
    sites = np.unique(np.concatenate([near, rng.integers(0, V, 300)]))
    for j in (0, 5, 11):
        eta = inputs.point_source(dims, src, j // 3, j % 3).reshape(V, 4, 3)[sites]
        r = eta - oracle.dirac_sites(dims, U, kappa, csw, prop[j], sites)
        assert np.max(np.abs(r)) <= 1e-10, (j, np.max(np.abs(r)))
