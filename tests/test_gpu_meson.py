"""GPU parity of the meson contraction (lqcd_meson_contract) against the
FP64 oracle, for the 16 Clifford spin matrices and dense random ones.

The contraction is defined for any 12-column array, so small cases use
random arrays (every entry exercised) and a solved propagator; the full
32^3x64 size is checked on two time slices by the oracle (the contraction
is site-local, so two slices cut out as a T = 2 lattice give the same
per-slice sums) and on every slice by two properties that hold at any size:
G = g5 equals the pion contraction, and the sum over the 16 Clifford
channels equals -4 sum_x tr_c[tr_s(S g_t) tr_s(g_t g5 S^dag g5)].
Gate: relative error <= 1e-12 (FP64 sums in a different order).
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


def clifford16():
    g = [oracle.gamma(mu) for mu in range(4)]
    out = [np.eye(4, dtype=complex)] + g
    out += [g[m] @ g[n] for m in range(4) for n in range(m + 1, 4)]
    out += [g[m] @ g[n] @ g[r] for m in range(4) for n in range(m + 1, 4) for r in range(n + 1, 4)]
    out.append(oracle.gamma(4))
    return np.array(out)


def random_prop(dims, seed):
    rng = np.random.default_rng(seed)
    shape = (12, dims[3], dims[2], dims[1], dims[0], 4, 3)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("dims,src_t", [((6, 4, 4, 10), 0), ((4, 6, 2, 8), 5), ((2, 2, 2, 2), 1)])
def test_meson_contract_matches_oracle(lq, dims, src_t):
    import torch
    rng = np.random.default_rng(7)
    gammas = np.concatenate([clifford16(), rng.normal(size=(2, 4, 4)) + 1j * rng.normal(size=(2, 4, 4))])
    prop = random_prop(dims, 11)
    want = oracle.meson_contract(dims, prop, src_t, gammas)
    lat = lq.lattice_create(dims)
    try:
        got = lq.meson_contract(lat, prop, src_t, gammas)
        assert rel(got, want) <= 1e-12
        for g in range(len(gammas)):
            assert rel(got[g], want[g]) <= 1e-12, g
        c = torch.zeros((len(gammas), dims[3]), dtype=torch.complex128, device="cuda")
        lq.meson_contract(lat, torch.from_numpy(prop).cuda(), src_t, gammas, corr=c)
        torch.cuda.synchronize()
        assert rel(c.cpu().numpy(), want) <= 1e-12
        # a single channel alone gives the same numbers
        one = lq.meson_contract(lat, prop, src_t, gammas[3:4])
        assert rel(one[0], want[3]) <= 1e-12
    finally:
        lq.lattice_destroy(lat)


def test_meson_on_a_solved_propagator(lq):
    """Point-source propagator from lqcd_pion_corr (FP64) on 6^3x8: every
    Clifford channel against the oracle's contraction of the oracle's own
    propagator, and the g5 channel against the pion correlator."""
    dims, kappa, csw = (6, 6, 6, 8), 0.125, 1.3
    src = (1, 2, 3, 5)
    U = inputs.gauge_field(dims, 0.3, seed=5)
    ref_corr, prop_ref, *_ = oracle.pion(dims, U, kappa, csw, src, tol=1e-13, want_prop=True)
    want = oracle.meson_contract(dims, prop_ref, src[3], clifford16())
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        corr, prop, info, rc = lq.pion_corr(lat, gid, lq.dirac_params(kappa, csw),
                                            lq.solver_params(tol=1e-10, maxiter=5000, precision="fp64"), src,
                                            dims=dims, want_prop=True)
        assert rc == lq.OK
        got = lq.meson_contract(lat, prop, src[3], clifford16())
    finally:
        lq.lattice_destroy(lat)
    # the propagators agree to ~1e-9 (solver tolerance), so do the channels
    # (measured against the largest channel: some channels are small on one
    # configuration)
    scale = max(np.linalg.norm(w) for w in want)
    for g in range(16):
        assert np.linalg.norm(got[g] - want[g]) <= 1e-7 * scale, g
    assert rel(got[15].real, corr) <= 1e-12
    assert np.max(np.abs(got[15].imag)) <= 1e-12 * np.max(corr)
    assert rel(got[15].real, ref_corr) <= 1e-8


@pytest.mark.parametrize("dims", [(16, 16, 16, 32), (32, 32, 32, 64)])
def test_meson_full_size(lq, dims):
    import torch
    T = dims[3]
    src_t = 3
    V = int(np.prod(dims))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(13)
    p = torch.randn((12, T, dims[2], dims[1], dims[0], 4, 3, 2), dtype=torch.float64, device="cuda",
                    generator=gen)
    prop = torch.view_as_complex(p)
    del p
    gam = clifford16()
    lat = lq.lattice_create(dims)
    try:
        c = torch.zeros((16, T), dtype=torch.complex128, device="cuda")
        lq.meson_contract(lat, prop, src_t, gam, corr=c)
        pc = torch.zeros(T, dtype=torch.float64, device="cuda")
        lq.pion_contract(lat, prop, src_t, corr=pc)
        torch.cuda.synchronize()
        got = c.cpu().numpy()
        pion = pc.cpu().numpy()
        # g5 channel = pion
        assert rel(got[15].real, pion) <= 1e-12
        # Fierz: sum over the 16 channels, right side from the propagator with torch ops
        gt = torch.from_numpy(oracle.gamma(3)).cuda()
        g5d = torch.from_numpy(np.diag(oracle.gamma(4)).copy()).cuda()
        S = prop.reshape(4, 3, T, -1, 4, 3).permute(2, 3, 4, 5, 0, 1)      # [t, site, A, a, B, b]
        M = torch.einsum("tsAaBb,BA->tsab", S, gt)
        Tm = torch.einsum("A,tsBbAa,B->tsAaBb", g5d, S.conj(), g5d)
        N = torch.einsum("AB,tsBaAb->tsab", gt, Tm)
        rhs_t = (-4 * torch.einsum("tsab,tsba->t", M, N)).cpu().numpy()
        del S, M, Tm, N
        rhs = np.array([rhs_t[(src_t + t) % T] for t in range(T)])
        assert rel(got.sum(axis=0), rhs) <= 1e-12
        # two slices by the oracle, cut out as a T = 2 lattice
        sl = [src_t, (src_t + 5) % T]
        sub = prop[:, sl].cpu().numpy()
        want = oracle.meson_contract((dims[0], dims[1], dims[2], 2), sub, 0, gam)
        assert rel(got[:, [0, 5]], want) <= 1e-12
    finally:
        lq.lattice_destroy(lat)
        del prop
        torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_noise_source_propagator(lq, prec):
    """Noise-source propagators (Sec. 3.3 propagator! with random sources):
    lqcd_cg_solve on a Z2 source on one time slice, against the oracle's
    solve of the same source, and the one-end estimator sum_x |psi|^2 per
    slice through lqcd_pion_contract (the column in slot 0, the others zero)."""
    dims, kappa, csw = (6, 4, 4, 8), 0.125, 1.4
    t0 = 3
    U = inputs.gauge_field(dims, 0.3, seed=9)
    eta = inputs.noise_source(dims, t0, seed=17, kind="z2")
    x_ref, it, res, ok = oracle.cgnr(dims, U, kappa, csw, eta, tol=1e-13)
    assert ok
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        x, info, rc = lq.cg_solve(lat, gid, lq.dirac_params(kappa, csw),
                                  lq.solver_params(tol=1e-10, maxiter=5000, precision=prec), eta)
        assert rc == lq.OK, info
        r = eta - oracle.dirac(dims, U, kappa, csw, x)
        assert np.linalg.norm(r) / np.linalg.norm(eta) <= 1e-10
        assert rel(x, x_ref) <= 1e-8
        cols = np.zeros((12,) + x.shape, dtype=np.complex128)
        cols[0] = x
        c = lq.pion_contract(lat, cols, t0)
    finally:
        lq.lattice_destroy(lat)
    want = np.sum(np.abs(x_ref) ** 2, axis=(1, 2, 3, 4, 5))
    want = np.array([want[(t0 + t) % dims[3]] for t in range(dims[3])])
    assert np.all(np.abs(c - want) <= 1e-8 * want)
