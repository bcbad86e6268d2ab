"""Seeded synthetic inputs for the Wilson-clover propagator path.

This module only *makes inputs*: random near-unit SU(3) gauge fields, random
spinor fields, point sources and random gauge transformations.  It holds none
of the Dirac-operator, solver or contraction arithmetic, so both the CUDA path
and the FP64 oracle can be fed from it without sharing any method code.

Layouts (the library's host layout, lexicographic with x fastest, t slowest):

* gauge field  ``U[t, z, y, x, mu, a, b]`` complex128, mu = 0,1,2,3 = x,y,z,t
  (the paper puts time last, Sec. 2.1), row-major 3x3 link matrices.
* spinor field ``psi[t, z, y, x, spin, colour]`` complex128 (index 3*spin+colour).

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw k of a
stream with seed ``s`` is ``mix(s + (k+1) * 0x9E3779B97F4A7C15)``.  Uniforms
are ``((z >> 11) + 0.5) * 2**-53`` in (0, 1); normals come in pairs from the
Box-Muller transform of consecutive uniforms.

Synthetic gauge links are ``U = exp(i eps H)`` with ``H = sum_a h_a lambda_a/2``
(Gell-Mann matrices, ``h_a ~ N(0,1)`` i.i.d.).  Draw order: site
lexicographic (x fastest), then mu, then a.  The paper generates its fields
with HMC (Sec. 3.1, 4); near-unit random SU(3) fields of this kind stand in
for those ensembles here.
"""
from __future__ import annotations

import os

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normals(seed: int, start: int, count: int) -> np.ndarray:
    """Standard normals n_start .. n_start+count-1 (Box-Muller on uniform pairs).

    Normal ``2j`` is ``r cos(2 pi u_{2j+1})`` and normal ``2j+1`` is
    ``r sin(2 pi u_{2j+1})`` with ``r = sqrt(-2 ln u_{2j})``.
    """
    if count == 0:
        return np.zeros(0)
    j0 = start // 2
    j1 = (start + count + 1) // 2
    u = uniforms(seed, 2 * j0, 2 * (j1 - j0)).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty(2 * (j1 - j0))
    out[0::2] = r * np.cos(ang)
    out[1::2] = r * np.sin(ang)
    off = start - 2 * j0
    return out[off:off + count]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def expm_i_hermitian(h: np.ndarray) -> np.ndarray:
    """exp(i h) for a stack of Hermitian 3x3 matrices h (..., 3, 3).

    Scaling and squaring: h is scaled by 2**-s so that its Frobenius norm is
    <= 1/2, the degree-15 Taylor polynomial is evaluated by the
    Paterson-Stockmeyer scheme (powers A^2, A^3, A^4, then Horner in A^4; 6
    matrix products) and the result is squared s times.  The truncation error
    (< 0.5^16/16!) is far below double rounding.
    """
    shape = h.shape
    h = h.reshape(-1, 3, 3)
    nrm = np.sqrt(np.sum(np.abs(h) ** 2, axis=(1, 2)))
    s = int(max(0, np.ceil(np.log2(max(float(nrm.max(initial=0.0)), 1e-300) / 0.5))))
    a = 1j * h / (2.0 ** s)
    eye = np.eye(3, dtype=np.complex128)
    a2 = np.matmul(a, a)
    a3 = np.matmul(a2, a)
    a4 = np.matmul(a2, a2)
    fact = [1.0]
    for k in range(1, 16):
        fact.append(fact[-1] * k)

    def block(m):  # sum_{r=0..3} A^r / (4m + r)!
        return (eye / fact[4 * m] + a / fact[4 * m + 1] + a2 / fact[4 * m + 2] + a3 / fact[4 * m + 3])

    out = block(3)
    for m in (2, 1, 0):
        out = np.matmul(out, a4) + block(m)
    for _ in range(s):
        out = np.matmul(out, out)
    return out.reshape(shape)


def volume(dims) -> int:
    lx, ly, lz, lt = dims
    return int(lx) * int(ly) * int(lz) * int(lt)


def _gauge_chunk(args):
    s0, s1, eps, seed = args
    lam = gell_mann() / 2.0
    h = normals(seed, s0 * 32, (s1 - s0) * 32).reshape(s1 - s0, 4, 8)
    return expm_i_hermitian(eps * np.einsum("sma,aij->smij", h, lam))


def _spawn_safe() -> bool:
    """True when spawned workers can re-import the main module (not a stdin script)."""
    import sys
    path = getattr(sys.modules.get("__main__"), "__file__", None)
    return path is None or os.path.exists(path)


def gauge_field(dims, eps: float, seed: int, chunk_sites: int = 1 << 16, workers: int | None = 1) -> np.ndarray:
    """Synthetic links U_mu(x) = exp(i eps H), shape (T, Z, Y, X, 4, 3, 3).

    ``dims = (Lx, Ly, Lz, T)``.  Sites are processed in chunks of
    ``chunk_sites`` (keep the default for reproducible values: the scaling
    step of the exponential is chosen per chunk); large fields are spread over
    a process pool (spawn context) of ``workers`` processes when ``workers``
    > 1, or ``None`` for up to 16 cores.  A pool re-imports the caller's main
    module in every worker, so pass ``workers`` only from a script whose main
    code sits under ``if __name__ == "__main__":`` (or from pytest).
    """
    lx, ly, lz, lt = dims
    nsite = volume(dims)
    out = np.empty((nsite, 4, 3, 3), dtype=np.complex128)
    jobs = [(s0, min(nsite, s0 + chunk_sites), eps, seed) for s0 in range(0, nsite, chunk_sites)]
    if workers is None:
        workers = min(16, len(os.sched_getaffinity(0))) if len(jobs) >= 8 else 1
    if workers > 1 and not _spawn_safe():
        workers = 1
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            for (s0, s1, _, _), blk in zip(jobs, pool.imap(_gauge_chunk, jobs)):
                out[s0:s1] = blk
    else:
        for job in jobs:
            out[job[0]:job[1]] = _gauge_chunk(job)
    return out.reshape(lt, lz, ly, lx, 4, 3, 3)


def unit_gauge_field(dims) -> np.ndarray:
    """All links equal to the identity (the free field)."""
    lx, ly, lz, lt = dims
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def spinor_field(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Gaussian complex spinor field(s): re and im parts ~ N(0, 1/2).

    Shape (T, Z, Y, X, 4, 3), or (nrhs, T, Z, Y, X, 4, 3) when ``nrhs`` is given.
    """
    lx, ly, lz, lt = dims
    n = 1 if nrhs is None else nrhs
    cnt = n * volume(dims) * 12
    g = normals(seed, 0, 2 * cnt).reshape(cnt, 2) / np.sqrt(2.0)
    psi = (g[:, 0] + 1j * g[:, 1]).reshape(n, lt, lz, ly, lx, 4, 3)
    return psi[0] if nrhs is None else psi


def point_source(dims, src, spin: int, colour: int) -> np.ndarray:
    """eta(x) = delta_{x, src} e_{spin, colour}; ``src = (x, y, z, t)``."""
    lx, ly, lz, lt = dims
    eta = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    eta[src[3], src[2], src[1], src[0], spin, colour] = 1.0
    return eta


def noise_source(dims, t0: int, seed: int, kind: str = "gauss") -> np.ndarray:
    """Stochastic source on time slice t0, zero elsewhere, shape (T, Z, Y, X, 4, 3).

    ``kind = "gauss"``: every spin-colour component of the slice complex
    Gaussian, re and im ~ N(0, 1/2) (E|eta|^2 = 1).  ``kind = "z2"``:
    (+-1 +- i)/sqrt(2) from the signs of two normals.  Either way
    E[eta_a eta_b^*] = delta_ab, so sum_x |D^-1 eta|^2 on slice t estimates
    the pion correlator summed over all source points of slice t0.
    """
    lx, ly, lz, lt = dims
    cnt = lx * ly * lz * 12
    g = normals(seed, 0, 2 * cnt).reshape(cnt, 2)
    if kind == "gauss":
        vals = (g[:, 0] + 1j * g[:, 1]) / np.sqrt(2.0)
    elif kind == "z2":
        vals = (np.sign(g[:, 0]) + 1j * np.sign(g[:, 1])) / np.sqrt(2.0)
    else:
        raise ValueError("kind must be 'gauss' or 'z2'")
    eta = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    eta[t0] = vals.reshape(lz, ly, lx, 4, 3)
    return eta


def gauge_transform(dims, seed: int, eps: float = 2.0) -> np.ndarray:
    """Random SU(3) matrix per site, g(x) = exp(i eps H(x)), shape (T, Z, Y, X, 3, 3)."""
    lx, ly, lz, lt = dims
    nsite = volume(dims)
    lam = gell_mann() / 2.0
    h = normals(seed, 0, nsite * 8).reshape(nsite, 8)
    g = expm_i_hermitian(eps * np.einsum("sa,aij->sij", h, lam))
    return g.reshape(lt, lz, ly, lx, 3, 3)


def kappa_values(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    """``count`` hopping parameters uniform in [lo, hi)."""
    return lo + (hi - lo) * uniforms(seed, 0, count)


def exponential_gaps(seed: int, count: int, rate: float) -> np.ndarray:
    """Inter-arrival gaps of a Poisson stream with the given rate (1/s)."""
    return -np.log(uniforms(seed, 0, count)) / rate
