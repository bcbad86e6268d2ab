"""Writes an oracle-solved point-source propagator summary as a golden file.

TEST INFRASTRUCTURE: this script calls only the FP64 CPU oracle (``oracle/``)
and the seeded input generators; nothing here comes from the CUDA path.

For one lattice it builds the synthetic gauge field U = exp(i eps H) (seeded),
solves the 12 point-source columns D x_j = eta_j (eta_j(x) = delta_{x,src} e_j,
j = 3 spin + colour) with the oracle's unpreconditioned CGNR to a true
relative residual ``tol`` (Sec. 3.3, CG! and propagator!), and stores

* ``corr``: the pion correlator C(t) = sum_xvec sum_j |S_j(xvec, src_t + t)|^2;
* ``corr_col``: the same per column j (C is their sum);
* ``x_norm2``: |x_j|^2 per column;
* ``iters`` and ``resid``: the oracle's iteration counts and true residuals;
* ``samples``: the 12 spinor components of every column at a few sites
  (the source, its neighbours, a far site and seeded random sites).

Columns are solved in parallel by worker processes (started with ``spawn``).
Usage (16^3 x 32, eps 0.4, kappa 0.130, csw 1.5, seed 1, source at the origin):

    python tests/golden/make_pion_golden.py --dims 16 16 16 32 --eps 0.4 \
        --kappa 0.130 --csw 1.5 --seed 1 --out tests/golden/pion_16c32_seed1.json
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)


def sample_sites(dims, src, seed, n_random):
    """The source, its 8 neighbours, the farthest site and n_random seeded sites."""
    from paper_2503_16994_gb300 import inputs

    L = list(dims)
    out = [list(src)]
    for mu in range(4):
        for d in (+1, -1):
            y = list(src)
            y[mu] = (y[mu] + d) % L[mu]
            out.append(y)
    out.append([(src[mu] + L[mu] // 2) % L[mu] for mu in range(4)])
    u = inputs.uniforms(seed, 0, 4 * n_random).reshape(n_random, 4)
    for k in range(n_random):
        out.append([int(u[k, mu] * L[mu]) for mu in range(4)])
    return out


def _solve_column(args):
    dims, eps, seed, kappa, csw, theta, src, tol, maxiter, j, sites = args
    import oracle
    from paper_2503_16994_gb300 import inputs

    U = inputs.gauge_field(dims, eps, seed=seed)
    b = inputs.point_source(dims, src, j // 3, j % 3)
    t0 = time.time()
    x, it, res, ok = oracle.cgnr(dims, U, kappa, csw, b, theta=theta, tol=tol, maxiter=maxiter)
    lx, ly, lz, lt = dims
    xs = x.reshape(lt, lz, ly, lx, 12)
    per_t = np.sum(np.abs(xs) ** 2, axis=(1, 2, 3, 4))
    corr_col = np.roll(per_t, -src[3])  # t counted from the source slice
    vals = [[[float(v.real), float(v.imag)] for v in xs[s[3], s[2], s[1], s[0]]] for s in sites]
    return dict(j=j, corr_col=corr_col.tolist(), x_norm2=float(np.sum(np.abs(x) ** 2)), iters=int(it),
                resid=float(res), ok=bool(ok), values=vals, seconds=time.time() - t0)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--eps", type=float, default=0.4)
    ap.add_argument("--kappa", type=float, default=0.130)
    ap.add_argument("--csw", type=float, default=1.5)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--src", type=int, nargs=4, default=[0, 0, 0, 0])
    ap.add_argument("--tol", type=float, default=1e-13)
    ap.add_argument("--maxiter", type=int, default=20000)
    ap.add_argument("--random-sites", type=int, default=6)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    theta = [1.0, 1.0, 1.0, -1.0]
    sites = sample_sites(a.dims, a.src, a.seed + 1000, a.random_sites)
    jobs = [(a.dims, a.eps, a.seed, a.kappa, a.csw, theta, a.src, a.tol, a.maxiter, j, sites) for j in range(12)]
    workers = a.workers or min(12, os.cpu_count() or 1)
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool:
        cols = sorted(pool.map(_solve_column, jobs), key=lambda c: c["j"])
    if not all(c["ok"] for c in cols):
        raise SystemExit("oracle CGNR did not converge for some column")
    corr = np.sum(np.array([c["corr_col"] for c in cols]), axis=0)
    doc = {
        "what": "oracle-solved 12-column point-source propagator and pion C(t)",
        "written_by": "tests/golden/make_pion_golden.py (FP64 CPU oracle, unpreconditioned CGNR)",
        "config": {"dims": a.dims, "eps": a.eps, "seed": a.seed, "kappa": a.kappa, "csw": a.csw,
                   "theta": theta, "src": a.src, "tol": a.tol},
        "corr": corr.tolist(),
        "corr_col": [c["corr_col"] for c in cols],
        "x_norm2": [c["x_norm2"] for c in cols],
        "iters": [c["iters"] for c in cols],
        "resid": [c["resid"] for c in cols],
        "samples": {"sites": sites, "values": [c["values"] for c in cols]},
        "wall_seconds": round(time.time() - t0, 1),
    }
    with open(a.out, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"wrote {a.out}: iters {doc['iters']}, max resid {max(doc['resid']):.2e}, {doc['wall_seconds']} s")


if __name__ == "__main__":
    main()
