"""The oracle-solved golden files are what their script writes.

tests/golden/make_pion_golden.py calls only the FP64 oracle; these checks
keep the stored files tied to it: the 4^4 file is re-derived from the oracle
here, and both files must be internally consistent (C(t) is the sum of the
per-column sums, every column converged to the oracle's 1e-13).
"""
import json
import os

import numpy as np

import oracle
from paper_2503_16994_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def test_golden_files_are_consistent():
    for name in ("pion_4c4_seed1.json", "pion_16c32_seed1.json"):
        d = load(name)
        T = d["config"]["dims"][3]
        col = np.asarray(d["corr_col"])
        assert col.shape == (12, T)
        assert np.allclose(col.sum(axis=0), d["corr"], rtol=1e-14, atol=0)
        assert np.all(np.asarray(d["corr"]) > 0)
        assert max(d["resid"]) <= 1e-13
        assert d["config"]["theta"] == [1.0, 1.0, 1.0, -1.0]
        vals = np.asarray(d["samples"]["values"])
        assert vals.shape == (12, len(d["samples"]["sites"]), 12, 2)


def test_small_golden_rederived_from_the_oracle():
    d = load("pion_4c4_seed1.json")
    c = d["config"]
    dims = tuple(c["dims"])
    U = inputs.gauge_field(dims, c["eps"], seed=c["seed"])
    corr, prop, iters, res, failed = oracle.pion(dims, U, c["kappa"], c["csw"], tuple(c["src"]), tol=c["tol"],
                                                 want_prop=True)
    assert failed == 0
    assert np.allclose(corr, d["corr"], rtol=1e-12, atol=0)
    vals = np.asarray(d["samples"]["values"])
    for j in range(12):
        for k, s in enumerate(d["samples"]["sites"]):
            got = prop[j, s[3], s[2], s[1], s[0]].reshape(12)
            want = vals[j, k, :, 0] + 1j * vals[j, k, :, 1]
            assert np.allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))
