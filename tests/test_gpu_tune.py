"""Autotuner decisions exported and imported (lqcd_tune_export / _import).

A shape imported for a (format, mode, sites, nrhs) key is used on the first
launch of that key without timing candidates, reported with source
"imported", and gives the same bits as the shape the tuner picks itself (all
shapes of the FP16 hop do the same arithmetic per lane).  The export lists
it so that a restarted process can load it again.
"""
import numpy as np
import pytest

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


def test_imported_shape_is_used_and_exported(lq):
    import torch
    dims, nrhs = (6, 6, 6, 10), 7  # a key no other test tunes
    vh = int(np.prod(dims)) // 2
    lq.tune_import(f"lqcd-tune 1\nf16 0 {vh} {nrhs} -4 1 1 1\nf16 1 {vh} {nrhs} 1 7 1 1\n")
    U = inputs.gauge_field(dims, 0.4, seed=95)
    x = torch.from_numpy(inputs.spinor_field(dims, seed=96, nrhs=nrhs)).cuda()
    lat = lq.lattice_create(dims)
    try:
        gid = lq.gauge_upload(lat, U)
        dp = lq.dirac_params(0.13, 1.5)
        got = lq.schur_apply(lat, gid, dp, x, precision="fp16", nrhs=nrhs).cpu().numpy()
        ref = lq.schur_apply(lat, gid, dp, x, precision="fp64", nrhs=nrhs).cpu().numpy()
    finally:
        lq.lattice_destroy(lat)
    rows = [t for t in lq.tune_report() if t["sites"] == vh and t["nrhs"] == nrhs and t["kernel"].startswith("hop_f16")]
    assert {(t["kernel"], t["variant"], t["source"]) for t in rows} == {
        ("hop_f16_hopclov", "prefetch", "imported"), ("hop_f16_selfclov", "scalar", "imported")}
    assert f"f16 0 {vh} {nrhs} -4 1 1 1" in lq.tune_export()
    assert np.linalg.norm(got - ref) <= 4e-3 * np.linalg.norm(ref)
    # the same field on a key the tuner times itself gives the same bits
    dims2 = (6, 6, 6, 10)
    lat = lq.lattice_create(dims2)
    try:
        gid = lq.gauge_upload(lat, U)
        x8 = torch.cat([x, x[:1]]).contiguous()  # nrhs 8: a fresh key, timed
        got8 = lq.schur_apply(lat, gid, lq.dirac_params(0.13, 1.5), x8, precision="fp16", nrhs=nrhs + 1).cpu().numpy()
    finally:
        lq.lattice_destroy(lat)
    assert np.array_equal(got8[:nrhs], got)
