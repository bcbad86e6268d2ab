"""Host-side checks of the C ABI that need no GPU.

The library must load, export every function that include/lqcd.h declares,
and reject bad arguments before touching the device.
"""
import ctypes
import os
import re

import pytest

from paper_2503_16994_gb300 import build as lqcd_build
from paper_2503_16994_gb300 import lqcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lqcd_build.build()
    return lqcd.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["lqcd_lattice_create", "lqcd_gauge_upload", "lqcd_dirac_apply", "lqcd_cg_solve",
                     "lqcd_pion_corr", "lqcd_serve_submit", "lqcd_serve_poll"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lqcd.abi_version() == 3


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 5), (0, 4, 4, 4), (4, 4, -2, 4)])
def test_lattice_create_rejects_bad_extents(lib, dims):
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lattice_create(dims)
    assert e.value.code == lqcd.EINVAL
    assert "even" in str(e.value)


def test_null_arguments_are_rejected(lib):
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.lqcd_lattice_create(d, 0, None) == lqcd.EINVAL
    assert lib.lqcd_lattice_create(None, 0, ctypes.byref(ctypes.c_void_p())) == lqcd.EINVAL
    assert lib.lqcd_gauge_upload(None, None, None) == lqcd.EINVAL
    assert lib.lqcd_dirac_apply(None, 0, None, None, None, 0, None) == lqcd.EINVAL
    assert lib.lqcd_cg_solve(None, 0, None, None, None, None, 1, None, 0, None) == lqcd.EINVAL
    assert lib.lqcd_pion_corr(None, 0, None, None, None, None, None, None, 0, None) == lqcd.EINVAL
    assert lib.lqcd_pion_contract(None, None, 0, None, 0, None) == lqcd.EINVAL
    assert lib.lqcd_meson_contract(None, None, 0, None, 1, None, 0, None) == lqcd.EINVAL
    assert lqcd.last_error() != ""
    assert lib.lqcd_lattice_destroy(None) == lqcd.OK


def test_no_device_is_an_error_not_a_crash(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a CUDA device is present")
    except ImportError:
        pass
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lattice_create((4, 4, 4, 4), device=0)
    assert e.value.code == lqcd.ECUDA


def test_tune_import_validates_before_loading(lib):
    # host-only: the tuner's table of shapes is read and checked without a GPU
    good = "lqcd-tune 1\nf16 0 331776 12 12 3 3 1\nf16 1 331776 12 0 2 4 8\nf64 0 331776 12 1 2 1 1\n"
    bad = [
        "f16 0 331776 12 12 3 3 1\n",                       # no header
        "lqcd-tune 2\nf16 0 331776 12 12 3 3 1\n",           # unknown version
        "lqcd-tune 1\nf16 0 331776 12 12 3 3\n",             # a field missing
        "lqcd-tune 1\nf16 0 331776 12 12 3 3 1 7\n",         # a field too many
        "lqcd-tune 1\nf64 0 331776 12 0 2 3 1\n",            # paired shape for FP64
        "lqcd-tune 1\nf32 1 331776 12 12 3 3 1\n",           # staged shape for FP32
        "lqcd-tune 1\nf16 2 331776 12 1 1 1 1\n",            # no such mode
        "lqcd-tune 1\nf16 0 331776 12 21 9 3 1\n",           # tile kernel with 9 pairs per block
        "lqcd-tune 1\nf16 0 331776 12 1 1 5 1\n",            # no such register cap
        "lqcd-tune 1\nbf16 0 331776 12 1 1 1 1\n",           # unknown format
        good + "f16 0 -4 12 1 1 1 1\n",                      # one bad line spoils the whole text
    ]
    before = lqcd.tune_export()
    assert before.startswith("lqcd-tune 1\n")
    for text in bad:
        with pytest.raises(lqcd.LqcdError) as e:
            lqcd.tune_import(text)
        assert e.value.code == lqcd.EINVAL, text
    assert lqcd.tune_export() == before  # nothing was loaded
    lqcd.tune_import(good)
    # imported shapes are used (and reported) on the first launch of their key only
    assert lqcd.tune_export() == before
    assert lib.lqcd_tune_import(None) == lqcd.EINVAL


def test_every_entry_point_checks_its_arguments_before_the_device(lib):
    """The remaining entry points: null handles, buffers and counts, and the
    ranges checked before any device work, return LQCD_EINVAL (and destroying
    a null server is a no-op) with no GPU present."""
    import numpy as np
    E = lqcd.EINVAL
    dp = lqcd.dirac_params(0.12, 1.0)
    sp = lqcd.solver_params(tol=1e-10, maxiter=10)
    info = (lqcd.SolveInfo * 12)()
    buf = np.zeros(64)
    p = ctypes.c_void_p(buf.ctypes.data)
    d4 = (ctypes.c_int * 4)(4, 4, 4, 4)
    calls = {
        "schur_apply": lambda: lib.lqcd_schur_apply(None, 0, ctypes.byref(dp), 0, None, None, 1, 1, 0, None),
        "gauge_free": lambda: lib.lqcd_gauge_free(None, 0),
        "boundary_corr": lambda: lib.lqcd_boundary_corr(None, 0, ctypes.byref(dp), ctypes.byref(sp), None, None,
                                                        None, info, 0, None),
        "gauge_flow": lambda: lib.lqcd_gauge_flow(None, 0, 0.01, 1, None),
        "fermion_flow": lambda: lib.lqcd_fermion_flow(None, 0, ctypes.byref(dp), None, 1, 0.01, 1, 0, None),
        "fermion_backflow": lambda: lib.lqcd_fermion_backflow(None, 0, ctypes.byref(dp), None, 1, 0.01, 1, 1, 0,
                                                              None),
        "gauge_observables": lambda: lib.lqcd_gauge_observables(None, 0, None, None, None, None, None),
        "hmc_trajectory": lambda: lib.lqcd_hmc_trajectory(None, 0, 6.0, 0.1, 5, None, 0.5, None, None, None),
        "gauge_download": lambda: lib.lqcd_gauge_download(None, 0, None, 0, None),
        "pion_corr_batch (no jobs)": lambda: lib.lqcd_pion_corr_batch(None, 1, ctypes.byref(sp), 0, None),
        "pion_corr_batch (njobs 0)": lambda: lib.lqcd_pion_corr_batch((lqcd.PionJob * 1)(), 0, ctypes.byref(sp), 0,
                                                                       None),
        "pion_corr_batch (chunk)": lambda: lib.lqcd_pion_corr_batch((lqcd.PionJob * 1)(), 1, ctypes.byref(sp), -1,
                                                                     None),
        "noalloc (null)": lambda: lib.lqcd_pion_contract_noalloc(None, p, 0, p, None),
        "noalloc (extent 0)": lambda: lib.lqcd_pion_contract_noalloc((ctypes.c_int * 4)(4, 0, 4, 4), p, 0, p, None),
        "noalloc (source time)": lambda: lib.lqcd_pion_contract_noalloc(d4, p, 4, p, None),
        "noalloc (too large)": lambda: lib.lqcd_pion_contract_noalloc((ctypes.c_int * 4)(2, 2, 2, 1 << 20), p, 0,
                                                                       p, None),
        "serve_create (null)": lambda: lib.lqcd_serve_create(0, 1 << 30, 4, None),
        "serve_create (slots)": lambda: lib.lqcd_serve_create(0, 1 << 30, 0, ctypes.byref(ctypes.c_void_p())),
        "serve_gauge": lambda: lib.lqcd_serve_gauge(None, d4, p, ctypes.byref(ctypes.c_int())),
        "serve_submit": lambda: lib.lqcd_serve_submit(None, 0, ctypes.byref(dp), ctypes.byref(sp), d4,
                                                      ctypes.byref(ctypes.c_uint64())),
        "serve_poll": lambda: lib.lqcd_serve_poll(None, 1, None, None, None, 0),
        "profile_read": lambda: lib.lqcd_profile_read(None, 0, None),
        "profile_read (no out)": lambda: lib.lqcd_profile_read(None, 4, ctypes.byref(ctypes.c_int())),
        "tune_report": lambda: lib.lqcd_tune_report(None, 16),
        "tune_export (len 0)": lambda: lib.lqcd_tune_export(ctypes.create_string_buffer(4), 0),
    }
    for name, call in calls.items():
        assert call() == E, name
        assert lqcd.last_error() != "", name
    assert lib.lqcd_serve_destroy(None) == lqcd.OK
