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
