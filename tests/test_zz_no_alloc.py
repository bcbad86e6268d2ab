"""lqcd_pion_contract_noalloc: the contraction for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc: their device memory is
owned by another allocator, or their loop must not synchronize the device.
This entry point keeps its scratch in a fixed array in the library's device
image.  These tests call it through the C ABI and compare it with
lqcd_pion_contract (which allocates its scratch) on two calls in a row.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

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


def test_noalloc_contraction_matches_allocating_entry_point(lq):
    import torch
    dims = (6, 4, 8, 10)
    lat = lq.lattice_create(dims)
    lib = lq.load()
    try:
        rng = np.random.default_rng(3)
        for call, src_t in enumerate((0, 7)):  # two calls in a row, different data
            prop = rng.normal(size=(12, 10, 8, 4, 6, 4, 3)) + 1j * rng.normal(size=(12, 10, 8, 4, 6, 4, 3))
            pt = torch.from_numpy(prop).cuda()
            want = torch.zeros(10, dtype=torch.float64, device="cuda")
            lq.pion_contract(lat, pt, src_t, corr=want)
            got = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
            d = (ctypes.c_int * 4)(*dims)
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            rc = lib.lqcd_pion_contract_noalloc(d, ctypes.c_void_p(pt.data_ptr()), src_t,
                                                ctypes.c_void_p(got.data_ptr()), stream)
            assert rc == lq.OK, lq.last_error()
            torch.cuda.synchronize()
            assert np.allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=1e-13, atol=0), call
    finally:
        lq.lattice_destroy(lat)


def test_noalloc_rejects_lattices_beyond_its_scratch(lq):
    import torch
    lib = lq.load()
    dims = (64, 64, 64, 128)  # needs 786432 partial sums > 262144
    d = (ctypes.c_int * 4)(*dims)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.lqcd_pion_contract_noalloc(d, ctypes.c_void_p(dummy.data_ptr()), 0, ctypes.c_void_p(dummy.data_ptr()),
                                        None)
    assert rc == lq.EINVAL
    assert "static scratch" in lq.last_error()
