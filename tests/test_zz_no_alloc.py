"""The allocation-free multi-dot entry point against the oracle's dot product.

rsv_mdot_noalloc serves callers that cannot allocate device memory when they
need a reduction; it keeps its scratch in a fixed device array.  This file is
named so that pytest collects it last; it must pass alone and after the
other tests (its scratch is shared by every call in the process).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsv():
    from tests.helpers import build_library
    build_library()
    import paper_1602_05901_gb300 as m
    return m


@pytest.mark.parametrize("n,k,ldv_pad", [(1_500_000, 30, 4), (12_345, 1, 0), (3 * 33 * 17 * 9, 64, 3)])
def test_mdot_noalloc_matches_oracle_twice(rsv, n, k, ldv_pad):
    import torch
    assert torch.cuda.is_available()
    ldv = n + ldv_pad
    g = torch.Generator(device="cpu").manual_seed(n + k)
    Vh = torch.randn(k * ldv, dtype=torch.float64, generator=g)
    wh = torch.randn(n, dtype=torch.float64, generator=g)
    V, w = Vh.cuda(), wh.cuda()
    Vn, wn = Vh.numpy().reshape(k, ldv)[:, :n], wh.numpy()
    ref = np.array([oracle.dot(wn, Vn[i]) for i in range(k)])
    scale = np.array([np.abs(wn * Vn[i]).sum() for i in range(k)])
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        got = np.zeros(k)
        st = rsv.rsv_mdot_noalloc(s, n, w.data_ptr(), V.data_ptr(), ldv, k, got.ctypes.data)
        assert st == rsv.RSV_OK
        assert np.all(np.abs(got - ref) <= 1e-13 * scale), np.abs(got - ref).max()


def test_mdot_noalloc_takes_no_device_memory(rsv):
    """After the first call (which may load the kernels' module), further calls leave the
    device's free memory unchanged, and the source names no allocator routine."""
    import torch
    n, k = 300_000, 16
    V = torch.randn(k * n, dtype=torch.float64, device="cuda")
    w = torch.randn(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    got = np.zeros(k)
    assert rsv.rsv_mdot_noalloc(s, n, w.data_ptr(), V.data_ptr(), n, k, got.ctypes.data) == rsv.RSV_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        assert rsv.rsv_mdot_noalloc(s, n, w.data_ptr(), V.data_ptr(), n, k, got.ctypes.data) == rsv.RSV_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    src = open(os.path.join(os.path.dirname(rsv.__file__), "csrc", "noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", src)
    assert not re.search(r"cudaMalloc|cudaFree|cudaMallocAsync|cudaFreeAsync|cudaMallocManaged|cudaMallocHost", code)


def test_mdot_noalloc_rejects_sizes_beyond_its_scratch(rsv):
    import torch
    w = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = np.zeros(65)
    s = torch.cuda.current_stream().cuda_stream
    assert rsv.rsv_mdot_noalloc(s, 16, w.data_ptr(), w.data_ptr(), 16, 65, out.ctypes.data) == rsv.RSV_EINVAL
    assert rsv.rsv_mdot_noalloc(s, 16, w.data_ptr(), w.data_ptr(), 16, 0, out.ctypes.data) == rsv.RSV_EINVAL
    assert rsv.rsv_mdot_noalloc(s, 16, w.data_ptr(), w.data_ptr(), 8, 1, out.ctypes.data) == rsv.RSV_EINVAL
