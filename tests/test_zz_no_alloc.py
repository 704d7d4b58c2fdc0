"""The allocation-free multi-dot entry point against the allocating rsv_dot.

rsv_mdot_noalloc serves callers that cannot allocate device memory when they
need a reduction; it keeps its scratch in a fixed device array.  This file is
named so that pytest collects it last; it must pass alone and after the
other tests (its scratch is shared by every call in the process).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsv():
    from tests.helpers import build_library
    build_library()
    import paper_1602_05901_gb300 as m
    return m


def _dots_with_rsv_dot(rsv, torch, n, w, V, ldv, k):
    s = torch.cuda.current_stream().cuda_stream
    out = np.zeros(k)
    val = ctypes.c_double()
    for i in range(k):
        assert rsv.rsv_dot(s, n, w.data_ptr(), V.data_ptr() + 8 * i * ldv, ctypes.byref(val)) == rsv.RSV_OK
        out[i] = val.value
    return out


@pytest.mark.parametrize("n,k,ldv_pad", [(1_500_000, 30, 4), (12_345, 1, 0), (3 * 33 * 17 * 9, 64, 3)])
def test_mdot_noalloc_matches_rsv_dot_twice(rsv, n, k, ldv_pad):
    import torch
    assert torch.cuda.is_available()
    ldv = n + ldv_pad
    g = torch.Generator(device="cpu").manual_seed(n + k)
    V = torch.randn(k * ldv, dtype=torch.float64, generator=g).cuda()
    w = torch.randn(n, dtype=torch.float64, generator=g).cuda()
    ref = _dots_with_rsv_dot(rsv, torch, n, w, V, ldv, k)
    s = torch.cuda.current_stream().cuda_stream
    scale = (w.abs().double().sum() * V.view(k, ldv)[:, :n].abs().amax(dim=1)).cpu().numpy()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        got = np.zeros(k)
        st = rsv.rsv_mdot_noalloc(s, n, w.data_ptr(), V.data_ptr(), ldv, k, got.ctypes.data)
        assert st == rsv.RSV_OK
        assert np.all(np.abs(got - ref) <= 1e-13 * scale), np.abs(got - ref).max()


def test_mdot_noalloc_rejects_sizes_beyond_its_scratch(rsv):
    import torch
    w = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = np.zeros(65)
    s = torch.cuda.current_stream().cuda_stream
    assert rsv.rsv_mdot_noalloc(s, 16, w.data_ptr(), w.data_ptr(), 16, 65, out.ctypes.data) == rsv.RSV_EINVAL
    assert rsv.rsv_mdot_noalloc(s, 16, w.data_ptr(), w.data_ptr(), 16, 0, out.ctypes.data) == rsv.RSV_EINVAL
    assert rsv.rsv_mdot_noalloc(s, 16, w.data_ptr(), w.data_ptr(), 8, 1, out.ctypes.data) == rsv.RSV_EINVAL
