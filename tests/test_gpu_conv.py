"""Tensor-core convolutions (forward, input gradient, weight gradient) against the FP64 oracle.

Both sides use the same BF16 operands; the GPU accumulates exact BF16
products in FP32, so the bound used is the classical one for a recursive FP32
sum of K terms, |err| <= K * 2^-24 * sum|terms| (doubled for margin), taken
element by element from the oracle's sum of absolute products.
"""
import ctypes

import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rsv():
    import paper_1602_05901_gb300 as rsv
    return rsv


def _bf16(torch, a):
    """(device BF16 tensor, the same values as float64 numpy)."""
    t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float32).to(torch.bfloat16)
    return t.cuda(), t.float().double().numpy()


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _vol(rng, nz, ny, nx, c, ld=None, scale=1.0):
    ld = ld or c
    a = np.zeros((nz, ny, nx, ld))
    a[..., :c] = rng.standard_normal((nz, ny, nx, c)) * scale
    return a


FWD_CASES = [
    # (nx, ny, nz, taps, ci, co, ldx, relu, bias)
    (16, 8, 4, 1, 64, 32, 64, False, False),      # plain GEMM, 4 tiles
    (20, 12, 6, 27, 32, 32, 40, False, False),    # BK = 32, ragged tiles (120 of 128 rows used), ldx > ci
    (16, 16, 8, 27, 128, 256, 128, True, True),   # coarsest U-Net level, BN = 256
    (8, 8, 4, 27, 384, 128, 384, True, True),     # concatenated input, 3 K blocks of 128
    (32, 8, 5, 27, 64, 96, 64, True, True),       # BN = 96, ragged z
    (24, 4, 3, 27, 96, 192, 104, False, True),    # ci = 96 (BK = 32), BN = 192, ragged x tiles
]


@pytest.mark.parametrize("case", FWD_CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}_t{c[3]}_ci{c[4]}_co{c[5]}" for c in FWD_CASES])
def test_conv_fwd_matches_oracle(rsv, case):
    torch = pytest.importorskip("torch")
    nx, ny, nz, taps, ci, co, ldx, relu, use_bias = case
    rng = np.random.default_rng(sum(case[:6]))
    xt, xh = _bf16(torch, _vol(rng, nz, ny, nx, ci, ldx))
    w = rng.standard_normal((co, taps, ci)) * np.sqrt(2.0 / (taps * ci))
    wt, wh = _bf16(torch, w)
    bias = rng.standard_normal(co).astype(np.float32) * 0.1 if use_bias else None
    bt = torch.tensor(bias).cuda() if use_bias else None
    y32 = torch.full((nz * ny * nx, co), float("nan"), device="cuda")
    ldy = co + 32
    yb = torch.zeros((nz * ny * nx, ldy), dtype=torch.bfloat16, device="cuda")
    st = rsv.rsv_conv3d_fwd(None, nx, ny, nz, taps, ci, co, _p(xt), ldx, _p(wt), _p(bt), int(relu), None, 0,
                            ctypes.c_void_p(yb.data_ptr() + 64), ldy, _p(y32))
    assert st == rsv.RSV_OK, rsv.status_string(st)
    x = xh[..., :ci]
    if taps == 27:
        ref = U.conv3(x, wh)
        absref = U.conv3(np.abs(x), np.abs(wh))
    else:
        ref = x @ wh[:, 0, :].T
        absref = np.abs(x) @ np.abs(wh[:, 0, :]).T
    if use_bias:
        ref = ref + bias
        absref = absref + np.abs(bias)
    if relu:
        ref = np.maximum(ref, 0)
    got = y32.cpu().double().numpy().reshape(ref.shape)
    tol = 2 * (taps * ci + 1) * U32 * absref + 1e-30
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
    # BF16 output: the round-to-nearest of the FP32 result, at channel offset 32 of rows of ldy
    gb = yb.float().cpu().double().numpy().reshape(nz, ny, nx, ldy)[..., 32:32 + co]
    assert np.array_equal(gb, U.bf16_round(got))
    assert np.all(yb.float().cpu().numpy().reshape(nz, ny, nx, ldy)[..., :32] == 0)


def test_conv_dgrad_with_relu_mask(rsv):
    torch = pytest.importorskip("torch")
    nx, ny, nz, ci, co = 16, 8, 4, 96, 32
    rng = np.random.default_rng(5)
    gyt, gyh = _bf16(torch, _vol(rng, nz, ny, nx, co))
    w = rng.standard_normal((co, 27, ci)) * 0.1
    wt, wh = _bf16(torch, w)
    mask = rng.standard_normal((nz, ny, nx, ci))
    mt, mh = _bf16(torch, mask)
    gx32 = torch.full((nz * ny * nx, ci), float("nan"), device="cuda")
    st = rsv.rsv_conv3d_dgrad(None, nx, ny, nz, ci, co, _p(gyt), co, _p(wt), _p(mt), ci, None, 0, _p(gx32))
    assert st == rsv.RSV_OK, rsv.status_string(st)
    ref = U.conv3_dgrad(gyh, wh) * (mh > 0)
    absref = U.conv3_dgrad(np.abs(gyh), np.abs(wh))
    got = gx32.cpu().double().numpy().reshape(ref.shape)
    assert np.all(np.abs(got - ref) <= 2 * 27 * co * U32 * absref + 1e-30)
    assert np.all(got[mh <= 0] == 0)


WG_CASES = [
    # (nx, ny, nz, taps, ci, co)
    (16, 8, 6, 27, 32, 32),
    (8, 8, 4, 27, 96, 32),
    (16, 4, 4, 1, 64, 32),
    (16, 16, 8, 27, 128, 256),
    (24, 5, 3, 27, 64, 96),      # no 64-voxel box fits: the voxel-major copy path
    (16, 8, 8, 27, 192, 64),     # ci > co: rows = (tap, output channel), N = 192
    (16, 8, 4, 27, 384, 128),    # ci > co: two N tiles of 192
    (32, 4, 3, 27, 96, 32),      # ci > co with ragged z chunks
]


@pytest.mark.parametrize("case", WG_CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}_t{c[3]}_ci{c[4]}_co{c[5]}" for c in WG_CASES])
def test_conv_wgrad_matches_oracle(rsv, case):
    torch = pytest.importorskip("torch")
    nx, ny, nz, taps, ci, co = case
    rng = np.random.default_rng(100 + sum(case))
    ldx = ci + 8
    xt, xh = _bf16(torch, _vol(rng, nz, ny, nx, ci, ldx))
    gyt, gyh = _bf16(torch, _vol(rng, nz, ny, nx, co))
    gw = torch.full((co, taps, ci), float("nan"), device="cuda")
    gb = torch.full((co,), float("nan"), device="cuda")
    st = rsv.rsv_conv3d_wgrad(None, nx, ny, nz, taps, ci, co, _p(xt), ldx, _p(gyt), co, _p(gw), _p(gb))
    assert st == rsv.RSV_OK, rsv.status_string(st)
    x = xh[..., :ci]
    if taps == 27:
        ref, absref = U.conv3_wgrad(gyh, x), U.conv3_wgrad(np.abs(gyh), np.abs(x))
    else:
        ref = (gyh.reshape(-1, co).T @ x.reshape(-1, ci))[:, None, :]
        absref = (np.abs(gyh).reshape(-1, co).T @ np.abs(x).reshape(-1, ci))[:, None, :]
    nvox = nx * ny * nz
    got = gw.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= 2 * nvox * U32 * absref + 1e-30), np.nanmax(np.abs(got - ref) / absref)
    gbr = gyh.reshape(-1, co).sum(axis=0)
    assert np.allclose(gb.cpu().double().numpy(), gbr, rtol=0, atol=2 * nvox * U32 * np.abs(gyh).reshape(-1, co).sum(0).max())


def test_conv_argument_checks(rsv):
    torch = pytest.importorskip("torch")
    x = torch.zeros(64 * 40, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(32 * 40, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(64 * 32, dtype=torch.float32, device="cuda")
    # ci not a multiple of 32, taps not 1 or 27, misaligned leading dimension
    assert rsv.rsv_conv3d_fwd(None, 4, 4, 4, 1, 40, 32, _p(x), 40, _p(w), None, 0, None, 0, None, 0, _p(y)) == rsv.RSV_EINVAL
    assert rsv.rsv_conv3d_fwd(None, 4, 4, 4, 9, 32, 32, _p(x), 32, _p(w), None, 0, None, 0, None, 0, _p(y)) == rsv.RSV_EINVAL
    assert rsv.rsv_conv3d_fwd(None, 4, 4, 4, 1, 32, 32, _p(x), 36, _p(w), None, 0, None, 0, None, 0, _p(y)) == rsv.RSV_EINVAL
    assert rsv.rsv_conv3d_wgrad(None, 6, 4, 4, 27, 32, 32, _p(x), 32, _p(x), 32, _p(y), None) == rsv.RSV_EINVAL
