"""Pins of the learned-stage oracle (oracle/unet.py) against facts fixed outside it.

Each test fails on a plausible slip in the oracle: a flipped tap offset, a
transposed weight, a missing 1/8 in the pooling adjoint, a dropped gradient
path through a skip connection, a wrong bias correction in Adam.
"""
import numpy as np
import pytest

from oracle import unet as U


def _rng(seed):
    return np.random.default_rng(seed)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([_rng(0).standard_normal(4000) * 10.0 ** _rng(1).integers(-20, 20, 4000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(x), ref)
    assert U.bf16_round(1.0 + 2.0 ** -8) == 1.0          # a tie rounds to even
    assert U.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_conv3_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    x = _rng(2).standard_normal((5, 6, 7, 3))
    w = _rng(3).standard_normal((4, 27, 3))
    b = _rng(4).standard_normal(4)
    y = U.conv3(x, w, b)
    for co in range(4):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[co, :, ci].reshape(3, 3, 3)   # k[dz+1, dy+1, dx+1]
            ref += ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        assert np.allclose(y[..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv3_identity_kernel_and_delta_input():
    x = _rng(5).standard_normal((4, 4, 4, 2))
    w = np.zeros((2, 27, 2))
    w[0, 13, 0] = w[1, 13, 1] = 1.0            # centre tap (0,0,0) is t = 13
    assert np.array_equal(U.conv3(x, w), x)
    # a delta at p gives y[p - off_t] = w[t]: the cross-correlation reads x[v + off_t]
    w = _rng(6).standard_normal((1, 27, 1))
    d = np.zeros((5, 5, 5, 1))
    d[2, 2, 2, 0] = 1.0
    y = U.conv3(d, w)
    for t, (dz, dy, dx) in enumerate(U.TAPS):
        assert y[2 - dz, 2 - dy, 2 - dx, 0] == w[0, t, 0]
    assert np.count_nonzero(y) == 27


def test_dgrad_wgrad_are_adjoints():
    x = _rng(7).standard_normal((4, 5, 6, 3))
    w = _rng(8).standard_normal((2, 27, 3))
    g = _rng(9).standard_normal((4, 5, 6, 2))
    lhs = np.sum(g * U.conv3(x, w))
    assert np.isclose(np.sum(U.conv3_dgrad(g, w) * x), lhs, rtol=1e-12)
    assert np.isclose(np.sum(U.conv3_wgrad(g, x) * w), lhs, rtol=1e-12)


def test_conv_gradients_by_finite_differences():
    x = _rng(10).standard_normal((3, 4, 3, 2))
    w = _rng(11).standard_normal((2, 27, 2))
    g = _rng(12).standard_normal((3, 4, 3, 2))
    f = lambda x_, w_: np.sum(g * U.conv3(x_, w_))
    gw, gx = U.conv3_wgrad(g, x), U.conv3_dgrad(g, w)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 13, 1), (0, 26, 1), (1, 4, 0)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert np.isclose((f(x, w + e) - f(x, w - e)) / (2 * h), gw[idx], rtol=1e-7, atol=1e-8)
    for idx in [(0, 0, 0, 0), (2, 3, 2, 1), (1, 2, 0, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert np.isclose((f(x + e, w) - f(x - e, w)) / (2 * h), gx[idx], rtol=1e-7, atol=1e-8)


def test_pool_and_upsample_adjoints():
    x = _rng(13).standard_normal((4, 6, 8, 3))
    gc = _rng(14).standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(U.avgpool2(x) * gc), np.sum(x * U.avgpool2_bwd(gc)), rtol=1e-13)
    assert np.isclose(np.sum(U.upsample2(gc) * x), np.sum(gc * U.upsample2_bwd(x)), rtol=1e-13)
    assert np.allclose(U.avgpool2(U.upsample2(gc)), gc, rtol=0, atol=1e-15)
    assert np.isclose(U.avgpool2(x)[1, 2, 3, 0], x[2:4, 4:6, 6:8, 0].mean())


def test_layer_shapes():
    s = U.layer_shapes()
    assert [n for n, *_ in s] == ["enc1a", "enc1b", "enc2a", "enc2b", "enc3a", "enc3b", "enc4a", "enc4b",
                                  "dec3a", "dec3b", "dec2a", "dec2b", "dec1a", "dec1b", "head"]
    d = {n: (co, ci) for n, co, ci, _ in s}
    assert d["enc1a"] == (32, 2) and d["enc4b"] == (256, 256) and d["dec3a"] == (128, 384)
    assert d["dec1a"] == (32, 96) and d["head"] == (1, 32)


def _params(base, levels, seed):
    r = _rng(seed)
    p = {}
    for n, co, ci, taps in U.layer_shapes(base, levels):
        if taps == 27:
            p[n] = (r.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci)), r.standard_normal(co) * 0.1)
        else:
            p[n] = (r.standard_normal((co, ci)) * 0.5, r.standard_normal(co) * 0.1)
    return p


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_unet_gradient_by_finite_differences(levels):
    base = 2
    p = _params(base, levels, 20 + levels)
    x = _rng(15).standard_normal((8, 8, 8, 2))
    tgt = _rng(16).standard_normal((8, 8, 8))

    def loss(pp):
        out, _ = U.forward(pp, x, base, levels)
        return U.mse_loss(out, tgt)[0]

    out, act = U.forward(p, x, base, levels)
    _, gout = U.mse_loss(out, tgt)
    grads = U.backward(p, act, gout, base, levels)
    assert set(grads) == set(p)
    h = 1e-6
    r = _rng(17)
    for name, (w, b) in p.items():
        for which, arr in ((0, w), (1, b)):
            for _ in range(2):
                idx = tuple(int(r.integers(0, s)) for s in arr.shape)
                q = {k: (v[0].copy(), v[1].copy()) for k, v in p.items()}
                q[name][which][idx] += h
                fp = loss(q)
                q[name][which][idx] -= 2 * h
                fm = loss(q)
                fd = (fp - fm) / (2 * h)
                an = grads[name][which][idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (name, which, idx, fd, an)


def test_unet_bf16_mode_rounds_activations():
    p = _params(2, 2, 30)
    x = _rng(18).standard_normal((8, 8, 8, 2))
    out64, _ = U.forward(p, x, 2, 2)
    out16, act = U.forward(p, x, 2, 2, bf16=True)
    for k in ("in", "enc1a", "enc2b", "dec1b", "pool1"):
        assert np.array_equal(act[k], U.bf16_round(act[k]))
    rel = np.linalg.norm(out16 - out64) / np.linalg.norm(out64)
    assert 0 < rel < 5e-2


def test_adam_first_step_closed_form():
    g = np.array([3.0, -1e-3, 0.25, -7.0])
    w = np.ones(4)
    w1, m, v = U.adam_step(w, g, np.zeros(4), np.zeros(4), 1, lr=1e-3)
    # at t = 1 the bias-corrected moments are g and g^2, so the step is lr * g / (|g| + eps)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_standardise():
    rp = _rng(19).standard_normal((2, 4, 4)) * 7.0
    lnk = _rng(20).standard_normal((2, 4, 4)) * 2.0 + 3.0
    x, s = U.standardise(rp, lnk)
    assert np.isclose(s, np.sqrt(np.mean(rp ** 2)))
    assert np.isclose(np.mean(x[..., 0] ** 2), 1.0)
    assert np.isclose(x[..., 1].mean(), 0.0, atol=1e-14) and np.isclose(x[..., 1].std(), 1.0)
    assert np.all(U.apply_stage(_params(2, 1, 1), np.zeros((2, 4, 4)), lnk, 2, 1) == 0)


def test_learned_cpr_with_zero_network_is_block_ilu0():
    """A network whose output is zero leaves only CPR's second stage: block ILU(0) of f."""
    import oracle as O
    import synth
    nx, ny, nz = 8, 4, 2
    p = synth.make_problem(nx, ny, nz, seed=2)
    params = {n: (np.zeros((co, 27, ci) if t == 27 else (co, ci)), np.zeros(co)) for n, co, ci, t in U.layer_shapes(2, 2)}
    f = np.random.default_rng(3).standard_normal(3 * p.nb)
    z = U.learned_cpr_apply(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, params, p.lnk, f, base=2, levels=2, bf16=False)
    st, lu, udinv, _ = O.bilu0_setup(p.row_ptr, p.col_idx, p.vals)
    assert np.array_equal(z, 0.0 + O.bilu0_apply(p.row_ptr, p.col_idx, lu, udinv, f))
