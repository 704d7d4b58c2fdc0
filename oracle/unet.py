"""CPU oracle of the learned pressure stage (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this module; the CUDA library never imports or falls back to it, and the two
share no code.

What it computes: a 3-D convolutional U-Net that maps the pressure residual
of the CPR pressure stage and the log-permeability to a pressure correction.
The paper's CPR preconditioner (Section "CPR", two-stage form) leaves the
pressure-stage solver open ("any AMG solver", Section "AMG"); the learned
stage replaces that solver by a network trained to imitate one V-cycle.
Architecture, precision and training follow the task's fixed reading:

* 4 levels with 32/64/128/256 channels; two (3x3x3 conv + bias + ReLU) per
  level; 2x2x2 average pooling down; nearest upsampling and concatenation
  ``[upsampled, skip]`` up; a final 1x1x1 conv to one channel; no
  normalisation layers.
* Inputs ``r_p / s`` with ``s = rms(r_p)`` and standardised ``ln k``; the
  output is multiplied back by ``s``.  Loss: mean squared error against the
  V-cycle correction scaled by the same ``s``.  Adam.
* Activations and conv weights in BF16, products accumulated exactly into
  FP32 sums, bias in FP32.  ``bf16=True`` rounds at exactly the points where
  the GPU stores a BF16 tensor, so both sides see the same operands; with
  ``bf16=False`` everything is FP64 (used by the finite-difference pins).

Layout: a volume is ``[D, H, W, C]`` (channels last) with D = nz, H = ny,
W = nx, so voxel ``(k, j, i)`` is grid cell ``c = nx*ny*k + nx*j + i``.  A
3x3x3 weight is ``w[co, t, ci]`` with tap ``t = 9*(dz+1) + 3*(dy+1) +
(dx+1)``, and the layer computes the cross-correlation
``y[z,y,x,co] = b[co] + sum_t sum_ci w[co,t,ci] * x[z+dz, y+dy, x+dx, ci]``
with zeros outside the grid.

Parity status (pins in ``tests/test_oracle_unet.py``): conv forward against
scipy's n-D correlation, identity kernel and delta input; dgrad and wgrad as
exact adjoints and by finite differences; pooling/upsampling adjoints; the
whole network's gradient by finite differences; BF16 rounding against
PyTorch's conversion; the Adam step against its closed form at step 1.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64.

    The value is first rounded to FP32 (the GPU's accumulator type), then its
    low 16 mantissa bits are rounded away.  NaN and overflow are not handled
    (the network never produces them on valid inputs).
    """
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(a, on):
    return bf16_round(a) if on else a


def shifted(x, dz, dy, dx):
    """s[z, y, x] = x[z+dz, y+dy, x+dx], zero where that index is outside."""
    D, H, W = x.shape[:3]
    s = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), min(D, D - dz)), slice(max(0, -dy), min(H, H - dy)), slice(max(0, -dx), min(W, W - dx))
    zt, yt, xt = slice(max(0, dz), min(D, D + dz)), slice(max(0, dy), min(H, H + dy)), slice(max(0, dx), min(W, W + dx))
    s[zs, ys, xs] = x[zt, yt, xt]
    return s


def conv3(x, w, b=None):
    """3x3x3 cross-correlation with zero padding: x [D,H,W,Ci], w [Co,27,Ci] -> [D,H,W,Co]."""
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += shifted(x, dz, dy, dx) @ w[:, t, :].T
    if b is not None:
        y += b
    return y


def conv3_dgrad(gy, w):
    """Gradient of sum(gy * conv3(x, w)) with respect to x."""
    gx = np.zeros(gy.shape[:3] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        gx += shifted(gy, -dz, -dy, -dx) @ w[:, t, :]
    return gx


def conv3_wgrad(gy, x):
    """Gradient of sum(gy * conv3(x, w)) with respect to w: [Co, 27, Ci]."""
    co, ci = gy.shape[3], x.shape[3]
    g2 = gy.reshape(-1, co)
    gw = np.zeros((co, 27, ci))
    for t, (dz, dy, dx) in enumerate(TAPS):
        gw[:, t, :] = g2.T @ shifted(x, dz, dy, dx).reshape(-1, ci)
    return gw


def avgpool2(x):
    """Mean over disjoint 2x2x2 blocks."""
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def avgpool2_bwd(g):
    """Adjoint of avgpool2: every fine voxel receives g / 8 of its block."""
    return np.repeat(np.repeat(np.repeat(g, 2, axis=0), 2, axis=1), 2, axis=2) / 8.0


def upsample2(x):
    """Nearest-neighbour upsampling by 2 along each axis."""
    return np.repeat(np.repeat(np.repeat(x, 2, axis=0), 2, axis=1), 2, axis=2)


def upsample2_bwd(g):
    """Adjoint of upsample2: the sum over each 2x2x2 block."""
    D, H, W, C = g.shape
    return g.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


# ---------------------------------------------------------------- the network

def layer_shapes(base=32, levels=4, cin=2):
    """Ordered (name, Co, Ci, taps) of every layer."""
    ch = [base * 2 ** l for l in range(levels)]
    out = []
    prev = cin
    for l in range(levels):
        out.append((f"enc{l + 1}a", ch[l], prev, 27))
        out.append((f"enc{l + 1}b", ch[l], ch[l], 27))
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        out.append((f"dec{l + 1}a", ch[l], ch[l + 1] + ch[l], 27))
        out.append((f"dec{l + 1}b", ch[l], ch[l], 27))
    out.append(("head", 1, ch[0], 1))
    return out


def forward(params, xin, base=32, levels=4, bf16=False):
    """U-Net forward.  xin [D,H,W,2] (standardised inputs) -> (out [D,H,W], cache).

    params: {name: (w, b)} with w [Co,27,Ci] for 3x3x3 layers and [1, Ci] for the head.
    """
    act = {}
    x = _r(xin, bf16)
    act["in"] = x
    skips = []
    h = x
    for l in range(levels):
        if l > 0:
            h = _r(avgpool2(skips[-1]), bf16)
            act[f"pool{l}"] = h
        for s in "ab":
            w, b = params[f"enc{l + 1}{s}"]
            h = _r(np.maximum(conv3(h, _r(w, bf16), b), 0.0), bf16)
            act[f"enc{l + 1}{s}"] = h
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([upsample2(h), skips[l]], axis=3)
        act[f"cat{l + 1}"] = cat
        h = cat
        for s in "ab":
            w, b = params[f"dec{l + 1}{s}"]
            h = _r(np.maximum(conv3(h, _r(w, bf16), b), 0.0), bf16)
            act[f"dec{l + 1}{s}"] = h
    wh, bh = params["head"]
    if bf16:
        wh = wh.astype(np.float32).astype(np.float64)
    out = h @ wh[0] + bh[0]
    if bf16:
        out = out.astype(np.float32).astype(np.float64)
    return out, act


def backward(params, act, gout, base=32, levels=4, bf16=False):
    """Gradients {name: (gw, gb)} of sum(gout * out) for the forward pass that made ``act``."""
    grads = {}
    wh, _ = params["head"]
    top = act["dec1b"] if levels > 1 else act["enc1b"]
    grads["head"] = ((gout.reshape(-1) @ top.reshape(-1, top.shape[3]))[None, :], np.array([gout.sum()]))
    g = _r(gout[..., None] * wh[0] * (top > 0), bf16)

    def conv_back(name, g, x):
        w, _ = params[name]
        grads[name] = (conv3_wgrad(g, x), g.reshape(-1, g.shape[3]).sum(axis=0))
        return conv3_dgrad(g, _r(w, bf16))

    skip_grad = {}
    # decoder, top level first
    for l in range(0, levels - 1):
        gx = conv_back(f"dec{l + 1}b", g, act[f"dec{l + 1}a"])
        g = _r(gx * (act[f"dec{l + 1}a"] > 0), bf16)
        gcat = _r(conv_back(f"dec{l + 1}a", g, act[f"cat{l + 1}"]), bf16)
        cup = gcat.shape[3] - act[f"enc{l + 1}b"].shape[3]
        skip_grad[l] = gcat[..., cup:]
        below = act[f"dec{l + 2}b"] if l + 2 <= levels - 1 else act[f"enc{levels}b"]
        g = _r(upsample2_bwd(gcat[..., :cup]) * (below > 0), bf16)
    # bottleneck and encoder, deepest level first
    for l in range(levels - 1, -1, -1):
        gx = conv_back(f"enc{l + 1}b", g, act[f"enc{l + 1}a"])
        g = _r(gx * (act[f"enc{l + 1}a"] > 0), bf16)
        xin = act[f"pool{l}"] if l > 0 else act["in"]
        gx = conv_back(f"enc{l + 1}a", g, xin)
        if l == 0:
            break
        gp = _r(gx, bf16)
        a = act[f"enc{l}b"]
        g = _r((skip_grad[l - 1] + avgpool2_bwd(gp)) * (a > 0), bf16)
    return grads


def mse_loss(out, target):
    """Mean squared error over voxels and its gradient with respect to out."""
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) at step t >= 1; returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def standardise(rp, lnk):
    """Network inputs [D,H,W,2] and the scale s = rms(r_p) (s = 0 gives zero inputs).

    rp and lnk are [D,H,W] arrays.  ln k is shifted to zero mean and scaled to
    unit (population) standard deviation over the grid.
    """
    s = float(np.sqrt(np.mean(rp * rp)))
    mu = float(lnk.mean())
    sd = float(np.sqrt(np.mean((lnk - mu) ** 2)))
    x = np.zeros(rp.shape + (2,))
    if s > 0:
        x[..., 0] = rp / s
    if sd > 0:
        x[..., 1] = (lnk - mu) / sd
    return x, s


def apply_stage(params, rp, lnk, base=32, levels=4, bf16=False):
    """The learned pressure correction s * U(r_p / s, ln k) on a [D,H,W] grid."""
    x, s = standardise(rp, lnk)
    if s == 0:
        return np.zeros_like(rp)
    if bf16:
        x = x.astype(np.float32).astype(np.float64)
    out, _ = forward(params, x, base, levels, bf16)
    return s * out


def learned_cpr_apply(nx, ny, nz, row_ptr, col_idx, vals, params, lnk, f, base=32, levels=4, bf16=True):
    """CPR two-stage preconditioner (Section "CPR") with the network as the pressure solver.

    Stage one: p = Pi_r f (quasi-IMPES weights), x = Pi_p (s U(p / s, ln k));
    stage two: x += ILU0^{-1} (f - A x).  The restriction, prolongation,
    SpMV and ILU(0) are the oracle's own routines (oracle.c).
    """
    import oracle as O
    st, w, _ = O.qi_setup(nx, ny, nz, row_ptr, col_idx, vals)
    assert st == 0
    p = O.restrict_pressure(w, f)
    xp = apply_stage(params, p.reshape(nz, ny, nx), np.asarray(lnk).reshape(nz, ny, nx), base, levels, bf16)
    x = O.prolong_pressure(xp.ravel())
    r = O.spmv(row_ptr, col_idx, vals, x, alpha=-1.0, beta=1.0, y=np.array(f, dtype=np.float64))
    st, lu, udinv, _ = O.bilu0_setup(row_ptr, col_idx, vals)
    assert st == 0
    return x + O.bilu0_apply(row_ptr, col_idx, lu, udinv, r)
