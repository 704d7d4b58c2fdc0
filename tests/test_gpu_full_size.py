"""The larger workloads at their full sizes, checked on outputs the oracle computes one by one.

* 256x256x128 channelised CPR (8.4M cells, 25.2M unknowns, 4.2 GB of FP64
  blocks): SpMV on sampled rows, and GMRES(30) + CPR to rtol 1e-8 in FP64 and
  in the FP32-inner / FP64-refinement form, the true residual recomputed by
  the oracle's own SpMV of the whole system.
* 128x128x64 learned-stage grid: the finest-level convolutions on sampled
  voxels and sampled weight-gradient entries, and an FGMRES + learned CPR
  solve to rtol 1e-8.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import unet as U

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_solves.json")


@pytest.fixture(scope="module")
def rsv():
    from tests.helpers import build_library
    build_library()
    import paper_1602_05901_gb300 as m
    return m


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def large():
    return synth.workload("large_256x256x128")


def test_large_spmv_sampled_rows(rsv, torch, large):
    p = large
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    x = np.random.default_rng(7).standard_normal(p.n)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    A.spmv(xd, yd)
    y = yd.cpu().numpy()
    rows = np.random.default_rng(8).choice(p.nb, 4000, replace=False)
    for c in rows:
        lo, hi = p.row_ptr[c], p.row_ptr[c + 1]
        blocks, cols = p.vals[lo:hi], p.col_idx[lo:hi]
        ref = sum(blocks[q] @ x[3 * cols[q]:3 * cols[q] + 3] for q in range(hi - lo))
        scale = sum(np.abs(blocks[q]) @ np.abs(x[3 * cols[q]:3 * cols[q] + 3]) for q in range(hi - lo))
        assert np.all(np.abs(y[3 * c:3 * c + 3] - ref) <= 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_cpr_solve(rsv, torch, large, precision):
    p = large
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=6000, precision=precision)
    s.setup("cpr")
    levels, _, _ = s.cpr_info(with_arrays=False)
    assert levels[0] == (256, 256, 128) and len(levels) == 6
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == 0, info
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8 and abs(relres - info["true_relres"]) <= 1e-10, (relres, info)
    # iteration count within 10% of the oracle's (FP64 GMRES, or its refinement model of the mixed solve)
    gold = json.load(open(GOLDEN))["large_256x256x128/" + ("gmres" if precision == "fp64" else "refine-gmres") + "/cpr"]
    print(f"LARGE_CPR_ITERS {precision} gpu {info['iters']} oracle {gold['iters']}", info)
    assert abs(info["iters"] - gold["iters"]) <= max(2, 0.1 * gold["iters"]), (info, gold)


def _bf16(torch, a):
    t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float32).to(torch.bfloat16)
    return t.cuda(), t.float().double().numpy()


def test_finest_level_convolutions_sampled(rsv, torch):
    """128x128x64, 96 -> 32 channels (the decoder's concatenated input): forward on
    sampled voxels, weight gradient on sampled entries, each summed directly."""
    nx, ny, nz, ci, co = 128, 128, 64, 96, 32
    rng = np.random.default_rng(11)
    xt, xh = _bf16(torch, rng.standard_normal((nz, ny, nx, ci)).astype(np.float32))
    wt, wh = _bf16(torch, (rng.standard_normal((co, 27, ci)) * 0.05).astype(np.float32))
    gyt, gyh = _bf16(torch, rng.standard_normal((nz, ny, nx, co)).astype(np.float32))
    y32 = torch.empty((nx * ny * nz, co), device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rsv.check(rsv.rsv_conv3d_fwd(None, nx, ny, nz, 27, ci, co, p(xt), ci, p(wt), None, 0, None, 0, None, 0, p(y32)))
    gw = torch.empty((co, 27, ci), device="cuda")
    rsv.check(rsv.rsv_conv3d_wgrad(None, nx, ny, nz, 27, ci, co, p(xt), ci, p(gyt), co, p(gw), None))
    y = y32.cpu().double().numpy().reshape(nz, ny, nx, co)
    g = gw.cpu().double().numpy()
    # forward: 3000 voxels, 27 taps x 96 channels each, zero outside the grid
    for _ in range(3000):
        z, yy, xx = rng.integers(0, nz), rng.integers(0, ny), rng.integers(0, nx)
        ref = np.zeros(co)
        absref = np.zeros(co)
        for t, (dz, dy, dx) in enumerate(U.TAPS):
            zz, y2, x2 = z + dz, yy + dy, xx + dx
            if 0 <= zz < nz and 0 <= y2 < ny and 0 <= x2 < nx:
                ref += wh[:, t, :] @ xh[zz, y2, x2]
                absref += np.abs(wh[:, t, :]) @ np.abs(xh[zz, y2, x2])
        assert np.all(np.abs(y[z, yy, xx] - ref) <= 2 * 27 * ci * U32 * absref + 1e-30)
    # weight gradient: 40 entries, each a sum over all 1,048,576 voxels
    for _ in range(40):
        o, t, c = rng.integers(0, co), rng.integers(0, 27), rng.integers(0, ci)
        sx = U.shifted(xh[..., c:c + 1], *U.TAPS[t])[..., 0]
        ref = np.sum(gyh[..., o] * sx)
        absref = np.sum(np.abs(gyh[..., o] * sx))
        assert abs(g[o, t, c] - ref) <= 2 * nx * ny * nz * U32 * absref, (o, t, c, g[o, t, c], ref)


def test_learned_cpr_full_size_converges(rsv):
    """FGMRES(30) + learned CPR on the 128x128x64 channelised workload (an untrained
    network; the fallback to the V-cycle keeps the solve converging)."""
    p = synth.workload("learned_128x128x64")
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    net = rsv.Unet(p.nx, p.ny, p.nz, base=32, levels=4)
    net.set_params(synth.unet_init(32, 4, seed=0))
    s = rsv.Solver(A, solver="fgmres", precision="fp64", rtol=1e-8, maxit=4000)
    s.set_learned(net, p.lnk, stall_window=30, stall_drop=0.10)
    s.setup("cpr_learned")
    x = np.zeros(p.n)
    st, info = s.solve(p.b.copy(), x)
    assert st == rsv.RSV_OK, info
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x)) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    assert -1 <= info["fallback_iter"] <= info["iters"]
