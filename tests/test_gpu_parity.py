"""GPU path (through the C ABI) against the CPU oracle on the same seeded inputs."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import per_entry_ratio, report_ratio

pytestmark = pytest.mark.gpu

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


def _mat(rsv, p):
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    assert np.array_equal(A.row_ptr, p.row_ptr) and np.array_equal(A.col_idx, p.col_idx)
    A.set_values(p.vals)
    return A


def _row_scale(p, x):
    """|A| |x| per scalar row: the scale of each SpMV entry's rounding error."""
    return oracle.spmv(p.row_ptr, p.col_idx, np.abs(p.vals), np.abs(x))


SPMV_DIMS = [(1, 1, 1), (2, 2, 1), (7, 5, 3), (20, 20, 10), (33, 17, 9), (100, 100, 50)]


@pytest.mark.parametrize("dims", SPMV_DIMS)
def test_spmv_fp64_per_entry(rsv, torch, dims):
    p = synth.make_problem(*dims, seed=31)
    A = _mat(rsv, p)
    rng = np.random.default_rng(32)
    x, y0 = rng.standard_normal(p.n), rng.standard_normal(p.n)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y0).cuda()
    A.spmv(xd, yd, alpha=-0.75, beta=1.25)
    torch.cuda.synchronize()
    ref = oracle.spmv(p.row_ptr, p.col_idx, p.vals, x, alpha=-0.75, beta=1.25, y=y0)
    scale = 0.75 * _row_scale(p, x) + 1.25 * np.abs(y0)
    err = np.abs(yd.cpu().numpy() - ref)
    assert np.all(err <= 1e-12 * scale), err.max()
    # beta = 0 must not read y (NaN garbage in y stays out)
    yd.fill_(float("nan"))
    A.spmv(xd, yd)
    ref0 = oracle.spmv(p.row_ptr, p.col_idx, p.vals, x)
    assert np.all(np.abs(yd.cpu().numpy() - ref0) <= 1e-12 * _row_scale(p, x))


@pytest.mark.parametrize("dims", [(7, 5, 3), (33, 17, 9)])
def test_spmv_fp32_per_entry(rsv, torch, dims):
    p = synth.make_problem(*dims, seed=33)
    A = _mat(rsv, p)
    x = np.random.default_rng(34).standard_normal(p.n).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    A.spmv(xd, yd)
    torch.cuda.synchronize()
    v32 = p.vals.astype(np.float32).astype(np.float64)
    ref = oracle.spmv(p.row_ptr, p.col_idx, v32, x.astype(np.float64))
    scale = _row_scale(p, x.astype(np.float64))
    assert np.all(np.abs(yd.cpu().numpy() - ref) <= 24 * 2.0 ** -24 * scale)


@pytest.mark.parametrize("n", [1, 1000, 3 * 33 * 17 * 9, 1_500_000])
def test_blas1(rsv, torch, n):
    import ctypes
    rng = np.random.default_rng(n)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = ctypes.c_double()
    s = torch.cuda.current_stream().cuda_stream
    assert rsv.rsv_dot(s, n, xd.data_ptr(), yd.data_ptr(), ctypes.byref(out)) == 0
    assert abs(out.value - oracle.dot(x, y)) <= 1e-13 * np.abs(x * y).sum()
    assert rsv.rsv_norm2(s, n, xd.data_ptr(), ctypes.byref(out)) == 0
    assert abs(out.value - oracle.norm2(x)) <= 1e-13 * oracle.norm2(x)
    zd = torch.empty_like(xd)
    assert rsv.rsv_axpby(s, n, 0.5, xd.data_ptr(), -2.0, yd.data_ptr(), zd.data_ptr()) == 0
    torch.cuda.synchronize()
    assert np.allclose(zd.cpu().numpy(), 0.5 * x - 2.0 * y, rtol=0, atol=1e-15 * (np.abs(x) + np.abs(y)).max())


@pytest.mark.parametrize("dims", [(1, 1, 1), (9, 1, 1), (7, 5, 3), (20, 20, 10), (33, 17, 9)])
@pytest.mark.parametrize("pc", ["bjacobi", "bilu0"])
def test_preconditioner_factor_and_apply(rsv, torch, dims, pc):
    p = synth.make_problem(*dims, seed=35)
    A = _mat(rsv, p)
    s = rsv.Solver(A)
    s.setup(pc)
    o = oracle.System.from_problem(p, pc=pc)
    assert o.setup_status == 0
    d_or, _, _ = o.factors()
    d_gpu = s.dinv()
    assert np.all(np.abs(d_gpu - d_or) <= 1e-12 * np.abs(d_or).max(axis=(1, 2), keepdims=True))
    r = np.random.default_rng(36).standard_normal(p.n)
    rd = torch.from_numpy(r).cuda()
    zd = torch.zeros_like(rd)
    s.apply(rd, zd)
    torch.cuda.synchronize()
    _, z_or = o.pc_apply(r)
    ratio = report_ratio(f"{pc}_apply_fp64_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-10)
    assert ratio <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ilu_apply_mid_full_size_per_entry(rsv, torch, precision):
    """Block ILU(0) apply at 100x100x50 (13x13 tiles of 8x4 pencils, the full
    edge hand-off protocol of the tile sweeps) against the oracle, per entry.
    FP32 (mixed): the GPU applies the FP32 factor in FP32; the oracle applies the
    same FP32-rounded factor in FP64."""
    p = synth.workload("mid_100x100x50")
    A = _mat(rsv, p)
    s = rsv.Solver(A, precision=precision)
    s.setup("bilu0")
    o = oracle.System.from_problem(p, pc="bilu0", float_round=(precision == "mixed"))
    r = np.random.default_rng(46).standard_normal(p.n)
    if precision == "mixed":
        r = r.astype(np.float32)
    rd = torch.from_numpy(r).cuda()
    zd = torch.zeros_like(rd)
    s.apply(rd, zd)
    torch.cuda.synchronize()
    _, z_or = o.pc_apply(r.astype(np.float64))
    bound = 1e-10 if precision == "fp64" else 1e-3
    ratio = report_ratio(f"bilu0_apply_{precision}_mid", per_entry_ratio(zd.cpu().numpy(), z_or), bound)
    assert ratio <= bound


SOLVES = [("bicgstab", "bjacobi"), ("gmres", "bilu0"), ("fgmres", "bilu0"), ("bicgstab", "bilu0"),
          ("gmres", "bjacobi"), ("gmres", "none")]


def _oracle_solve(p, solver, pc, m=30, maxit=2000):
    o = oracle.System.from_problem(p, pc=pc)
    if solver == "bicgstab":
        return o.bicgstab(p.b, maxit=maxit)
    return o.gmres(p.b, m=m, flexible=(solver == "fgmres"), maxit=maxit)


def _iters_close(a, b):
    return abs(a - b) <= max(2, 0.10 * b)


def _oracle_iter_range(p, solver, pc, trials=8, maxit=4000):
    """Oracle iteration counts over right-hand sides perturbed at the rounding level
    (relative 1e-15).  BiCGSTAB's count is a chaotic function of rounding, so the GPU
    count is compared against this spread widened by 10%, not a single run."""
    its = []
    for t in range(trials):
        b = p.b if t == 0 else p.b * (1 + 1e-15 * np.random.default_rng(1000 + t).standard_normal(p.n))
        o = oracle.System.from_problem(p, pc=pc)
        st, _, info = o.bicgstab(b, maxit=maxit) if solver == "bicgstab" else o.gmres(
            b, m=30, flexible=(solver == "fgmres"), maxit=maxit)
        assert st == 0
        its.append(info["iters"])
    return min(its), max(its)


@pytest.mark.parametrize("solver,pc", SOLVES)
@pytest.mark.parametrize("dims", [(20, 20, 10), (13, 7, 5)])
def test_solve_tiny_matches_oracle(rsv, torch, solver, pc, dims):
    p = synth.make_problem(*dims, seed=0 if dims == (20, 20, 10) else 37)
    A = _mat(rsv, p)
    s = rsv.Solver(A, solver=solver, restart=30, rtol=1e-8, maxit=4000)
    s.setup(pc)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    xh = x.cpu().numpy()
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, xh)) / np.linalg.norm(p.b)
    assert relres <= 1e-8 and abs(relres - info["true_relres"]) <= 1e-12
    if solver == "bicgstab":
        # BiCGSTAB's count is a chaotic function of rounding: compare with the oracle's spread
        lo, hi = _oracle_iter_range(p, solver, pc)
        assert 0.9 * lo - 2 <= info["iters"] <= 1.1 * hi + 2, (info, lo, hi)
    else:
        ost, _, oinfo = _oracle_solve(p, solver, pc, maxit=4000)
        assert ost == 0 and _iters_close(info["iters"], oinfo["iters"]), (info, oinfo)


def test_host_buffers_match_device_buffers(rsv, torch):
    p = synth.make_problem(11, 9, 7, seed=38)
    A = _mat(rsv, p)
    s = rsv.Solver(A, solver="gmres")
    s.setup("bilu0")
    xh = np.zeros(p.n)
    st, info = s.solve(p.b.copy(), xh)
    b = torch.from_numpy(p.b).cuda()
    xd = torch.zeros_like(b)
    st2, info2 = s.solve(b, xd)
    assert st == st2 == 0 and info["iters"] == info2["iters"]
    assert np.array_equal(xh, xd.cpu().numpy())


def test_maxit_reports_noconv_with_iterate(rsv, torch):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = _mat(rsv, p)
    for solver in ("gmres", "bicgstab"):
        s = rsv.Solver(A, solver=solver, maxit=7)
        s.setup("bjacobi")
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = s.solve(torch.from_numpy(p.b).cuda(), x)
        assert st == rsv.RSV_ENOCONV and info["status"] == rsv.RSV_ENOCONV
        assert info["iters"] == 7 and 0 < info["true_relres"] < 1.0


def test_zero_rhs_and_nonfinite_rhs(rsv, torch):
    p = synth.make_problem(6, 5, 4, seed=39)
    A = _mat(rsv, p)
    s = rsv.Solver(A)
    s.setup("bilu0")
    b = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == 0 and info["iters"] == 0 and float(x.abs().max()) == 0.0
    b[5] = float("nan")
    st, info = s.solve(b, x)
    assert st == rsv.RSV_ENAN


def test_singular_block_reported_at_setup(rsv, torch):
    p = synth.make_problem(5, 4, 3, seed=40)
    vals = p.vals.copy()
    d = p.row_ptr[7] + [q for q in range(p.row_ptr[7], p.row_ptr[8]) if p.col_idx[q] == 7][0] - p.row_ptr[7]
    vals[d] = np.array([[1.0, 2, 3], [2, 4, 6], [1, 1, 1]])  # rank 2
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(vals)
    s = rsv.Solver(A)
    with pytest.raises(rsv.RsvError) as e:
        s.setup("bjacobi")
    assert e.value.status == rsv.RSV_ESINGULAR


def test_state_errors(rsv, torch):
    p = synth.make_problem(4, 4, 4, seed=41)
    A = _mat(rsv, p)
    s = rsv.Solver(A)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, _ = s.solve(b, x)
    assert st == rsv.RSV_EINVAL  # no preconditioner yet
    s.setup("bilu0")
    A.set_values(p.vals)  # new values invalidate the factor
    st, _ = s.solve(b, x)
    assert st == rsv.RSV_EINVAL
    with pytest.raises(rsv.RsvError):
        rsv.Solver(A, restart=0)


@pytest.mark.parametrize("dims", [(7, 5, 3), (20, 20, 10), (33, 17, 9)])
@pytest.mark.parametrize("pc", ["bjacobi", "bilu0"])
def test_mixed_preconditioner_fp32(rsv, torch, dims, pc):
    """Mixed precision: the factor is computed in FP64 from the FP32-rounded matrix
    (compared with the oracle on the same rounded values to 1e-12) and applied in
    FP32 (compared with the oracle's FP64 application of the FP32-rounded factor)."""
    p = synth.make_problem(*dims, seed=44)
    A = _mat(rsv, p)
    s = rsv.Solver(A, precision="mixed")
    s.setup(pc)
    v32 = p.vals.astype(np.float32).astype(np.float64)
    o = oracle.System(p.nx, p.ny, p.nz, p.row_ptr, p.col_idx, v32, pc=pc)
    d_or, _, _ = o.factors()
    d_gpu = s.dinv()
    assert np.all(np.abs(d_gpu - d_or) <= 1e-12 * np.abs(d_or).max(axis=(1, 2), keepdims=True))
    of = oracle.System.from_problem(p, pc=pc, float_round=True)
    r = np.random.default_rng(45).standard_normal(p.n).astype(np.float32)
    rd = torch.from_numpy(r).cuda()
    zd = torch.zeros_like(rd)
    s.apply(rd, zd)
    torch.cuda.synchronize()
    _, z_or = of.pc_apply(r.astype(np.float64))
    ratio = report_ratio(f"{pc}_apply_fp32_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-3)
    assert ratio <= 1e-3


@pytest.mark.parametrize("solver,pc", [("gmres", "bilu0"), ("bicgstab", "bilu0"), ("gmres", "bjacobi"),
                                       ("fgmres", "bilu0")])
def test_mixed_solve_reaches_fp64_tolerance(rsv, torch, solver, pc):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = _mat(rsv, p)
    s = rsv.Solver(A, solver=solver, precision="mixed", rtol=1e-8, inner_rtol=1e-5, maxit=6000, max_outer=10)
    s.setup(pc)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    xh = x.cpu().numpy()
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, xh)) / np.linalg.norm(p.b)
    assert relres <= 1e-8 and abs(relres - info["true_relres"]) <= 1e-12
    assert info["outer_iters"] >= 2
    outer = oracle.System.from_problem(p, pc="none")
    inner = oracle.System.from_problem(p, pc=pc, float_round=True)
    its = []
    # GMRES: the oracle's refinement count itself; BiCGSTAB: its spread under rounding-level
    # perturbations of b (the count is a chaotic function of rounding)
    for t in range(1 if solver != "bicgstab" else 6):
        bb = p.b if t == 0 else p.b * (1 + 1e-15 * np.random.default_rng(2000 + t).standard_normal(p.n))
        ost, _, oinfo = oracle.refine(outer, inner, bb, solver="bicgstab" if solver == "bicgstab" else "gmres",
                                      maxit=6000)
        assert ost == 0
        its.append(oinfo["iters"])
    print(f"MIXED_ITERS {solver}/{pc} gpu {info['iters']} oracle {its}")
    assert 0.9 * min(its) - 2 <= info["iters"] <= 1.1 * max(its) + 2, (info, its)


def test_watchdog_timeout_returns_status_and_context_survives(rsv, torch):
    """A 1 microsecond wait limit makes the tile sweeps' cross-warp waits run out:
    the solve reports ETIMEOUT (no trap, no hang) and the next solve with the
    normal limit succeeds on the same context."""
    p = synth.make_problem(24, 40, 20, seed=43)
    A = _mat(rsv, p)
    b = torch.from_numpy(p.b).cuda()
    s = rsv.Solver(A, solver="gmres", watchdog=1)
    s.setup("bilu0")
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_ETIMEOUT, (st, info)
    s2 = rsv.Solver(A, solver="gmres")
    s2.setup("bilu0")
    x.zero_()
    st, info = s2.solve(b, x)
    assert st == rsv.RSV_OK and info["true_relres"] <= 1e-8
    # the timed-out solver recovers too once its limit is back to normal
    st, info = s.solve(b, x)
    assert st in (rsv.RSV_OK, rsv.RSV_ETIMEOUT)


def test_spmv_wait_timeout_reports_status_and_nan(rsv, torch):
    """The SpMV stages each CTA's blocks with a bulk copy and waits on it with the
    solver's time limit.  A 1 microsecond limit (without a preconditioner, so the
    SpMV holds the only waits) runs out before a 100x100x50 CTA's 66 KB arrive: the
    solve reports ETIMEOUT instead of iterating on stale values, and a solver with
    the normal limit then solves on the same context."""
    p = synth.workload("mid_100x100x50")
    A = _mat(rsv, p)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    s = rsv.Solver(A, solver="gmres", watchdog=1, maxit=5)
    s.setup("none")
    st, info = s.solve(b, x)
    assert st == rsv.RSV_ETIMEOUT, (st, info)
    s2 = rsv.Solver(A, solver="gmres", maxit=5)
    s2.setup("none")
    x.zero_()
    st, info = s2.solve(b, x)
    assert st == rsv.RSV_ENOCONV and np.isfinite(x.cpu().numpy()).all() and info["iters"] == 5


def test_mid_mixed_gmres_bilu0_full_size(rsv, torch):
    p = synth.workload("mid_100x100x50")
    A = _mat(rsv, p)
    s = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=4000, precision="mixed")
    s.setup("bilu0")
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == 0, info
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    gold = json.load(open(GOLDEN))["mid_100x100x50/refine-gmres/bilu0"]
    print(f"MIXED_ITERS mid gmres/bilu0 gpu {info['iters']} oracle {gold['iters']}")
    assert _iters_close(info["iters"], gold["iters"]), (info, gold)


def test_mid_gmres_bilu0_full_size(rsv, torch):
    """100x100x50 (500k cells, 1.5M unknowns), layered permeability: the benchmark workload."""
    gold = json.load(open(GOLDEN))["mid_100x100x50/gmres/bilu0"]
    p = synth.workload("mid_100x100x50")
    A = _mat(rsv, p)
    s = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=2000)
    s.setup("bilu0")
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == 0, info
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    assert _iters_close(info["iters"], gold["iters"]), (info, gold)
    # factor parity at full size on sampled cells
    st_, lu, udinv, _ = oracle.bilu0_setup(p.row_ptr, p.col_idx, p.vals)
    d = s.dinv()
    idx = np.random.default_rng(42).choice(p.nb, 2000, replace=False)
    assert np.all(np.abs(d[idx] - udinv[idx]) <= 1e-12 * np.abs(udinv[idx]).max(axis=(1, 2), keepdims=True))
