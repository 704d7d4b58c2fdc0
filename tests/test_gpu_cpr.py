"""CPR preconditioner on the GPU (quasi-IMPES, GMG V-cycle, two-stage apply) against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import per_entry_ratio, report_ratio

pytestmark = pytest.mark.gpu

DIMS = [(20, 20, 10), (13, 7, 5), (33, 17, 9), (1, 1, 1), (40, 24, 16)]


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


def _setup(rsv, p, precision="fp64", **pcp):
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, precision=precision)
    s.setup("cpr", **pcp)
    return A, s


@pytest.mark.parametrize("dims", DIMS)
def test_hierarchy_matches_oracle(rsv, torch, dims):
    p = synth.make_problem(*dims, seed=51)
    A, s = _setup(rsv, p)
    levels, w, a7s = s.cpr_info()
    o = oracle.System.from_problem(p, pc="cpr")
    assert o.setup_status == 0
    _, w_or, a7_or = o.factors()
    assert len(levels) == o.gmg_levels()
    assert levels[0] == dims
    assert np.allclose(w, w_or, rtol=1e-13, atol=1e-15)
    scale = np.abs(a7_or).max(axis=1, keepdims=True)
    assert np.all(np.abs(a7s[0] - a7_or) <= 1e-12 * scale)
    cur, cdims = a7_or, dims
    for lv in range(1, len(levels)):
        cdims, cur = oracle.gmg_coarsen(*cdims, cur)
        assert tuple(cdims) == levels[lv]
        sc = np.abs(cur).max(axis=1, keepdims=True)
        assert np.all(np.abs(a7s[lv] - cur) <= 1e-12 * sc), lv


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("sweeps,coarse", [(2, 512), (1, 8), (0, 64)])
def test_vcycle_matches_oracle(rsv, torch, dims, sweeps, coarse):
    p = synth.make_problem(*dims, seed=52)
    A, s = _setup(rsv, p, gmg_sweeps=sweeps, gmg_max_coarse=coarse)
    _, _, a7 = oracle.System.from_problem(p, pc="cpr").factors()
    b = np.random.default_rng(53).standard_normal(p.nb)
    st, e_or, nl = oracle.gmg_vcycle(*dims, a7, b, max_levels=6, max_coarse=coarse, sweeps=sweeps)
    assert st == 0
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    s.vcycle(bd, xd)
    torch.cuda.synchronize()
    e = xd.cpu().numpy()
    ratio = report_ratio(f"vcycle_{dims}_{sweeps}_{coarse}", per_entry_ratio(e, e_or), 1e-9)
    assert ratio <= 1e-9


@pytest.mark.parametrize("dims", DIMS)
def test_cpr_apply_matches_oracle(rsv, torch, dims):
    p = synth.make_problem(*dims, seed=54)
    A, s = _setup(rsv, p)
    o = oracle.System.from_problem(p, pc="cpr")
    f = np.random.default_rng(55).standard_normal(p.n)
    st, z_or = o.pc_apply(f)
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"cpr_apply_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-9)
    assert ratio <= 1e-9


@pytest.mark.parametrize("dims", [(20, 20, 10), (33, 17, 9)])
def test_cpr_apply_fp32_matches_oracle(rsv, torch, dims):
    p = synth.make_problem(*dims, seed=56)
    A, s = _setup(rsv, p, precision="mixed")
    of = oracle.System.from_problem(p, pc="cpr", float_round=True)
    f = np.random.default_rng(57).standard_normal(p.n).astype(np.float32)
    _, z_or = of.pc_apply(f.astype(np.float64))
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"cpr_apply_fp32_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-3)
    assert ratio <= 1e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("solver", ["gmres", "bicgstab", "fgmres"])
def test_cpr_solve_tiny(rsv, torch, precision, solver):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, solver=solver, precision=precision, maxit=4000)
    s.setup("cpr")
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    if precision == "fp64" and solver != "bicgstab":
        o = oracle.System.from_problem(p, pc="cpr")
        ost, _, oinfo = o.gmres(p.b, flexible=(solver == "fgmres"), maxit=4000)
        assert ost == 0 and abs(info["iters"] - oinfo["iters"]) <= max(2, 0.1 * oinfo["iters"]), (info, oinfo)
    elif precision == "fp64":
        # BiCGSTAB's count is a chaotic function of rounding: compare with the oracle's spread
        its = []
        for t in range(6):
            bb = p.b if t == 0 else p.b * (1 + 1e-15 * np.random.default_rng(1000 + t).standard_normal(p.n))
            o = oracle.System.from_problem(p, pc="cpr")
            ost, _, oinfo = o.bicgstab(bb, maxit=4000) if solver == "bicgstab" else o.gmres(
                bb, flexible=(solver == "fgmres"), maxit=4000)
            assert ost == 0
            its.append(oinfo["iters"])
        assert 0.9 * min(its) - 2 <= info["iters"] <= 1.1 * max(its) + 2, (info, its)


def test_cpr_mid_full_size(rsv, torch):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_solves.json")))
    p = synth.workload("mid_100x100x50")
    for precision in ("fp64", "mixed"):
        A = rsv.Matrix(p.nx, p.ny, p.nz)
        A.set_values(p.vals)
        s = rsv.Solver(A, solver="gmres", precision=precision, maxit=4000)
        s.setup("cpr")
        levels, _, _ = s.cpr_info(with_arrays=False)
        assert levels[0] == (100, 100, 50) and len(levels) == 5 and levels[-1] == (7, 7, 4)
        b = torch.from_numpy(p.b).cuda()
        x = torch.zeros_like(b)
        st, info = s.solve(b, x)
        assert st == 0, info
        relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(
            p.b)
        assert relres <= 1e-8
        # iteration counts against the oracle's: FP64 GMRES, and the refinement model of the mixed solve
        g = gold["mid_100x100x50/" + ("gmres" if precision == "fp64" else "refine-gmres") + "/cpr"]
        print(f"CPR_MID_ITERS {precision} gpu {info['iters']} oracle {g['iters']}")
        assert abs(info["iters"] - g["iters"]) <= max(2, 0.1 * g["iters"]), (precision, info, g)


# ---- the other stage orders of Section "CPR-like preconditioners" (FP, FPF, FFPF)

ORDERS = ["cpr_fp", "cpr_fpf", "cpr_ffpf"]


def _setup_order(rsv, p, pc, precision="fp64"):
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, precision=precision)
    s.setup(pc)
    return A, s


@pytest.mark.parametrize("pc", ORDERS)
@pytest.mark.parametrize("dims", [(20, 20, 10), (13, 7, 5), (1, 1, 1), (40, 24, 16)])
def test_cpr_order_apply_matches_oracle(rsv, torch, pc, dims):
    p = synth.make_problem(*dims, seed=58)
    A, s = _setup_order(rsv, p, pc)
    o = oracle.System.from_problem(p, pc=pc)
    f = np.random.default_rng(59).standard_normal(p.n)
    st, z_or = o.pc_apply(f)
    assert st == 0
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"{pc}_apply_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-9)
    assert ratio <= 1e-9


@pytest.mark.parametrize("pc", ORDERS)
def test_cpr_order_apply_fp32_matches_oracle(rsv, torch, pc):
    p = synth.make_problem(33, 17, 9, seed=60)
    A, s = _setup_order(rsv, p, pc, precision="mixed")
    of = oracle.System.from_problem(p, pc=pc, float_round=True)
    f = np.random.default_rng(61).standard_normal(p.n).astype(np.float32)
    _, z_or = of.pc_apply(f.astype(np.float64))
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"{pc}_apply_fp32", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-3)
    assert ratio <= 1e-3


@pytest.mark.parametrize("pc", ORDERS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cpr_order_gmres_solve(rsv, torch, pc, precision):
    p = synth.make_problem(20, 20, 10, seed=0)
    A, _ = _setup_order(rsv, p, "none")
    s = rsv.Solver(A, solver="gmres", precision=precision, maxit=4000)
    s.setup(pc)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    if precision == "fp64":
        o = oracle.System.from_problem(p, pc=pc)
        ost, _, oinfo = o.gmres(p.b, maxit=4000)
        assert ost == 0 and abs(info["iters"] - oinfo["iters"]) <= max(2, 0.1 * oinfo["iters"]), (info, oinfo)


# ---- ABF decoupling (rsv_pc_params.decoupling = 1)

@pytest.mark.parametrize("pc", ["cpr", "cpr_fpf"])
@pytest.mark.parametrize("dims", [(20, 20, 10), (13, 7, 5), (1, 1, 1)])
def test_abf_cpr_apply_matches_oracle(rsv, torch, pc, dims):
    p = synth.make_problem(*dims, seed=62)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A)
    s.setup(pc, decoupling="abf")
    o = oracle.System.from_problem(p, pc=pc, decoupling="abf")
    _, w_or, a7_or = o.factors()
    levels, w, a7 = s.cpr_info()
    assert np.allclose(w, w_or, rtol=1e-12, atol=1e-14 * np.abs(w_or).max())
    f = np.random.default_rng(63).standard_normal(p.n)
    st, z_or = o.pc_apply(f)
    assert st == 0
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"abf_{pc}_apply_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-9)
    assert ratio <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_abf_cpr_fpf_gmres_solve(rsv, torch, precision):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, solver="gmres", precision=precision, maxit=4000)
    s.setup("cpr_fpf", decoupling="abf")
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    if precision == "fp64":
        o = oracle.System.from_problem(p, pc="cpr_fpf", decoupling="abf")
        ost, _, oinfo = o.gmres(p.b, maxit=4000)
        assert ost == 0 and abs(info["iters"] - oinfo["iters"]) <= max(2, 0.1 * oinfo["iters"]), (info, oinfo)


def test_decoupling_argument_checked(rsv, torch):
    p = synth.make_problem(4, 3, 2, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A)
    with pytest.raises(rsv.RsvError) as e:
        s.setup("cpr", decoupling=2)
    assert e.value.status == rsv.RSV_EINVAL


# ---- true-IMPES decoupling (rsv_pc_params.decoupling = 2, accumulation blocks given)

@pytest.mark.parametrize("pc", ["cpr", "cpr_fpf"])
@pytest.mark.parametrize("dims", [(20, 20, 10), (13, 7, 5), (1, 1, 1)])
def test_true_impes_cpr_apply_matches_oracle(rsv, torch, pc, dims):
    p = synth.make_problem(*dims, seed=64)
    acc = p.accumulation()
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A)
    s.set_accumulation(acc)
    s.setup(pc, decoupling="timpes")
    o = oracle.System.from_problem(p, pc=pc, decoupling="timpes", acc=acc)
    assert o.setup_status == 0
    _, w_or, a7_or = o.factors()
    levels, w, a7 = s.cpr_info()
    assert np.allclose(w, w_or, rtol=1e-13, atol=0)
    assert np.all(np.abs(a7[0] - a7_or) <= 1e-12 * np.abs(a7_or).max(axis=1, keepdims=True))
    f = np.random.default_rng(65).standard_normal(p.n)
    st, z_or = o.pc_apply(f)
    assert st == 0
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"timpes_{pc}_apply_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-9)
    assert ratio <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_true_impes_gmres_solve(rsv, torch, precision):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, solver="gmres", precision=precision, maxit=4000)
    s.set_accumulation(torch.from_numpy(p.accumulation()).cuda())
    s.setup("cpr", decoupling="timpes")
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    if precision == "fp64":
        o = oracle.System.from_problem(p, pc="cpr", decoupling="timpes", acc=p.accumulation())
        ost, _, oinfo = o.gmres(p.b, maxit=4000)
        assert ost == 0 and abs(info["iters"] - oinfo["iters"]) <= max(2, 0.1 * oinfo["iters"]), (info, oinfo)


def test_true_impes_needs_accumulation_blocks(rsv, torch):
    p = synth.make_problem(4, 3, 2, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A)
    with pytest.raises(rsv.RsvError) as e:
        s.setup("cpr", decoupling="timpes")
    assert e.value.status == rsv.RSV_EINVAL
    acc = p.accumulation()
    acc[3] = 0.0  # a singular accumulation block
    s.set_accumulation(acc)
    with pytest.raises(rsv.RsvError) as e:
        s.setup("cpr", decoupling="timpes")
    assert e.value.status == rsv.RSV_ESINGULAR
    s.set_accumulation(None)
    with pytest.raises(rsv.RsvError) as e:
        s.setup("cpr", decoupling="timpes")
    assert e.value.status == rsv.RSV_EINVAL


# ---- algebraic coarsening of the pressure stage (rsv_pc_params.coarsening = 1)

AMG_DIMS = [(20, 20, 10), (13, 7, 5), (33, 17, 9), (40, 24, 16)]


def _amg_setup(rsv, p, precision="fp64", pc="cpr", coarse=64):
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, precision=precision)
    s.setup(pc, coarsening="amg", gmg_max_levels=8, gmg_max_coarse=coarse)
    return A, s


@pytest.mark.parametrize("dims", AMG_DIMS)
def test_amg_hierarchy_and_vcycle_match_oracle(rsv, torch, dims):
    """The same PMIS splitting level by level (points and nonzeros equal), and one
    V-cycle per entry against the oracle's."""
    p = synth.make_problem(*dims, seed=66)
    A, s = _amg_setup(rsv, p)
    _, _, a7 = oracle.System.from_problem(p, pc="cpr").factors()
    ref = oracle.amg_hierarchy(*dims, a7, max_levels=8, max_coarse=64)
    assert s.amg_info() == ref and len(ref) >= 2
    b = np.random.default_rng(67).standard_normal(p.nb)
    st, e_or, nl = oracle.amg_vcycle(*dims, a7, b, max_levels=8, max_coarse=64, sweeps=2)
    assert st == 0 and nl == len(ref)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    s.vcycle(bd, xd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"amg_vcycle_{dims}", per_entry_ratio(xd.cpu().numpy(), e_or), 1e-9)
    assert ratio <= 1e-9


@pytest.mark.parametrize("dims", [(20, 20, 10), (40, 24, 16)])
def test_cpr_amg_apply_matches_oracle(rsv, torch, dims):
    p = synth.make_problem(*dims, seed=68)
    A, s = _amg_setup(rsv, p)
    o = oracle.System.from_problem(p, pc="cpr", coarsening="amg", gmg_levels=8, gmg_coarse=64)
    assert o.setup_status == 0
    f = np.random.default_rng(69).standard_normal(p.n)
    st, z_or = o.pc_apply(f)
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"cpr_amg_apply_{dims}", per_entry_ratio(zd.cpu().numpy(), z_or), 1e-9)
    assert ratio <= 1e-9
    # FP32: the GPU applies the FP32-rounded hierarchy in FP32, the oracle the same rounded values in FP64
    A32, s32 = _amg_setup(rsv, p, precision="mixed")
    of = oracle.System.from_problem(p, pc="cpr", coarsening="amg", gmg_levels=8, gmg_coarse=64, float_round=True)
    f32 = f.astype(np.float32)
    _, z32_or = of.pc_apply(f32.astype(np.float64))
    f32d = torch.from_numpy(f32).cuda()
    z32d = torch.zeros_like(f32d)
    s32.apply(f32d, z32d)
    torch.cuda.synchronize()
    ratio = report_ratio(f"cpr_amg_apply_fp32_{dims}", per_entry_ratio(z32d.cpu().numpy(), z32_or), 1e-3)
    assert ratio <= 1e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cpr_amg_gmres_solve(rsv, torch, precision):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, solver="gmres", precision=precision, maxit=4000)
    s.setup("cpr", coarsening="amg", gmg_max_levels=8, gmg_max_coarse=64)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK, (st, info)
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    if precision == "fp64":
        o = oracle.System.from_problem(p, pc="cpr", coarsening="amg", gmg_levels=8, gmg_coarse=64)
        ost, _, oinfo = o.gmres(p.b, maxit=4000)
        assert ost == 0 and abs(info["iters"] - oinfo["iters"]) <= max(2, 0.1 * oinfo["iters"]), (info, oinfo)


def test_amg_hierarchy_matches_oracle_at_100x100x50(rsv, torch):
    """500,000 pressure points: six algebraic levels, equal to the oracle's, and the
    V-cycle per entry."""
    p = synth.workload("mid_100x100x50")
    A, s = _amg_setup(rsv, p, coarse=512)
    _, _, a7 = oracle.System.from_problem(p, pc="cpr").factors()
    ref = oracle.amg_hierarchy(p.nx, p.ny, p.nz, a7, max_levels=8, max_coarse=512)
    assert s.amg_info() == ref, (s.amg_info(), ref)
    b = np.random.default_rng(70).standard_normal(p.nb)
    st, e_or, _ = oracle.amg_vcycle(p.nx, p.ny, p.nz, a7, b, max_levels=8, max_coarse=512, sweeps=2)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    s.vcycle(bd, xd)
    torch.cuda.synchronize()
    ratio = report_ratio("amg_vcycle_mid", per_entry_ratio(xd.cpu().numpy(), e_or), 1e-9)
    assert ratio <= 1e-9
