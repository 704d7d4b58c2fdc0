"""The smoother's large-level forms against the oracle.

On a level with at least 2^20 cells of one colour the red-black half sweeps take
four cells per thread, and the first post-smoothing half sweep becomes a
prolongation pass (a 16-byte form when nx is a multiple of 4, FP32) followed by
a plain half sweep.  These forms run only on grids of about two million cells
or more, so they are checked here, per entry, on 160x128x104 (nx a multiple of
4) and 161x128x104 (odd rows: a row's two colours differ in count).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import per_entry_ratio, report_ratio

pytestmark = pytest.mark.gpu

WIDE = [(160, 128, 104), (161, 128, 104)]


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


@pytest.fixture(scope="module", params=WIDE, ids=lambda d: "x".join(map(str, d)))
def problem(request):
    return synth.make_problem(*request.param, seed=58)


def _solver(rsv, p, precision):
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, precision=precision)
    s.setup("cpr")
    return A, s


def test_wide_vcycle_fp64_matches_oracle(rsv, torch, problem):
    p = problem
    assert (p.nx + 1) // 2 * p.ny * p.nz >= 1 << 20  # the finest level takes the large-level forms
    A, s = _solver(rsv, p, "fp64")
    _, _, a7 = oracle.System.from_problem(p, pc="cpr").factors()
    b = np.random.default_rng(59).standard_normal(p.nb)
    st, e_or, _ = oracle.gmg_vcycle(p.nx, p.ny, p.nz, a7, b, max_levels=6, max_coarse=512, sweeps=2)
    assert st == 0
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    s.vcycle(bd, xd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"wide_vcycle_{p.nx}x{p.ny}x{p.nz}", per_entry_ratio(xd.cpu().numpy(), e_or), 1e-9)
    assert ratio <= 1e-9


def test_wide_cpr_apply_fp32_matches_oracle(rsv, torch, problem):
    """FP32 CPR-PF apply (its V-cycle on the large-level forms) against the oracle in FP64 on the
    same FP32-rounded data, per entry."""
    p = problem
    A, s = _solver(rsv, p, "mixed")
    of = oracle.System.from_problem(p, pc="cpr", float_round=True)
    f = np.random.default_rng(60).standard_normal(p.n).astype(np.float32)
    _, z_or = of.pc_apply(f.astype(np.float64))
    fd = torch.from_numpy(f).cuda()
    zd = torch.zeros_like(fd)
    s.apply(fd, zd)
    torch.cuda.synchronize()
    ratio = report_ratio(f"wide_cpr_apply_fp32_{p.nx}x{p.ny}x{p.nz}",
                         per_entry_ratio(zd.cpu().numpy().astype(np.float64), z_or), 1e-3)
    assert ratio <= 1e-3
