"""Batched independent solves (one block-diagonal matrix, per-system BiCGSTAB) against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsv():
    from tests.helpers import build_library
    build_library()
    import paper_1602_05901_gb300 as m
    return m


def _batch_problems(dims_list, seed0=1000):
    return [synth.make_problem(*d, seed=seed0 + s) for s, d in enumerate(dims_list)]


def _concat(probs):
    vals = np.concatenate([p.vals for p in probs])
    b = np.concatenate([p.b for p in probs])
    return vals, b


DIMS = [(8, 6, 4), (12, 5, 7), (3, 3, 3), (16, 9, 5), (1, 1, 1), (20, 20, 10), (9, 17, 6)]


def test_batch_pattern_is_block_diagonal(rsv):
    probs = _batch_problems(DIMS)
    A = rsv.Matrix.batch(DIMS)
    assert A.nsys == len(DIMS)
    off = 0
    rp_all, ci_all = A.row_ptr, A.col_idx
    for p, c0 in zip(probs, A.cell_offsets[:-1]):
        assert c0 == off
        rows = slice(off, off + p.nb)
        rp = rp_all[off:off + p.nb + 1] - rp_all[off]
        assert np.array_equal(rp, p.row_ptr)
        assert np.array_equal(ci_all[rp_all[off]:rp_all[off + p.nb]] - off, p.col_idx)
        off += p.nb
    assert A.cell_offsets[-1] == off


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("pc", ["bilu0", "bjacobi"])
def test_batched_bicgstab_matches_per_system_oracle(rsv, precision, pc):
    import torch
    probs = _batch_problems(DIMS)
    vals, b = _concat(probs)
    A = rsv.Matrix.batch(DIMS)
    A.set_values(vals)
    s = rsv.Solver(A, solver="bicgstab", precision=precision, rtol=1e-8, maxit=4000)
    s.setup(pc)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, infos = s.solve_batched(bd, x)
    assert st == rsv.RSV_OK, (st, infos)
    xh = x.cpu().numpy()
    off = 0
    for p, info in zip(probs, infos):
        xs = xh[3 * off:3 * (off + p.nb)]
        rel = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, xs)) / np.linalg.norm(p.b)
        assert rel <= 1e-8 and abs(rel - info["true_relres"]) <= 1e-12 * max(1.0, rel / 1e-8), (rel, info)
        assert info["status"] == 0
        if precision == "fp64":
            its = []
            for t in range(6):
                bb = p.b if t == 0 else p.b * (1 + 1e-15 * np.random.default_rng(2000 + t).standard_normal(p.n))
                ost, _, oinfo = oracle.System.from_problem(p, pc=pc).bicgstab(bb, maxit=4000)
                assert ost == 0
                its.append(oinfo["iters"])
            assert 0.9 * min(its) - 2 <= info["iters"] <= 1.1 * max(its) + 2, (info, its)
        else:
            assert info["outer_iters"] >= 1
        off += p.nb


def test_batch_matches_single_system_solves(rsv):
    """The same systems solved one by one (rsv_solve) need the same iterations (within rounding)."""
    import torch
    probs = _batch_problems(DIMS[:4], seed0=3000)
    vals, b = _concat(probs)
    A = rsv.Matrix.batch(DIMS[:4])
    A.set_values(vals)
    s = rsv.Solver(A, solver="bicgstab", precision="fp64")
    s.setup("bilu0")
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    st, infos = s.solve_batched(torch.from_numpy(b).cuda(), x)
    assert st == 0
    for p, info in zip(probs, infos):
        Ai = rsv.Matrix(p.nx, p.ny, p.nz)
        Ai.set_values(p.vals)
        si = rsv.Solver(Ai, solver="bicgstab", precision="fp64")
        si.setup("bilu0")
        xi = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        sti, ii = si.solve(torch.from_numpy(p.b).cuda(), xi)
        assert sti == 0
        assert abs(ii["iters"] - info["iters"]) <= max(3, 0.15 * ii["iters"]), (ii, info)


def test_batch_64_uneven_systems_mixed(rsv):
    """The 64-system ensemble recipe at reduced sizes (every grid halved per dimension)."""
    import torch
    dims = [(max(2, a // 2), max(2, b_ // 2), max(2, c // 2)) for a, b_, c in synth.batch_sizes()]
    probs = _batch_problems(dims)
    vals, b = _concat(probs)
    A = rsv.Matrix.batch(dims)
    A.set_values(vals)
    s = rsv.Solver(A, solver="bicgstab", precision="mixed", maxit=4000)
    s.setup("bilu0")
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    st, infos = s.solve_batched(torch.from_numpy(b).cuda(), x)
    assert st == 0, [i for i in infos if i["status"]]
    xh = x.cpu().numpy()
    off = 0
    for p, info in zip(probs, infos):
        xs = xh[3 * off:3 * (off + p.nb)]
        rel = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, xs)) / np.linalg.norm(p.b)
        assert rel <= 1e-8
        off += p.nb


def test_batch_64_uneven_systems_full_size(rsv):
    """The 64-system ensemble at its full sizes (grids from 16^3 to 96x96x48, 6.17M cells,
    18.5M unknowns): BiCGSTAB + block ILU(0), FP32 inner solves under FP64 refinement, one
    batched call; every system's true residual, recomputed by the oracle's SpMV of that
    system alone, meets rtol 1e-8, and no system runs away toward maxit (every count stays
    below 1,000)."""
    import torch
    dims = synth.batch_sizes()
    probs = _batch_problems(dims)
    vals, b = _concat(probs)
    A = rsv.Matrix.batch(dims)
    assert A.nb == sum(p.nb for p in probs) == 6171613
    A.set_values(torch.from_numpy(vals).cuda())
    del vals
    s = rsv.Solver(A, solver="bicgstab", precision="mixed", rtol=1e-8, maxit=4000)
    s.setup("bilu0")
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    st, infos = s.solve_batched(torch.from_numpy(b).cuda(), x)
    assert st == 0, [i for i in infos if i["status"]]
    xh = x.cpu().numpy()
    off = 0
    its = []
    for p, info in zip(probs, infos):
        xs = xh[3 * off:3 * (off + p.nb)]
        rel = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, xs)) / np.linalg.norm(p.b)
        assert rel <= 1e-8 and abs(rel - info["true_relres"]) <= 1e-12 * max(1.0, rel / 1e-8), (rel, info)
        assert info["status"] == 0 and info["outer_iters"] >= 1
        its.append(info["iters"])
        off += p.nb
    assert max(its) < 1000, its
    print(f"BATCH64_FULL iters min/median/max {min(its)}/{int(np.median(its))}/{max(its)}")
