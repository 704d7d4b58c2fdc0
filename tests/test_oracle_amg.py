"""Pins of the oracle's algebraic multigrid (PMIS coarsening, direct interpolation,
Galerkin coarse operators, l1-Jacobi V-cycle) for the CPR pressure stage.

Section "Algebraic Multigrid Methods" (AMG setup algorithm: strength matrix,
coarse set, prolongation, R = P^T, A_{l+1} = R A_l P, smoothers; V-cycle
algorithm).  Each check uses something the oracle's code does not share:
properties that define the PMIS splitting, constants reproduced by direct
interpolation on a zero-row-sum operator, the dense triple product, the
V-cycle's dense error operator built from the hierarchy's parts, spectral
contraction on the Laplacian, and mutated copies of the oracle that the
dense pin must reject.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import stencil_to_dense
from tests.test_oracle_pins import _laplacian_a7

THETA = 0.5


def _pressure_a7(dims, seed):
    p = synth.make_problem(*dims, seed=seed)
    st, _, a7 = oracle.qi_setup(*dims, p.row_ptr, p.col_idx, p.vals)
    assert st == 0
    return a7


def _strength(A):
    """Dense strength matrix: S[i, j] when j != i and -a_ij >= theta max_{k != i} -a_ik > 0."""
    n = A.shape[0]
    off = -A.copy()
    np.fill_diagonal(off, -np.inf)
    mx = off.max(axis=1)
    S = np.zeros((n, n), dtype=bool)
    for i in range(n):
        if mx[i] > 0:
            S[i] = (off[i] >= THETA * mx[i]) & (A[i] != 0)
            S[i, i] = False
    return S


def _dense(rp, ci, v, ncols):
    n = len(rp) - 1
    M = np.zeros((n, ncols))
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            M[i, ci[q]] += v[q]
    return M


CASES = [((8, 6, 4), 17), ((10, 7, 5), 18), ((6, 6, 6), 19)]


def _measure(S):
    """PMIS measure lambda_i = |S_i^T| + u_i, u_i the top 53 bits of splitmix64 (Steele, Lea
    and Flood) of the point index, as a uniform in [0, 1)."""
    n = S.shape[0]
    z = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    return S.sum(axis=0) + u


@pytest.mark.parametrize("dims,seed", CASES)
def test_pmis_splitting_properties(dims, seed):
    """What PMIS guarantees: every point is decided; every F point either influences
    no point strongly (measure below 1) or strongly depends on a C point; and a C point
    depends strongly on another C point only when its own measure is the larger (a point
    that depends on an earlier C point is made F, and two C points chosen in one round
    are not strong neighbours)."""
    a7 = _pressure_a7(dims, seed)
    A = stencil_to_dense(*dims, a7)
    S = _strength(A)
    lam = _measure(S)
    cf, _, _ = oracle.amg_level(*dims, a7, 0, max_coarse=40)
    assert set(np.unique(cf)) <= {-1, 1} and (cf == 1).any() and (cf == -1).any()
    C = cf == 1
    for i in np.flatnonzero(~C):
        assert lam[i] < 1.0 or S[i, C].any(), i
    for j in np.flatnonzero(C):
        for i in np.flatnonzero(C & S[j]):
            assert lam[j] > lam[i], (j, i)
    # the measure's local maxima among all points are C points
    sym = S | S.T
    for i in range(len(cf)):
        nb = np.flatnonzero(sym[i])
        if lam[i] >= 1.0 and len(nb) and (lam[i] > lam[nb]).all():
            assert C[i], i


@pytest.mark.parametrize("dims,seed", CASES)
def test_direct_interpolation_and_galerkin_product(dims, seed):
    a7 = _pressure_a7(dims, seed)
    A = stencil_to_dense(*dims, a7)
    S = _strength(A)
    cf, (prp, pci, pv), (arp, aci, av) = oracle.amg_level(*dims, a7, 0, max_coarse=40)
    C = np.flatnonzero(cf == 1)
    nc = len(C)
    P = _dense(prp, pci, pv, nc)
    # C points: unit rows at their coarse index, in fine-index order
    assert np.array_equal(P[C], np.eye(nc))
    # F points: only strong C neighbours, with the direct-interpolation weights
    for i in np.flatnonzero(cf == -1):
        cols = np.flatnonzero(P[i])
        strong_c = [j for j in C if S[i, j]]
        assert set(C[cols]) <= set(strong_c)
        if len(cols):
            off = A[i].copy()
            off[i] = 0.0
            alpha = off.sum() / A[i, strong_c].sum()
            ref = -alpha * A[i, strong_c] / A[i, i]
            assert np.allclose(P[i, [list(C).index(j) for j in strong_c]], ref, rtol=1e-13)
    # Galerkin coarse operator: the dense triple product
    Ac = _dense(arp, aci, av, nc)
    assert np.allclose(Ac, P.T @ A @ P, rtol=1e-12, atol=1e-12 * np.abs(A).max())


def test_direct_interpolation_reproduces_constants_on_zero_row_sums():
    """On the Neumann Laplacian every row sums to zero, so each interpolated F row sums to 1."""
    dims = (8, 8, 6)
    a7 = _laplacian_a7(*dims, dirichlet=False)
    cf, (prp, pci, pv), _ = oracle.amg_level(*dims, a7, 0, max_coarse=40)
    P = _dense(prp, pci, pv, int((cf == 1).sum()))
    rows = P.sum(axis=1)
    interpolated = (P != 0).any(axis=1)
    assert interpolated.mean() > 0.95
    assert np.allclose(rows[interpolated], 1.0, rtol=1e-13)


def _l1_jacobi_vcycle_operator(dims, a7, sweeps, max_coarse, levels_P):
    """Dense B with e = B b for one AMG V-cycle from a zero guess, from dense parts:
    the hierarchy's prolongations, Galerkin products, l1-Jacobi sweeps and the exact
    coarsest inverse."""
    A = [stencil_to_dense(*dims, a7)]
    for P in levels_P:
        A.append(P.T @ A[-1] @ P)

    def cycle(l):
        Al = A[l]
        n = Al.shape[0]
        if l == len(A) - 1:
            return np.linalg.inv(Al)
        Dinv = np.diag(1.0 / np.abs(Al).sum(axis=1))
        eye = np.eye(n)
        X = np.zeros((n, n))
        for _ in range(sweeps):
            X = X + Dinv @ (eye - Al @ X)
        P = levels_P[l]
        X = X + P @ (cycle(l + 1) @ (P.T @ (eye - Al @ X)))
        for _ in range(sweeps):
            X = X + Dinv @ (eye - Al @ X)
        return X
    return cycle(0)


def _levels_P(dims, a7, max_coarse, nlev):
    Ps = []
    for l in range(nlev - 1):
        cf, (prp, pci, pv), _ = oracle.amg_level(*dims, a7, l, max_coarse=max_coarse)
        Ps.append(_dense(prp, pci, pv, int((cf == 1).sum())))
    return Ps


def _oracle_cycle_operator(vcycle, dims, a7, sweeps, max_coarse):
    n = int(np.prod(dims))
    cols = []
    nlev = None
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        st, x, nlev = vcycle(*dims, a7, e, max_coarse=max_coarse, sweeps=sweeps)
        assert st == 0
        cols.append(x)
    return np.column_stack(cols), nlev


@pytest.mark.parametrize("dims,sweeps", [((8, 6, 4), 2), ((6, 6, 6), 1), ((10, 7, 5), 3)])
def test_amg_vcycle_equals_dense_error_operator(dims, sweeps):
    a7 = _pressure_a7(dims, seed=21)
    max_coarse = 40
    levels = oracle.amg_hierarchy(*dims, a7, max_coarse=max_coarse)
    assert len(levels) >= 3
    Ps = _levels_P(dims, a7, max_coarse, len(levels))
    B_ref = _l1_jacobi_vcycle_operator(dims, a7, sweeps, max_coarse, Ps)
    B_or, nlev = _oracle_cycle_operator(oracle.amg_vcycle, dims, a7, sweeps, max_coarse)
    assert nlev == len(levels)
    assert np.max(np.abs(B_or - B_ref)) <= 1e-11 * np.max(np.abs(B_ref))


def test_amg_vcycle_contracts_on_laplacian_and_preconditions_gmres():
    dims = (10, 10, 8)
    a7 = _laplacian_a7(*dims, dirichlet=True)
    Ps = _levels_P(dims, a7, 40, len(oracle.amg_hierarchy(*dims, a7, max_coarse=40)))
    B = _l1_jacobi_vcycle_operator(dims, a7, 2, 40, Ps)
    A = stencil_to_dense(*dims, a7)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(A.shape[0]) - B @ A)))
    assert rho < 0.6, rho


# ----------------------------------------------------------- mutation checks

MUTATIONS = {
    # the plain Jacobi diagonal a_ii instead of the l1 row norm
    "jacobi_diagonal": ("g->dl1[q2][i] += fabs(g->A[q2].v[p]);",
                        "g->dl1[q2][i] += (g->A[q2].ci[p] == i) ? fabs(g->A[q2].v[p]) : 0.0;"),
    # no coarse correction below the finest level
    "no_correction_below_finest": ("g->x[l][f] += s;", "g->x[l][f] += (l >= 1) ? 0.0 : s;"),
    # post-smoothing dropped
    "no_post_smoothing": ("    for (int s = 0; s < g->sweeps; ++s) {\n        csr_residual(A, g->b[l], g->x[l], g->r[l]);\n"
                          "        for (int i = 0; i < n; ++i) g->x[l][i] += g->r[l][i] / g->dl1[l][i];\n    }\n    return OR_OK;",
                          "    return OR_OK;"),
}


def _mutant(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    c_path, so_path = tmp_path / f"o_{name}.c", tmp_path / f"libo_{name}.so"
    c_path.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so_path),
                           str(c_path), "-lm"])
    L = ctypes.CDLL(str(so_path))
    P, I = ctypes.c_void_p, ctypes.c_int
    L.or_amg_vcycle.restype = I
    L.or_amg_vcycle.argtypes = [I, I, I, P, I, I, I, P, P, P]

    def vcycle(nx, ny, nz, a7, rhs, max_levels=8, max_coarse=512, sweeps=2):
        a7 = np.ascontiguousarray(a7, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        e = np.zeros_like(rhs)
        nl = ctypes.c_int(0)
        st = L.or_amg_vcycle(nx, ny, nz, a7.ctypes.data, max_levels, max_coarse, sweeps, rhs.ctypes.data,
                             e.ctypes.data, ctypes.byref(nl))
        return st, e, nl.value
    return vcycle


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_dense_pin_rejects_mutated_amg_vcycle(tmp_path, name):
    dims, sweeps, max_coarse = (8, 6, 4), 2, 40
    a7 = _pressure_a7(dims, seed=21)
    levels = oracle.amg_hierarchy(*dims, a7, max_coarse=max_coarse)
    Ps = _levels_P(dims, a7, max_coarse, len(levels))
    B_ref = _l1_jacobi_vcycle_operator(dims, a7, sweeps, max_coarse, Ps)
    B_mut, _ = _oracle_cycle_operator(_mutant(tmp_path, name), dims, a7, sweeps, max_coarse)
    assert np.max(np.abs(B_mut - B_ref)) > 1e-8 * np.max(np.abs(B_ref)), name


def test_cpr_with_amg_pressure_stage_solves_to_the_dense_solution():
    p = synth.make_problem(9, 7, 6, seed=27)
    s = oracle.System.from_problem(p, pc="cpr", coarsening="amg", gmg_levels=8, gmg_coarse=40)
    assert s.setup_status == 0 and s.gmg_levels() >= 3
    st, x, info = s.gmres(p.b, rtol=1e-10, maxit=500)
    from tests.helpers import bsr_to_dense
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    assert st == 0 and np.linalg.norm(p.b - A @ x) <= 1e-10 * np.linalg.norm(p.b)
    assert np.allclose(x, np.linalg.solve(A, p.b), rtol=1e-6, atol=1e-8)
