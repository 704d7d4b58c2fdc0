"""Pins of the CPU oracle against mathematics it does not share code with.

Each test checks one oracle routine against something fixed independently of
it: dense linear algebra (numpy/LAPACK), closed-form spectra, defining
properties of the method (the ILU(0) pattern identity, Galerkin triple
products, finite termination of GMRES) or invariants of the inputs.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import bsr_to_dense, kron_bsr, stencil_to_dense

TINY = [(2, 2, 1), (3, 2, 2), (4, 3, 2)]


def _prob(dims, seed=0):
    return synth.make_problem(*dims, seed=seed)


# ---------------------------------------------------------------- SpMV

@pytest.mark.parametrize("dims", TINY + [(5, 1, 1)])
def test_spmv_equals_dense_product(dims):
    p = _prob(dims)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(p.n), rng.standard_normal(p.n)
    got = oracle.spmv(p.row_ptr, p.col_idx, p.vals, x, alpha=-0.7, beta=1.3, y=y)
    ref = -0.7 * (A @ x) + 1.3 * y
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(A).sum(1).max())
    assert np.allclose(oracle.spmv(p.row_ptr, p.col_idx, p.vals, x), A @ x, rtol=1e-13, atol=1e-9)


def test_blas1():
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(1001), rng.standard_normal(1001)
    assert abs(oracle.dot(x, y) - np.dot(x, y)) < 1e-12 * np.abs(x * y).sum()
    assert abs(oracle.norm2(x) - np.linalg.norm(x)) < 1e-13 * np.linalg.norm(x)


# ------------------------------------------------------- dense + 3x3 inverse

def test_inv3_and_dense_solve():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.standard_normal((3, 3))
        st, ai = oracle.inv3(a)
        assert st == 0 and np.allclose(ai, np.linalg.inv(a), rtol=1e-10, atol=1e-12)
    st, _ = oracle.inv3(np.array([[1.0, 2, 3], [2, 4, 6], [0, 1, 1]]))
    assert st == oracle.ESINGULAR
    A = rng.standard_normal((40, 40)) + 40 * np.eye(40)
    b = rng.standard_normal(40)
    st, x = oracle.dense_solve(A, b)
    assert st == 0 and np.allclose(x, np.linalg.solve(A, b), rtol=1e-12)
    # a zero leading pivot needs the row exchange
    P = np.array([[0.0, 1.0], [1.0, 0.0]])
    st, x = oracle.dense_solve(P, np.array([2.0, 3.0]))
    assert st == 0 and np.allclose(x, [3.0, 2.0])


# ------------------------------------------------------------ block Jacobi

def test_block_jacobi_inverts_diagonal_blocks():
    p = _prob((4, 3, 2))
    st, dinv = oracle.bj_setup(p.row_ptr, p.col_idx, p.vals)
    assert st == 0
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    for c in range(p.nb):
        assert np.allclose(dinv[c] @ A[3 * c:3 * c + 3, 3 * c:3 * c + 3], np.eye(3), atol=1e-12)
    r = np.random.default_rng(4).standard_normal(p.n)
    z = oracle.bj_apply(dinv, r)
    D = np.zeros_like(A)
    for c in range(p.nb):
        D[3 * c:3 * c + 3, 3 * c:3 * c + 3] = A[3 * c:3 * c + 3, 3 * c:3 * c + 3]
    assert np.allclose(z, np.linalg.solve(D, r), rtol=1e-10, atol=1e-14)


# ------------------------------------------------------------ block ILU(0)

def _ilu_dense(p, lu, udinv):
    nb = p.nb
    L = np.eye(3 * nb)
    U = np.zeros((3 * nb, 3 * nb))
    for r in range(nb):
        for q in range(p.row_ptr[r], p.row_ptr[r + 1]):
            c = p.col_idx[q]
            blk = lu[q]
            if c < r:
                L[3 * r:3 * r + 3, 3 * c:3 * c + 3] = blk
            else:
                U[3 * r:3 * r + 3, 3 * c:3 * c + 3] = blk
    return L, U


@pytest.mark.parametrize("dims", TINY + [(3, 3, 3)])
def test_ilu0_matches_a_on_pattern(dims):
    """Defining property of ILU(0): (LU)_ij = A_ij on every block of pattern(A)."""
    p = _prob(dims, seed=5)
    st, lu, udinv, off = oracle.bilu0_setup(p.row_ptr, p.col_idx, p.vals)
    assert st == 0
    assert off == 0  # seven-point graph has no triangles: only diagonal blocks change
    L, U = _ilu_dense(p, lu, udinv)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    LU = L @ U
    mask = np.zeros_like(A, dtype=bool)
    for r in range(p.nb):
        for q in range(p.row_ptr[r], p.row_ptr[r + 1]):
            c = p.col_idx[q]
            mask[3 * r:3 * r + 3, 3 * c:3 * c + 3] = True
    assert np.allclose(LU[mask], A[mask], rtol=1e-12, atol=1e-10)
    for c in range(p.nb):
        assert np.allclose(udinv[c] @ U[3 * c:3 * c + 3, 3 * c:3 * c + 3], np.eye(3), atol=1e-10)
    r = np.random.default_rng(6).standard_normal(p.n)
    z = oracle.bilu0_apply(p.row_ptr, p.col_idx, lu, udinv, r)
    assert np.allclose(z, np.linalg.solve(LU, r), rtol=1e-9, atol=1e-12)


def test_ilu0_is_exact_lu_in_one_dimension():
    """On an n x 1 x 1 grid the matrix is block tridiagonal and ILU(0) is exact."""
    p = _prob((9, 1, 1), seed=7)
    st, lu, udinv, _ = oracle.bilu0_setup(p.row_ptr, p.col_idx, p.vals)
    L, U = _ilu_dense(p, lu, udinv)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    assert np.allclose(L @ U, A, rtol=1e-12, atol=1e-10)
    s = oracle.System.from_problem(p, pc="bilu0")
    st, x, info = s.gmres(p.b, rtol=1e-12)
    assert st == 0 and info["iters"] == 1
    assert np.allclose(x, np.linalg.solve(A, p.b), rtol=1e-10)


# ------------------------------------------------- quasi-IMPES, Pi_r, Pi_p

def test_qi_reduces_to_pressure_block_when_diagonal_blocks_are_diagonal():
    nx, ny, nz = 3, 2, 2
    rp, ci, vals = kron_bsr(nx, ny, nz, np.diag([2.0, 3.0, 4.0]), np.diag([0.5, 0.6, 0.7]),
                            trans=lambda r, c: 1.0 + 0.1 * (r + c))
    st, w, a7 = oracle.qi_setup(nx, ny, nz, rp, ci, vals)
    assert st == 0
    assert np.allclose(w, np.tile([1.0, 0.0, 0.0], (nx * ny * nz, 1)))
    A = bsr_to_dense(rp, ci, vals)
    App = A[0::3, 0::3]
    assert np.allclose(stencil_to_dense(nx, ny, nz, a7), App)


@pytest.mark.parametrize("dims", TINY)
def test_qi_pressure_matrix_is_weighted_product(dims):
    """A_pp = W A Pi_p with W = blockdiag(w_i^T), as an explicit dense product."""
    p = _prob(dims, seed=8)
    st, w, a7 = oracle.qi_setup(*dims, p.row_ptr, p.col_idx, p.vals)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    W = np.zeros((p.nb, p.n))
    Pp = np.zeros((p.n, p.nb))
    for c in range(p.nb):
        W[c, 3 * c:3 * c + 3] = w[c]
        Pp[3 * c, c] = 1.0
        d = A[3 * c:3 * c + 3, 3 * c:3 * c + 3]
        # the weights cancel the diagonal-block coupling of each secondary unknown's
        # own equation into the pressure column (diagonal approximation)
        assert np.isclose(w[c, 1] * d[1, 1], -d[0, 1]) and np.isclose(w[c, 2] * d[2, 2], -d[0, 2])
    assert np.allclose(stencil_to_dense(*dims, a7), W @ A @ Pp, rtol=1e-12, atol=1e-9)
    r = np.random.default_rng(9).standard_normal(p.n)
    assert np.allclose(oracle.restrict_pressure(w, r), W @ r)
    q = np.random.default_rng(10).standard_normal(p.nb)
    assert np.array_equal(oracle.restrict_pressure(np.tile([1.0, 0, 0], (p.nb, 1)),
                                                   oracle.prolong_pressure(q)), q)
    assert np.array_equal(oracle.prolong_pressure(q), Pp @ q)


# --------------------------------------------------------------- Laplacian

def _laplacian_a7(nx, ny, nz, dirichlet):
    """Scalar seven-point Laplacian; Dirichlet adds a ghost-face coefficient per missing face."""
    a7 = np.zeros((nx * ny * nz, 7))
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), None, (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    for c in range(nx * ny * nz):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        for s, o in enumerate(offs):
            if o is None:
                continue
            ii, jj, kk = i + o[0], j + o[1], k + o[2]
            inside = 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz
            if inside:
                a7[c, s] = -1.0
                a7[c, 3] += 1.0
            elif dirichlet:
                a7[c, 3] += 1.0
    return a7


@pytest.mark.parametrize("dims", [(4, 3, 2), (5, 5, 3), (6, 4, 4)])
def test_stencil_operator_has_closed_form_laplacian_spectrum(dims):
    nx, ny, nz = dims
    for dirichlet in (True, False):
        a7 = _laplacian_a7(nx, ny, nz, dirichlet)
        n = nx * ny * nz
        A = np.column_stack([oracle.stencil_apply(nx, ny, nz, a7, e) for e in np.eye(n)])
        ev = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))
        if dirichlet:
            f = [4 * np.sin(np.pi * np.arange(1, d + 1) / (2 * (d + 1))) ** 2 for d in dims]
        else:
            f = [4 * np.sin(np.pi * np.arange(0, d) / (2 * d)) ** 2 for d in dims]
        ref = np.sort((f[0][None, None, :] + f[1][None, :, None] + f[2][:, None, None]).ravel())
        assert np.allclose(A, A.T)
        assert np.allclose(ev, ref, atol=1e-12)


def test_bsr_spmv_kron_laplacian_spectrum():
    """With M = I and zero accumulation the Jacobian is L (x) I_3 (Neumann L)."""
    nx, ny, nz = 4, 3, 2
    rp, ci, vals = kron_bsr(nx, ny, nz, np.eye(3), np.zeros((3, 3)))
    n = 3 * nx * ny * nz
    A = np.column_stack([oracle.spmv(rp, ci, vals, e) for e in np.eye(n)])
    f = [4 * np.sin(np.pi * np.arange(0, d) / (2 * d)) ** 2 for d in (nx, ny, nz)]
    lam = (f[0][None, None, :] + f[1][None, :, None] + f[2][:, None, None]).ravel()
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(np.repeat(lam, 3)), atol=1e-12)


# --------------------------------------------------------- multigrid pieces

@pytest.mark.parametrize("dims", [(4, 4, 2), (5, 3, 3), (3, 1, 2)])
def test_galerkin_coarsening_is_triple_product(dims):
    nx, ny, nz = dims
    p = _prob(dims, seed=11)
    _, _, a7 = oracle.qi_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals)
    (cx, cy, cz), ac = oracle.gmg_coarsen(nx, ny, nz, a7)
    P = np.zeros((nx * ny * nz, cx * cy * cz))
    for c in range(nx * ny * nz):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        P[c, cx * cy * (k // 2) + cx * (j // 2) + i // 2] = 1.0
    A = stencil_to_dense(nx, ny, nz, a7)
    assert np.allclose(stencil_to_dense(cx, cy, cz, ac), P.T @ A @ P, rtol=1e-12, atol=1e-9)


def test_red_black_gs_equals_serial_gs_in_colour_order():
    nx, ny, nz = 5, 4, 3
    p = _prob((nx, ny, nz), seed=12)
    _, _, a7 = oracle.qi_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals)
    A = stencil_to_dense(nx, ny, nz, a7)
    rng = np.random.default_rng(13)
    b, x0 = rng.standard_normal(nx * ny * nz), rng.standard_normal(nx * ny * nz)
    x = oracle.gs_colour(nx, ny, nz, a7, b, x0, 0)
    x = oracle.gs_colour(nx, ny, nz, a7, b, x, 1)
    colour = np.array([(c % nx + (c // nx) % ny + c // (nx * ny)) % 2 for c in range(nx * ny * nz)])
    perm = np.concatenate([np.flatnonzero(colour == 0), np.flatnonzero(colour == 1)])
    Ap, bp, xp = A[np.ix_(perm, perm)], b[perm], x0[perm]
    Lw = np.tril(Ap)  # forward Gauss-Seidel in the red-then-black order
    ref = np.linalg.solve(Lw, bp - np.triu(Ap, 1) @ xp)
    assert np.allclose(x[perm], ref, rtol=1e-12, atol=1e-12)


def test_vcycle_single_level_is_exact_and_two_grid_reduces_error():
    nx, ny, nz = 6, 6, 4
    a7 = _laplacian_a7(nx, ny, nz, dirichlet=True)
    A = stencil_to_dense(nx, ny, nz, a7)
    rhs = np.random.default_rng(14).standard_normal(nx * ny * nz)
    st, e, nl = oracle.gmg_vcycle(nx, ny, nz, a7, rhs, max_levels=1)
    assert st == 0 and nl == 1 and np.allclose(e, np.linalg.solve(A, rhs), rtol=1e-12)
    st, e, nl = oracle.gmg_vcycle(nx, ny, nz, a7, rhs, max_levels=2, max_coarse=1)
    assert nl == 2
    x_true = np.linalg.solve(A, rhs)
    # error propagation of one V-cycle as an iteration: ||x - V(b)||_A < ||x||_A
    err = x_true - e
    assert err @ A @ err < 0.5 * (x_true @ A @ x_true)
    # the level rule: halve while above max_coarse cells, at most max_levels levels
    st, e, nl = oracle.gmg_vcycle(nx, ny, nz, a7, rhs, max_levels=6, max_coarse=8)
    assert nl == 3  # 144 -> 18 -> 4 cells (3x3x2 -> 2x2x1)


# -------------------------------------------------------------------- CPR

def test_cpr_pressure_stage_exact_on_component_decoupled_system():
    """If every block is diagonal the pressure stage with an exact coarse solve
    gives the exact pressure, and the full stage does not disturb it."""
    nx, ny, nz = 4, 3, 2
    rp, ci, vals = kron_bsr(nx, ny, nz, np.diag([1.0, 0.5, 0.3]), np.diag([0.2, 0.4, 0.6]),
                            trans=lambda r, c: 1.0 + ((r * 7 + c * 3) % 5))
    s = oracle.System(nx, ny, nz, rp, ci, vals, pc="cpr", gmg_levels=1)
    assert s.setup_status == 0 and s.gmg_levels() == 1
    A = bsr_to_dense(rp, ci, vals)
    f = np.random.default_rng(15).standard_normal(3 * nx * ny * nz)
    st, x = s.pc_apply(f)
    assert st == 0
    assert np.allclose(x[0::3], np.linalg.solve(A[0::3, 0::3], f[0::3]), rtol=1e-10)


def test_cpr_apply_matches_dense_two_stage_formula():
    nx, ny, nz = 4, 3, 2
    p = _prob((nx, ny, nz), seed=16)
    s = oracle.System.from_problem(p, pc="cpr", gmg_levels=1)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    _, w, a7 = s.factors()
    st, lu, udinv, _ = oracle.bilu0_setup(p.row_ptr, p.col_idx, p.vals)
    L, U = _ilu_dense(p, lu, udinv)
    App = stencil_to_dense(nx, ny, nz, a7)
    W = np.zeros((p.nb, p.n))
    for c in range(p.nb):
        W[c, 3 * c:3 * c + 3] = w[c]
    f = np.random.default_rng(17).standard_normal(p.n)
    x1 = np.zeros(p.n)
    x1[0::3] = np.linalg.solve(App, W @ f)
    ref = x1 + np.linalg.solve(L @ U, f - A @ x1)
    st, x = s.pc_apply(f)
    assert st == 0 and np.allclose(x, ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("dims", [(4, 3, 2), (7, 5, 3)])
def test_abf_weights_are_first_row_of_diagonal_block_inverse(dims):
    """ABF premultiplies each block row by the inverse of its diagonal block, so the
    pressure weights are the first row of D^{-1} (checked against numpy's inverse),
    every pressure-matrix diagonal entry is exactly (D^{-1} D)_00 = 1 up to rounding,
    and A_pp is the weighted product W A P."""
    p = _prob(dims, seed=22)
    nx, ny, nz = dims
    st, w, a7 = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "abf")
    assert st == 0
    for c in range(p.nb):
        q = next(q for q in range(p.row_ptr[c], p.row_ptr[c + 1]) if p.col_idx[q] == c)
        assert np.allclose(w[c], np.linalg.inv(p.vals[q])[0], rtol=1e-12, atol=1e-14 * np.abs(w[c]).max())
    assert np.allclose(a7[:, 3], 1.0, rtol=0, atol=1e-12)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    W = np.zeros((p.nb, p.n))
    for c in range(p.nb):
        W[c, 3 * c:3 * c + 3] = w[c]
    assert np.allclose(stencil_to_dense(nx, ny, nz, a7), W @ A[:, 0::3], rtol=1e-12, atol=1e-12)
    # the quasi-IMPES reading is unchanged by the switch
    st, wq, _ = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "qi")
    st2, wq2, _ = oracle.qi_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals)
    assert st == 0 and st2 == 0 and np.array_equal(wq, wq2)


def test_abf_pressure_stage_exact_on_component_decoupled_system():
    """Diagonal blocks: ABF weights are (1/D00, 0, 0), and the pressure stage with an
    exact coarse solve returns the exact pressure."""
    nx, ny, nz = 4, 3, 2
    rp, ci, vals = kron_bsr(nx, ny, nz, np.diag([1.0, 0.5, 0.3]), np.diag([0.2, 0.4, 0.6]),
                            trans=lambda r, c: 1.0 + ((r * 7 + c * 3) % 5))
    s = oracle.System(nx, ny, nz, rp, ci, vals, pc="cpr", gmg_levels=1, decoupling="abf")
    assert s.setup_status == 0
    A = bsr_to_dense(rp, ci, vals)
    f = np.random.default_rng(23).standard_normal(3 * nx * ny * nz)
    st, x = s.pc_apply(f)
    assert st == 0
    assert np.allclose(x[0::3], np.linalg.solve(A[0::3, 0::3], f[0::3]), rtol=1e-10)


@pytest.mark.parametrize("dims", [(4, 3, 2), (7, 5, 3)])
def test_true_impes_weights_remove_secondary_unknowns_from_accumulation(dims):
    """True-IMPES takes the weights from each cell's accumulation block C_c:
    w_c = first row of C_c^{-1} (numpy's inverse), so w_c C_c = (1, 0, 0), and A_pp
    is the weighted product W A P.  With C_c = D_c (the diagonal block of A) it is
    ABF exactly; with the generator's diagonal accumulation blocks the weights are
    (1/C_00, 0, 0) and A_pp is the pressure-pressure block scaled per row."""
    p = _prob(dims, seed=24)
    nx, ny, nz = dims
    rng = np.random.default_rng(25)
    C = rng.standard_normal((p.nb, 3, 3)) + 3 * np.eye(3)
    st, w, a7 = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "timpes", acc=C)
    assert st == 0
    for c in range(p.nb):
        assert np.allclose(w[c], np.linalg.inv(C[c])[0], rtol=1e-12, atol=1e-14 * np.abs(w[c]).max())
        assert np.allclose(w[c] @ C[c], [1.0, 0.0, 0.0], atol=1e-12)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    W = np.zeros((p.nb, p.n))
    for c in range(p.nb):
        W[c, 3 * c:3 * c + 3] = w[c]
    assert np.allclose(stencil_to_dense(nx, ny, nz, a7), W @ A[:, 0::3], rtol=1e-12, atol=1e-12)
    # C = D: the ABF weights
    D = np.stack([p.vals[next(q for q in range(p.row_ptr[c], p.row_ptr[c + 1]) if p.col_idx[q] == c)]
                  for c in range(p.nb)])
    _, w_d, a7_d = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "timpes", acc=D)
    _, w_abf, a7_abf = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "abf")
    assert np.array_equal(w_d, w_abf) and np.array_equal(a7_d, a7_abf)
    # the generator's accumulation blocks are diagonal
    acc = p.accumulation()
    _, w_g, a7_g = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "timpes", acc=acc)
    assert np.allclose(w_g[:, 0], 1.0 / acc[:, 0, 0], rtol=1e-15) and np.all(w_g[:, 1:] == 0.0)
    assert np.allclose(stencil_to_dense(nx, ny, nz, a7_g), A[0::3, 0::3] / acc[:, 0, 0][:, None], rtol=1e-13)
    # without accumulation blocks true-IMPES is refused
    st, _, _ = oracle.decouple_setup(nx, ny, nz, p.row_ptr, p.col_idx, p.vals, "timpes")
    assert st == oracle.EINVAL


def test_true_impes_cpr_solves_to_the_dense_solution():
    p = _prob((6, 5, 4), seed=26)
    s = oracle.System.from_problem(p, pc="cpr", decoupling="timpes", acc=p.accumulation())
    assert s.setup_status == 0
    st, x, info = s.gmres(p.b, rtol=1e-10, maxit=500)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    assert st == 0 and np.allclose(x, np.linalg.solve(A, p.b), rtol=1e-7, atol=1e-9)


CPR_ORDERS = [("cpr", "PF"), ("cpr_fp", "FP"), ("cpr_fpf", "FPF"), ("cpr_ffpf", "FFPF")]


@pytest.mark.parametrize("pc,stages", CPR_ORDERS)
def test_cpr_order_error_operator_is_product_of_stage_error_operators(pc, stages):
    """Section "CPR-like preconditioners" (Algorithms CPR-FP, CPR-PF, CPR-FPF,
    CPR-FFPF): every stage after the first acts on the residual f - A x and adds
    to x, so the error operator I - M^{-1} A is the product of the stages' error
    operators I - B A, the last stage leftmost.  The stage operators are formed
    densely and independently of the oracle's apply: B_F = (LU)^{-1} from the
    ILU(0) factors, B_P = Pi_p A_pp^{-1} Pi_r from the pressure stencil (one
    level, so the V-cycle is an exact solve).  A stage in the wrong place, a
    residual of the wrong sign or a stage that overwrites x fails."""
    nx, ny, nz = 4, 3, 2
    p = _prob((nx, ny, nz), seed=18)
    s = oracle.System.from_problem(p, pc=pc, gmg_levels=1)
    assert s.setup_status == 0 and s.gmg_levels() == 1
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    _, w, a7 = s.factors()
    st, lu, udinv, _ = oracle.bilu0_setup(p.row_ptr, p.col_idx, p.vals)
    assert st == 0
    L, U = _ilu_dense(p, lu, udinv)
    App = stencil_to_dense(nx, ny, nz, a7)
    W = np.zeros((p.nb, p.n))
    Pp = np.zeros((p.n, p.nb))
    for c in range(p.nb):
        W[c, 3 * c:3 * c + 3] = w[c]
        Pp[3 * c, c] = 1.0
    I = np.eye(p.n)
    B = {"F": np.linalg.inv(L @ U), "P": Pp @ np.linalg.solve(App, W)}
    E = I.copy()
    for stage in stages:
        E = (I - B[stage] @ A) @ E
    Minv = np.zeros((p.n, p.n))
    for i in range(p.n):
        st, Minv[:, i] = s.pc_apply(I[i])
        assert st == 0
    assert np.allclose(I - Minv @ A, E, rtol=0, atol=1e-9 * max(1.0, np.abs(E).max()))


@pytest.mark.parametrize("pc,stages", CPR_ORDERS)
def test_cpr_orders_are_exact_where_ilu0_is_exact(pc, stages):
    """On a one-cell-wide grid the matrix is block tridiagonal, ILU(0) is its exact
    LU, and so every CPR order (each ends with a full stage, or starts with one
    and the later stages see a zero residual) returns A^{-1} f."""
    p = _prob((40, 1, 1), seed=19)
    s = oracle.System.from_problem(p, pc=pc)
    assert s.setup_status == 0
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    f = np.random.default_rng(20).standard_normal(p.n)
    st, x = s.pc_apply(f)
    assert st == 0
    ref = np.linalg.solve(A, f)
    assert np.allclose(x, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("pc", ["cpr_fp", "cpr_fpf", "cpr_ffpf"])
def test_cpr_orders_precondition_gmres_to_the_dense_solution(pc):
    p = _prob((10, 8, 4), seed=21)
    s = oracle.System.from_problem(p, pc=pc)
    st, x, info = s.gmres(p.b, rtol=1e-10, maxit=500)
    assert st == 0
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    assert np.linalg.norm(A @ x - p.b) <= 1.0001e-10 * np.linalg.norm(p.b)


# ----------------------------------------------------------------- Krylov

def test_gmres_finite_termination():
    """Without restarts GMRES solves an n x n system in at most n steps."""
    p = _prob((2, 2, 1), seed=18)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    s = oracle.System.from_problem(p, pc="none")
    st, x, info = s.gmres(p.b, m=p.n, rtol=1e-13, maxit=p.n)
    assert st == 0 and info["iters"] <= p.n
    assert np.allclose(x, np.linalg.solve(A, p.b), rtol=1e-9)


def test_gmres_steps_bounded_by_distinct_eigenvalues():
    nx, ny, nz = 4, 3, 2
    rp, ci, vals = kron_bsr(nx, ny, nz, np.eye(3), 0.5 * np.eye(3))
    s = oracle.System(nx, ny, nz, rp, ci, vals, pc="none")
    b = np.random.default_rng(19).standard_normal(3 * nx * ny * nz)
    f = [4 * np.sin(np.pi * np.arange(0, d) / (2 * d)) ** 2 for d in (nx, ny, nz)]
    lam = np.unique(np.round((f[0][None, None, :] + f[1][None, :, None] + f[2][:, None, None]).ravel(), 9))
    st, x, info = s.gmres(b, m=60, rtol=1e-11, maxit=60)
    assert st == 0 and info["iters"] <= len(lam)


@pytest.mark.parametrize("pc", ["none", "bjacobi", "bilu0", "cpr"])
def test_solvers_reach_dense_solution(pc):
    dims = (4, 3, 3)
    p = _prob(dims, seed=20)
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    xref = np.linalg.solve(A, p.b)
    s = oracle.System.from_problem(p, pc=pc)
    assert s.setup_status == 0
    for solve in (lambda: s.gmres(p.b, rtol=1e-12, maxit=3000),
                  lambda: s.gmres(p.b, rtol=1e-12, maxit=3000, flexible=True),
                  lambda: s.bicgstab(p.b, rtol=1e-12, maxit=3000)):
        st, x, info = solve()
        assert st == 0, info
        assert np.linalg.norm(p.b - A @ x) <= 1.0001e-12 * np.linalg.norm(p.b)
        assert abs(info["relres"] - np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b)) < 1e-14
        assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)


def test_fgmres_with_fixed_preconditioner_matches_gmres():
    p = _prob((5, 4, 3), seed=21)
    s = oracle.System.from_problem(p, pc="bilu0")
    st1, x1, i1 = s.gmres(p.b, m=10, rtol=1e-10)
    st2, x2, i2 = s.gmres(p.b, m=10, rtol=1e-10, flexible=True)
    assert st1 == st2 == 0 and abs(i1["iters"] - i2["iters"]) <= 1
    assert np.linalg.norm(x1 - x2) <= 1e-7 * np.linalg.norm(x1)


def test_gmres_reports_noconv_and_keeps_iterate():
    p = _prob((6, 5, 4), seed=22)
    s = oracle.System.from_problem(p, pc="none")
    st, x, info = s.gmres(p.b, m=5, rtol=1e-12, maxit=7)
    assert st == oracle.ENOCONV and info["iters"] == 7 and info["relres"] < 1.0


def test_bicgstab_breakdown_on_orthogonal_shadow():
    """A skew matrix with r orthogonal to A r makes <rh, v> vanish: breakdown reported."""
    nx, ny, nz = 2, 1, 1
    rp, ci = synth.seven_point_pattern(nx, ny, nz)
    vals = np.zeros((len(ci), 3, 3))
    S = np.array([[0.0, 1, 0], [-1, 0, 0], [0, 0, 0]])
    for q in range(len(ci)):
        vals[q] = S if ci[q] == 0 and q < 2 else np.zeros((3, 3))
    vals[0] = np.array([[0.0, 1, 0], [-1, 0, 0], [0, 0, 1.0]])
    vals[3] = np.eye(3)
    s = oracle.System(nx, ny, nz, rp, ci, vals, pc="none")
    b = np.array([1.0, 0, 0, 0, 0, 0])
    st, x, info = s.bicgstab(b, rtol=1e-12, btol=1e-30)
    assert st == oracle.EBREAKDOWN


def test_mixed_refinement_reaches_fp64_tolerance():
    p = _prob((8, 6, 4), seed=23)
    outer = oracle.System.from_problem(p, pc="none")
    inner = oracle.System.from_problem(p, pc="bilu0", float_round=True)
    st, x, info = oracle.refine(outer, inner, p.b, solver="gmres")
    A = bsr_to_dense(p.row_ptr, p.col_idx, p.vals)
    assert st == 0 and info["outer"] >= 2
    assert np.linalg.norm(p.b - A @ x) <= 1e-8 * np.linalg.norm(p.b)


def _true_relres_scipy(p, x):
    """||b - A x|| / ||b|| with scipy's BSR product (independent of the oracle's SpMV)."""
    import scipy.sparse as sp
    A = sp.bsr_matrix((p.vals, p.col_idx, p.row_ptr), shape=(p.n, p.n))
    return np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b)


def test_refinement_last_step_runs_only_to_what_the_target_needs():
    """The refinement's inner tolerance is inner_rtol relative to the current outer
    residual, except that a step whose residual is within 1/inner_rtol of the target
    runs only to max(inner_rtol, 0.5 tol / ||r||).  With an unrounded inner system
    (inner solves in exact FP64) that gives exactly two outer steps and a final
    residual between tol/100 and tol: a fixed 1e-5 would land near 1e-10."""
    p = synth.workload("tiny_20x20x10")
    outer = oracle.System.from_problem(p, pc="none")
    exact_inner = oracle.System.from_problem(p, pc="bilu0", float_round=False)
    st, x, info = oracle.refine(outer, exact_inner, p.b, solver="gmres", rtol=1e-8, inner_rtol=1e-5)
    rel = _true_relres_scipy(p, x)
    assert st == 0 and info["outer"] == 2
    assert 1e-10 < rel <= 1e-8, rel
    # the float-rounded inner system of the mixed-precision model reaches the target too
    inner = oracle.System.from_problem(p, pc="bilu0", float_round=True)
    for solver in ("gmres", "bicgstab"):
        st, x, info = oracle.refine(outer, inner, p.b, solver=solver, rtol=1e-8, inner_rtol=1e-5, maxit=6000)
        assert st == 0 and _true_relres_scipy(p, x) <= 1e-8


def test_recorded_refinement_solves_reach_the_target():
    """The stored refinement solves (written by tests/golden/make_golden.py from the
    oracle alone) end with status OK at a true residual at or below 1e-8."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "oracle_solves.json")))
    keys = [k for k in gold if "/refine-" in k]
    assert keys
    for k in keys:
        assert gold[k]["status"] == 0 and gold[k]["relres"] <= 1e-8, (k, gold[k])
