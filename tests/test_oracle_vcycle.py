"""Pin of the oracle's multi-level V-cycle against its dense error operator.

Section "Algebraic Multigrid Methods" (V-cycle algorithm; R = P^T and the
Galerkin product A_{l+1} = R A_l P; one cycle, 2 relaxation sweeps by
default) defines one V-cycle from a zero guess as a linear map b -> e = B b.
Here B is built densely for every level from parts that do not touch the
oracle's code:

* A_0 is the dense seven-point operator; A_{l+1} = P_l^T A_l P_l with the
  piecewise-constant P_l of the 2x2x2 boxes (dims ceil(d/2)), built densely;
* one red-black Gauss-Seidel half-sweep on colour c ((i+j+k) mod 2) is
  x <- x + S_c (b - A x) with S_c = diag(1/a_ii) on colour c and 0
  elsewhere (same-colour cells do not couple in a seven-point stencil);
* pre-smoothing red then black, `sweeps` times; restrict the residual with
  P^T; recurse; add P e_c; post-smoothing black then red, `sweeps` times;
  the coarsest level is solved exactly.

The oracle's cycle, applied to every unit vector, must reproduce B.  The
mutation tests then compile copies of the oracle with one plausible mistake
each (post-smoothing red-then-black, one sweep instead of `sweeps`, no
prolongation on the coarser levels) and check that this pin rejects them.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import stencil_to_dense

ORACLE_SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")


def _dims_of_levels(nx, ny, nz, max_levels, max_coarse):
    dims = [(nx, ny, nz)]
    while len(dims) < max_levels and np.prod(dims[-1]) > max_coarse:
        dims.append(tuple((d + 1) // 2 for d in dims[-1]))
    return dims


def _prolongation(fine, coarse):
    nx, ny, nz = fine
    cx, cy, _ = coarse
    P = np.zeros((nx * ny * nz, int(np.prod(coarse))))
    for c in range(nx * ny * nz):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        P[c, cx * cy * (k // 2) + cx * (j // 2) + i // 2] = 1.0
    return P


def _colour_masks(dims):
    nx, ny, nz = dims
    c = np.arange(nx * ny * nz)
    parity = (c % nx + (c // nx) % ny + c // (nx * ny)) % 2
    return parity == 0, parity == 1


def dense_vcycle_operator(nx, ny, nz, a7, max_levels, max_coarse, sweeps):
    """B with e = B b for one V-cycle from a zero guess, from dense parts only."""
    dims = _dims_of_levels(nx, ny, nz, max_levels, max_coarse)
    A = [stencil_to_dense(nx, ny, nz, a7)]
    Ps = []
    for l in range(len(dims) - 1):
        P = _prolongation(dims[l], dims[l + 1])
        Ps.append(P)
        A.append(P.T @ A[l] @ P)

    def cycle(l):
        Al = A[l]
        n = Al.shape[0]
        if l == len(dims) - 1:
            return np.linalg.inv(Al)
        red, black = _colour_masks(dims[l])
        d = np.diag(Al)
        S = {0: np.diag(np.where(red, 1.0 / d, 0.0)), 1: np.diag(np.where(black, 1.0 / d, 0.0))}
        eye = np.eye(n)
        X = np.zeros((n, n))          # column q: the iterate for right-hand side e_q
        for _ in range(sweeps):
            for c in (0, 1):
                X = X + S[c] @ (eye - Al @ X)
        Bc = cycle(l + 1)
        X = X + Ps[l] @ (Bc @ (Ps[l].T @ (eye - Al @ X)))
        for _ in range(sweeps):
            for c in (1, 0):
                X = X + S[c] @ (eye - Al @ X)
        return X

    return cycle(0), len(dims)


def _pressure_stencil(dims, seed):
    p = synth.make_problem(*dims, seed=seed)
    st, _, a7 = oracle.qi_setup(*dims, p.row_ptr, p.col_idx, p.vals)
    assert st == 0
    return a7


def _oracle_operator(vcycle, nx, ny, nz, a7, max_levels, max_coarse, sweeps):
    n = nx * ny * nz
    cols, nlev = [], None
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        st, x, nlev = vcycle(nx, ny, nz, a7, e, max_levels, max_coarse, sweeps)
        assert st == 0
        cols.append(x)
    return np.column_stack(cols), nlev


def _matches(B_or, B_ref):
    return np.max(np.abs(B_or - B_ref)) <= 1e-11 * np.max(np.abs(B_ref))


CASES = [
    # (dims, max_levels, max_coarse, sweeps): two- and three-level cycles
    ((6, 4, 4), 2, 1, 2),
    ((6, 4, 4), 6, 8, 2),
    ((8, 6, 4), 6, 8, 2),
    ((8, 6, 4), 6, 8, 1),
    ((8, 6, 4), 6, 8, 3),
    ((5, 3, 3), 6, 4, 2),   # odd dims: boxes of width one on the far faces
]


@pytest.mark.parametrize("dims,max_levels,max_coarse,sweeps", CASES)
def test_vcycle_equals_dense_error_operator(dims, max_levels, max_coarse, sweeps):
    a7 = _pressure_stencil(dims, seed=31)
    B_ref, nlev_ref = dense_vcycle_operator(*dims, a7, max_levels, max_coarse, sweeps)
    B_or, nlev = _oracle_operator(oracle.gmg_vcycle, *dims, a7, max_levels, max_coarse, sweeps)
    assert nlev == nlev_ref >= 2
    assert _matches(B_or, B_ref), np.max(np.abs(B_or - B_ref))


def test_vcycle_three_levels_on_laplacian_is_a_contraction():
    """On the Dirichlet Laplacian the cycle's iteration matrix I - B A contracts."""
    from tests.test_oracle_pins import _laplacian_a7
    dims = (8, 6, 4)
    a7 = _laplacian_a7(*dims, dirichlet=True)
    B, nlev = dense_vcycle_operator(*dims, a7, 6, 8, 2)
    B_or, _ = _oracle_operator(oracle.gmg_vcycle, *dims, a7, 6, 8, 2)
    assert nlev == 3 and _matches(B_or, B)
    A = stencil_to_dense(*dims, a7)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(A.shape[0]) - B @ A)))
    assert rho < 0.5


# ----------------------------------------------------------- mutation checks

_PRE = ("        or_gs_colour(nx, ny, nz, g->a7[l], g->b[l], g->x[l], 1);\n"
        "        or_gs_colour(nx, ny, nz, g->a7[l], g->b[l], g->x[l], 0);\n")
MUTATIONS = {
    # post-smoothing in the pre-smoothing order (red then black)
    "post_red_then_black": (_PRE, _PRE.replace(", 1);\n", ", @);\n").replace(", 0);\n", ", 1);\n")
                            .replace(", @);\n", ", 0);\n")),
    # one smoothing sweep whatever `sweeps` says
    "single_sweep": ("for (int s = 0; s < g->sweeps; ++s)", "for (int s = 0; s < 1; ++s)"),
    # the coarse correction dropped on every level below the finest
    "no_prolongation_below_finest": ("g->x[l][(int64_t)nx * ny * k + (int64_t)nx * j + i] +=",
                                     "g->x[l][(int64_t)nx * ny * k + (int64_t)nx * j + i] += (l >= 1) ? 0.0 :"),
}


def _mutant_vcycle(tmp_path, name):
    src = open(ORACLE_SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation {name}: pattern not found in oracle.c"
    mutated = src.replace(old, new)
    c_path = tmp_path / f"oracle_{name}.c"
    so_path = tmp_path / f"liboracle_{name}.so"
    c_path.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                           str(so_path), str(c_path), "-lm"])
    L = ctypes.CDLL(str(so_path))
    P, I = ctypes.c_void_p, ctypes.c_int
    L.or_gmg_vcycle.restype = I
    L.or_gmg_vcycle.argtypes = [I, I, I, P, I, I, I, P, P, P]

    def vcycle(nx, ny, nz, a7, rhs, max_levels, max_coarse, sweeps):
        a7 = np.ascontiguousarray(a7, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        e = np.zeros_like(rhs)
        nl = ctypes.c_int(0)
        st = L.or_gmg_vcycle(nx, ny, nz, a7.ctypes.data, max_levels, max_coarse, sweeps, rhs.ctypes.data,
                             e.ctypes.data, ctypes.byref(nl))
        return st, e, nl.value
    return vcycle


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_dense_pin_rejects_mutated_vcycle(tmp_path, name):
    dims, max_levels, max_coarse, sweeps = (8, 6, 4), 6, 8, 2
    a7 = _pressure_stencil(dims, seed=31)
    B_ref, _ = dense_vcycle_operator(*dims, a7, max_levels, max_coarse, sweeps)
    vcycle = _mutant_vcycle(tmp_path, name)
    B_mut, nlev = _oracle_operator(vcycle, *dims, a7, max_levels, max_coarse, sweeps)
    assert nlev == 3
    assert not _matches(B_mut, B_ref), f"the dense pin accepts the '{name}' mutation"
