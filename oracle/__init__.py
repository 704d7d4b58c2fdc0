"""CPU FP64 oracle for the reservoir linear-solve path (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package.  The CUDA library never imports, links or falls back to it,
and the two share no code: the arithmetic lives in ``oracle.c`` (plain C,
sequential, FP64), built by :func:`build` with gcc.

Parity status of each routine (pins live in ``tests/test_oracle_pins.py``):
SpMV, 3x3 inverse, dense solve, block Jacobi, block ILU(0), quasi-IMPES,
Galerkin coarsening, red-black Gauss-Seidel, V-cycle, CPR, GMRES, FGMRES,
BiCGSTAB and iterative refinement are each pinned against dense linear
algebra, closed forms or invariants; so are the CPR stage orders (FP, FPF,
FFPF).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_variant = "serial"

OK, EINVAL, ENOMEM, ESINGULAR, EBREAKDOWN, ENOCONV, ENAN = 0, 1, 2, 5, 6, 7, 9
# "cpr" is CPR-PF (pressure stage, then full stage); the other orders follow the
# paper's CPR-FP, CPR-FPF and CPR-FFPF algorithms
PC = {"none": 0, "bjacobi": 1, "bilu0": 2, "cpr": 3, "cpr_fp": 5, "cpr_fpf": 6, "cpr_ffpf": 7}
DECOUPLING = {"qi": 0, "abf": 1, "timpes": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (sequential: the parity oracle) and
    liboracle_omp.so (the same source with OpenMP: the CPU timing baseline).

    -ffp-contract=off keeps every a*b+c as two rounded operations, so the oracle
    rounds identically on x86-64 and AArch64 hosts.
    """
    for path, extra in ((_LIB_PATH, []), (_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, path)
    return _LIB_PATH


def use_threads(threads: int) -> int:
    """Route every later oracle call through the OpenMP build with `threads`
    threads (threads <= 1: the sequential build).  Returns the thread count in
    use.  Parity tests keep the sequential build; the benchmark's CPU baseline
    uses this."""
    global _lib, _variant
    want = "omp" if threads > 1 else "serial"
    if want != _variant:
        _lib, _variant = None, want
    return lib().or_set_threads(max(1, threads))


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OMP_PATH if _variant == "omp" else _LIB_PATH)
        P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "or_dot": (D, [I64, P, P]), "or_norm2": (D, [I64, P]),
            "or_spmv": (I, [I, P, P, P, D, P, D, P]),
            "or_dense_solve": (I, [I, P, P, P]), "or_inv3": (I, [P, P]),
            "or_bj_setup": (I, [I, P, P, P, P]), "or_bj_apply": (None, [I, P, P, P]),
            "or_bilu0_setup": (I, [I, P, P, P, P, P, P]),
            "or_bilu0_apply": (None, [I, P, P, P, P, P, P]),
            "or_qi_setup": (I, [I, I, I, P, P, P, P, P]),
            "or_restrict_pressure": (None, [I, P, P, P]),
            "or_prolong_pressure": (None, [I, P, P]),
            "or_stencil_apply": (None, [I, I, I, P, P, P]),
            "or_gmg_coarsen": (None, [I, I, I, P, P]),
            "or_gs_colour": (None, [I, I, I, P, P, P, I]),
            "or_gmg_vcycle": (I, [I, I, I, P, I, I, I, P, P, P]),
            "or_create": (P, [I, I, I, P, P, P, I]), "or_destroy": (None, [P]),
            "or_setup": (I, [P, I, I, I, I, I, I]), "or_decouple_setup": (I, [I, I, I, P, P, P, I, P, P, P]), "or_set_accumulation": (None, [P, P]), "or_pc_apply": (I, [P, P, P]),
            "or_get_factors": (None, [P, P, P, P]), "or_gmg_levels": (I, [P]),
            "or_gmres": (I, [P, P, P, I, D, I, I, P]),
            "or_bicgstab": (I, [P, P, P, D, D, I, P]),
            "or_refine": (I, [P, P, P, P, I, I, D, D, I, I, P]),
            "or_set_threads": (I, [I]),
            "or_set_coarsening": (None, [P, I]),
            "or_amg_hierarchy": (I, [I, I, I, P, I, I, P]),
            "or_amg_vcycle": (I, [I, I, I, P, I, I, I, P, P, P]),
            "or_amg_level": (I, [I, I, I, P, I, I, I, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------- primitives

def spmv(row_ptr, col_idx, vals, x, alpha=1.0, beta=0.0, y=None):
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    nb = len(rp) - 1
    x = _f64(x)
    y = np.zeros(3 * nb) if y is None else _f64(y).copy()
    lib().or_spmv(nb, _p(rp), _p(ci), _p(v), alpha, _p(x), beta, _p(y))
    return y


def dot(x, y):
    x, y = _f64(x), _f64(y)
    return lib().or_dot(len(x), _p(x), _p(y))


def norm2(x):
    x = _f64(x)
    return lib().or_norm2(len(x), _p(x))


def dense_solve(A, b):
    A, b = _f64(A), _f64(b)
    x = np.zeros_like(b)
    st = lib().or_dense_solve(len(b), _p(A), _p(b), _p(x))
    return st, x


def inv3(a):
    a = _f64(a).reshape(3, 3)
    out = np.zeros((3, 3))
    st = lib().or_inv3(_p(a), _p(out))
    return st, out


def bj_setup(row_ptr, col_idx, vals):
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    nb = len(rp) - 1
    dinv = np.zeros((nb, 3, 3))
    st = lib().or_bj_setup(nb, _p(rp), _p(ci), _p(v), _p(dinv))
    return st, dinv


def bj_apply(dinv, r):
    dinv, r = _f64(dinv), _f64(r)
    z = np.zeros_like(r)
    lib().or_bj_apply(len(r) // 3, _p(dinv), _p(r), _p(z))
    return z


def bilu0_setup(row_ptr, col_idx, vals):
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    nb = len(rp) - 1
    lu = np.zeros_like(v)
    udinv = np.zeros((nb, 3, 3))
    off = ctypes.c_int64(0)
    st = lib().or_bilu0_setup(nb, _p(rp), _p(ci), _p(v), _p(lu), _p(udinv), ctypes.byref(off))
    return st, lu, udinv, off.value


def bilu0_apply(row_ptr, col_idx, lu, udinv, r):
    rp, ci, lu, udinv, r = _i32(row_ptr), _i32(col_idx), _f64(lu), _f64(udinv), _f64(r)
    z = np.zeros_like(r)
    lib().or_bilu0_apply(len(rp) - 1, _p(rp), _p(ci), _p(lu), _p(udinv), _p(r), _p(z))
    return z


def qi_setup(nx, ny, nz, row_ptr, col_idx, vals):
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    nb = nx * ny * nz
    w = np.zeros((nb, 3))
    a7 = np.zeros((nb, 7))
    st = lib().or_qi_setup(nx, ny, nz, _p(rp), _p(ci), _p(v), _p(w), _p(a7))
    return st, w, a7


def decouple_setup(nx, ny, nz, row_ptr, col_idx, vals, decoupling="qi", acc=None):
    """Weights w [nb,3] and pressure stencil [nb,7] for decoupling "qi" (quasi-IMPES), "abf" or
    "timpes" (true-IMPES: needs the accumulation blocks acc [nb,3,3])."""
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    nb = nx * ny * nz
    w = np.zeros((nb, 3))
    a7 = np.zeros((nb, 7))
    keep = _f64(acc) if acc is not None else None   # alive across the call
    accp = _p(keep) if keep is not None else None
    st = lib().or_decouple_setup(nx, ny, nz, _p(rp), _p(ci), _p(v), DECOUPLING[decoupling], accp, _p(w), _p(a7))
    return st, w, a7


def restrict_pressure(w, r):
    w, r = _f64(w), _f64(r)
    p = np.zeros(len(r) // 3)
    lib().or_restrict_pressure(len(p), _p(w), _p(r), _p(p))
    return p


def prolong_pressure(p):
    p = _f64(p)
    x = np.zeros(3 * len(p))
    lib().or_prolong_pressure(len(p), _p(p), _p(x))
    return x


def stencil_apply(nx, ny, nz, a7, x):
    a7, x = _f64(a7), _f64(x)
    y = np.zeros(nx * ny * nz)
    lib().or_stencil_apply(nx, ny, nz, _p(a7), _p(x), _p(y))
    return y


def gmg_coarsen(nx, ny, nz, a7):
    a7 = _f64(a7)
    cx, cy, cz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    ac = np.zeros((cx * cy * cz, 7))
    lib().or_gmg_coarsen(nx, ny, nz, _p(a7), _p(ac))
    return (cx, cy, cz), ac


def gs_colour(nx, ny, nz, a7, b, x, colour):
    a7, b = _f64(a7), _f64(b)
    x = _f64(x).copy()
    lib().or_gs_colour(nx, ny, nz, _p(a7), _p(b), _p(x), colour)
    return x


def gmg_vcycle(nx, ny, nz, a7, rhs, max_levels=6, max_coarse=512, sweeps=2):
    a7, rhs = _f64(a7), _f64(rhs)
    e = np.zeros_like(rhs)
    nl = ctypes.c_int(0)
    st = lib().or_gmg_vcycle(nx, ny, nz, _p(a7), max_levels, max_coarse, sweeps, _p(rhs), _p(e),
                             ctypes.byref(nl))
    return st, e, nl.value


COARSENING = {"gmg": 0, "amg": 1}


def amg_hierarchy(nx, ny, nz, a7, max_levels=8, max_coarse=512):
    """[(points, nonzeros)] per level of the algebraic (PMIS) hierarchy, finest first."""
    a7 = _f64(a7)
    sizes = np.zeros(32, dtype=np.int32)
    nl = lib().or_amg_hierarchy(nx, ny, nz, _p(a7), max_levels, max_coarse, _p(sizes))
    if nl < 0:
        raise ValueError(f"AMG setup failed: status {-nl}")
    return [(int(sizes[2 * l]), int(sizes[2 * l + 1])) for l in range(nl)]


def amg_vcycle(nx, ny, nz, a7, rhs, max_levels=8, max_coarse=512, sweeps=2):
    a7, rhs = _f64(a7), _f64(rhs)
    e = np.zeros_like(rhs)
    nl = ctypes.c_int(0)
    st = lib().or_amg_vcycle(nx, ny, nz, _p(a7), max_levels, max_coarse, sweeps, _p(rhs), _p(e), ctypes.byref(nl))
    return st, e, nl.value


def amg_level(nx, ny, nz, a7, level, max_levels=8, max_coarse=512):
    """Level `level` of the AMG hierarchy: (cf [n], P as dense-free CSR (rp, ci, v), A_coarse CSR (rp, ci, v))."""
    levels = amg_hierarchy(nx, ny, nz, a7, max_levels, max_coarse)
    n, _ = levels[level]
    nc, nnzc = levels[level + 1]
    a7 = _f64(a7)
    cf = np.zeros(n, dtype=np.int32)
    prp = np.zeros(n + 1, dtype=np.int32)
    cap = 8 * n + 1
    pci = np.zeros(cap, dtype=np.int32)
    pv = np.zeros(cap)
    arp = np.zeros(nc + 1, dtype=np.int32)
    aci = np.zeros(nnzc, dtype=np.int32)
    av = np.zeros(nnzc)
    nnzp = lib().or_amg_level(nx, ny, nz, _p(a7), max_levels, max_coarse, level, _p(cf), _p(prp), _p(pci), _p(pv),
                              _p(arp), _p(aci), _p(av))
    assert 0 <= nnzp <= cap
    return cf, (prp, pci[:nnzp].copy(), pv[:nnzp].copy()), (arp, aci, av)


# ------------------------------------------------------------------ system

class System:
    """A BSR system plus one preconditioner, driven through the C oracle."""

    def __init__(self, nx, ny, nz, row_ptr, col_idx, vals, pc="none", float_round=False,
                 gmg_levels=6, gmg_coarse=512, gmg_sweeps=2, decoupling="qi", acc=None, coarsening="gmg"):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nb = nx * ny * nz
        self._rp, self._ci = _i32(row_ptr), _i32(col_idx)
        self._v = _f64(vals)
        self._h = lib().or_create(nx, ny, nz, _p(self._rp), _p(self._ci), _p(self._v), int(float_round))
        if not self._h:
            raise MemoryError("oracle system allocation failed")
        if acc is not None:
            lib().or_set_accumulation(self._h, _p(_f64(acc)))
        lib().or_set_coarsening(self._h, COARSENING[coarsening])
        self.setup_status = lib().or_setup(self._h, PC[pc], gmg_levels, gmg_coarse, gmg_sweeps,
                                           int(float_round), DECOUPLING[decoupling])
        self.pc = pc

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    @classmethod
    def from_problem(cls, p, pc="none", **kw):
        return cls(p.nx, p.ny, p.nz, p.row_ptr, p.col_idx, p.vals, pc=pc, **kw)

    def pc_apply(self, r):
        r = _f64(r)
        z = np.zeros_like(r)
        st = lib().or_pc_apply(self._h, _p(r), _p(z))
        return st, z

    def factors(self):
        """(dinv or U_ii^{-1} [nb,3,3], quasi-IMPES w [nb,3], pressure stencil [nb,7])."""
        d = np.zeros((self.nb, 3, 3))
        w = np.zeros((self.nb, 3))
        a7 = np.zeros((self.nb, 7))
        lib().or_get_factors(self._h, _p(d), _p(w), _p(a7))
        return d, w, a7

    def gmg_levels(self):
        return lib().or_gmg_levels(self._h)

    def gmres(self, b, x0=None, m=30, rtol=1e-8, maxit=2000, flexible=False):
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        stats = np.zeros(4)
        st = lib().or_gmres(self._h, _p(b), _p(x), m, rtol, maxit, int(flexible), _p(stats))
        return st, x, dict(iters=int(stats[0]), restarts=int(stats[1]), relres=stats[2],
                           pc_applies=int(stats[3]))

    def bicgstab(self, b, x0=None, rtol=1e-8, btol=1e-30, maxit=2000):
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        stats = np.zeros(4)
        st = lib().or_bicgstab(self._h, _p(b), _p(x), rtol, btol, maxit, _p(stats))
        return st, x, dict(iters=int(stats[0]), relres=stats[2], pc_applies=int(stats[3]))


def refine(outer: System, inner: System, b, solver="gmres", m=30, rtol=1e-8, inner_rtol=1e-5,
           max_outer=10, maxit=2000):
    b = _f64(b)
    x = np.zeros_like(b)
    stats = np.zeros(4)
    st = lib().or_refine(outer._h, inner._h, _p(b), _p(x), 0 if solver == "gmres" else 1, m, rtol,
                         inner_rtol, max_outer, maxit, _p(stats))
    return st, x, dict(iters=int(stats[0]), outer=int(stats[1]), relres=stats[2])
