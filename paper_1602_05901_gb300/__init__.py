"""Python binding of librsv, the GB300 reservoir linear-solver library.

Argument marshalling only: every step of the solve runs in the CUDA kernels
of ``librsv.so`` behind the C ABI declared in ``include/rsv.h``.  PyTorch
supplies device memory (tensor ``data_ptr()``) and streams.  Importing this
package loads the library and raises if it is missing; there is no CPU
fallback.  Build it with ``paper_1602_05901_gb300._build.build()``.

The module-level functions carry the C names (``rsv_grid_create`` ...) and
return ``(status, outputs...)``; :class:`Matrix` and :class:`Solver` wrap
the handles and raise :class:`RsvError` on a non-zero status.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsv.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"librsv.so not built at {LIB_PATH}: run paper_1602_05901_gb300._build.build() "
                      "(requires nvcc); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

RSV_OK, RSV_EINVAL, RSV_ENOMEM, RSV_ECUDA, RSV_ENOTSUP, RSV_ESINGULAR = 0, 1, 2, 3, 4, 5
RSV_EBREAKDOWN, RSV_ENOCONV, RSV_ETIMEOUT, RSV_ENAN = 6, 7, 8, 9
RSV_PC_NONE, RSV_PC_BJACOBI, RSV_PC_BILU0, RSV_PC_CPR, RSV_PC_CPR_LEARNED = 0, 1, 2, 3, 4
RSV_PC_CPR_FP, RSV_PC_CPR_FPF, RSV_PC_CPR_FFPF = 5, 6, 7
RSV_GMRES, RSV_BICGSTAB, RSV_FGMRES = 0, 1, 2
RSV_PREC_FP64, RSV_PREC_MIXED = 0, 1
PC_TYPES = {"none": RSV_PC_NONE, "bjacobi": RSV_PC_BJACOBI, "bilu0": RSV_PC_BILU0, "cpr": RSV_PC_CPR,
            "cpr_learned": RSV_PC_CPR_LEARNED, "cpr_fp": RSV_PC_CPR_FP, "cpr_fpf": RSV_PC_CPR_FPF,
            "cpr_ffpf": RSV_PC_CPR_FFPF}
SOLVERS = {"gmres": RSV_GMRES, "bicgstab": RSV_BICGSTAB, "fgmres": RSV_FGMRES}


class rsv_solver_params(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("restart", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("btol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("watchdog", ctypes.c_longlong)]


class rsv_pc_params(ctypes.Structure):
    _fields_ = [("gmg_max_levels", ctypes.c_int), ("gmg_max_coarse", ctypes.c_int), ("gmg_sweeps", ctypes.c_int),
                ("decoupling", ctypes.c_int), ("coarsening", ctypes.c_int)]


class rsv_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("status", ctypes.c_int), ("true_relres", ctypes.c_double), ("ms_setup", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("fallback_iter", ctypes.c_int), ("pad_", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


_P, _I, _D, _F, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_int64
_PP = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "rsv_solver_params_default": (None, [ctypes.POINTER(rsv_solver_params)]),
    "rsv_pc_params_default": (None, [ctypes.POINTER(rsv_pc_params)]),
    "rsv_status_string": (ctypes.c_char_p, [_I]),
    "rsv_last_cuda_error": (ctypes.c_char_p, []),
    "rsv_kernel_launches": (ctypes.c_uint64, []),
    "rsv_grid_create": (_I, [_I, _I, _I, _PP]),
    "rsv_grid_destroy": (None, [_P]),
    "rsv_mat_create": (_I, [_P, _P, _PP]),
    "rsv_mat_create_bsr": (_I, [_P, _I, _I, _P, _PP]),
    "rsv_vec_create": (_I, [_P, _I, _P, _PP]),
    "rsv_vec_wrap": (_I, [_P, _I64, _I, _PP]),
    "rsv_vec_set": (_I, [_P, _P, _I, _P]),
    "rsv_vec_get": (_I, [_P, _P, _I, _P]),
    "rsv_vec_info": (_I, [_P, _PP, ctypes.POINTER(_I64), ctypes.POINTER(_I)]),
    "rsv_vec_destroy": (None, [_P]),
    "rsv_mat_destroy": (None, [_P]),
    "rsv_mat_create_batch": (_I, [_I, _P, _P, _PP]),
    "rsv_mat_get_batch": (_I, [_P, ctypes.POINTER(_I), _P]),
    "rsv_mat_get_pattern": (_I, [_P, _PP, _PP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "rsv_mat_set_values": (_I, [_P, _P, _I]),
    "rsv_spmv": (_I, [_P, _D, _P, _D, _P]),
    "rsv_spmv_f32": (_I, [_P, _F, _P, _F, _P]),
    "rsv_dot": (_I, [_P, _I64, _P, _P, ctypes.POINTER(_D)]),
    "rsv_norm2": (_I, [_P, _I64, _P, ctypes.POINTER(_D)]),
    "rsv_axpby": (_I, [_P, _I64, _D, _P, _D, _P, _P]),
    "rsv_mdot_noalloc": (_I, [_P, _I64, _P, _P, _I64, _I, _P]),
    "rsv_solver_create": (_I, [_P, ctypes.POINTER(rsv_solver_params), _PP]),
    "rsv_solver_destroy": (None, [_P]),
    "rsv_precond_setup": (_I, [_P, _I, ctypes.POINTER(rsv_pc_params)]),
    "rsv_precond_set_accumulation": (_I, [_P, _P, _I]),
    "rsv_precond_apply": (_I, [_P, _P, _P]),
    "rsv_precond_apply_f32": (_I, [_P, _P, _P]),
    "rsv_precond_get_dinv": (_I, [_P, _P]),
    "rsv_cpr_info": (_I, [_P, ctypes.POINTER(_I), _P, _P, _P]),
    "rsv_cpr_vcycle": (_I, [_P, _P, _P]),
    "rsv_amg_info": (_I, [_P, ctypes.POINTER(_I), _P]),
    "rsv_solve": (_I, [_P, _P, _P, ctypes.POINTER(rsv_solve_info)]),
    "rsv_solve_ptr": (_I, [_P, _P, _P, _I, ctypes.POINTER(rsv_solve_info)]),
    "rsv_solve_batched": (_I, [_P, _P, _P, _P]),
    "rsv_solve_batched_ptr": (_I, [_P, _P, _P, _I, _P]),
    "rsv_conv3d_fwd": (_I, [_P, _I, _I, _I, _I, _I, _I, _P, _I, _P, _P, _I, _P, _I, _P, _I, _P]),
    "rsv_conv3d_dgrad": (_I, [_P, _I, _I, _I, _I, _I, _P, _I, _P, _P, _I, _P, _I, _P]),
    "rsv_conv3d_wgrad": (_I, [_P, _I, _I, _I, _I, _I, _I, _P, _I, _P, _I, _P, _P]),
    "rsv_unet_create": (_I, [_P, _I, _I, _I, _I, _I, _PP]),
    "rsv_unet_destroy": (None, [_P]),
    "rsv_unet_num_params": (_I, [_P, ctypes.POINTER(_I64)]),
    "rsv_unet_set_params": (_I, [_P, _P, _I]),
    "rsv_unet_get_params": (_I, [_P, _P, _I]),
    "rsv_unet_get_grads": (_I, [_P, _P, _I]),
    "rsv_unet_save": (_I, [_P, ctypes.c_char_p]),
    "rsv_unet_load": (_I, [_P, ctypes.c_char_p]),
    "rsv_unet_apply": (_I, [_P, _P, _P, _P]),
    "rsv_unet_train_step": (_I, [_P, _P, _P, _P, _F, ctypes.POINTER(_D)]),
    "rsv_unet_train_batch": (_I, [_P, _I, _P, _P, _P, _F, _P]),
    "rsv_solver_set_learned": (_I, [_P, _P, _P, _I, _I, _D]),
    "rsv_solver_record_pressure": (_I, [_P, _P, _I]),
    "rsv_solver_recorded": (_I, [_P, ctypes.POINTER(_I)]),
}
EXPORTS = tuple(_SIGS)

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class RsvError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.rsv_status_string(status).decode()
        if status in (RSV_ECUDA, RSV_ENOMEM):
            msg += f" ({_lib.rsv_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg} [{status}]")


def check(status, where="rsv"):
    if status != RSV_OK:
        raise RsvError(status, where)
    return status


def status_string(status: int) -> str:
    return _lib.rsv_status_string(status).decode()


def _ptr(t):
    """Raw address of a torch tensor or numpy array (contiguous)."""
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous()
        return ctypes.c_void_p(t.data_ptr())
    assert t.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(t.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def solver_params(solver="gmres", restart=30, rtol=1e-8, atol=0.0, btol=1e-30, maxit=2000, precision="fp64",
                  inner_rtol=1e-5, max_outer=10, watchdog=None):
    p = rsv_solver_params()
    _lib.rsv_solver_params_default(ctypes.byref(p))
    p.solver = SOLVERS[solver] if isinstance(solver, str) else solver
    p.restart, p.rtol, p.atol, p.btol, p.maxit = restart, rtol, atol, btol, maxit
    p.precision = {"fp64": RSV_PREC_FP64, "mixed": RSV_PREC_MIXED}[precision] if isinstance(precision, str) else precision
    p.inner_rtol, p.max_outer = inner_rtol, max_outer
    if watchdog is not None:
        p.watchdog = watchdog
    return p


DECOUPLING = {"qi": 0, "abf": 1, "timpes": 2}


COARSENING = {"gmg": 0, "amg": 1}


def pc_params(gmg_max_levels=6, gmg_max_coarse=512, gmg_sweeps=2, decoupling="qi", coarsening="gmg"):
    p = rsv_pc_params()
    _lib.rsv_pc_params_default(ctypes.byref(p))
    p.gmg_max_levels, p.gmg_max_coarse, p.gmg_sweeps = gmg_max_levels, gmg_max_coarse, gmg_sweeps
    p.decoupling = DECOUPLING[decoupling] if isinstance(decoupling, str) else decoupling
    p.coarsening = COARSENING[coarsening] if isinstance(coarsening, str) else coarsening
    return p


class Matrix:
    """Seven-point 3x3-block BSR matrix of an nx*ny*nz grid, resident on the GPU.

    ``Matrix.batch([(nx, ny, nz), ...])`` builds the block-diagonal matrix of a
    batch of independent grids (solve it with ``Solver.solve_batched``)."""

    def __init__(self, nx, ny, nz, stream=None, _batch_dims=None, precision="mixed"):
        """precision "fp64": FP64 values only (FP64 solvers); "mixed": also the FP32 copy."""
        self.nx, self.ny, self.nz = nx, ny, nz
        self.stream = _stream_ptr(stream)
        h = ctypes.c_void_p()
        if _batch_dims is None:
            g = ctypes.c_void_p()
            check(_lib.rsv_grid_create(nx, ny, nz, ctypes.byref(g)), "rsv_grid_create")
            try:
                prec = {"fp64": RSV_PREC_FP64, "mixed": RSV_PREC_MIXED}[precision]
                check(_lib.rsv_mat_create_bsr(g, 3, prec, self.stream, ctypes.byref(h)), "rsv_mat_create_bsr")
            finally:
                _lib.rsv_grid_destroy(g)
        else:
            dims = np.ascontiguousarray(np.asarray(_batch_dims, dtype=np.int32).reshape(-1, 3))
            check(_lib.rsv_mat_create_batch(len(dims), _ptr(dims), self.stream, ctypes.byref(h)),
                  "rsv_mat_create_batch")
        self.handle = h
        nsys = ctypes.c_int()
        check(_lib.rsv_mat_get_batch(h, ctypes.byref(nsys), None))
        self.nsys = nsys.value
        self.cell_offsets = np.zeros(self.nsys + 1, dtype=np.int64)
        check(_lib.rsv_mat_get_batch(h, None, _ptr(self.cell_offsets)))
        rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
        nb, nnzb = _I64(), _I64()
        check(_lib.rsv_mat_get_pattern(h, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nb), ctypes.byref(nnzb)))
        self.nb, self.nnzb = nb.value, nnzb.value
        self.row_ptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(ctypes.c_int32)), (self.nb + 1,)).copy()
        self.col_idx = np.ctypeslib.as_array(ctypes.cast(ci, ctypes.POINTER(ctypes.c_int32)), (self.nnzb,)).copy()

    @property
    def n(self):
        return 3 * self.nb

    @classmethod
    def batch(cls, dims, stream=None):
        d0 = dims[0]
        return cls(d0[0], d0[1], d0[2], stream=stream, _batch_dims=dims)

    def set_values(self, vals):
        """vals: float64 [nnzb,3,3] as a numpy array (host) or CUDA torch tensor."""
        on_dev = int(hasattr(vals, "is_cuda") and vals.is_cuda)
        if not on_dev:
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        assert vals.size == 9 * self.nnzb if not on_dev else vals.numel() == 9 * self.nnzb
        check(_lib.rsv_mat_set_values(self.handle, _ptr(vals), on_dev), "rsv_mat_set_values")

    def spmv(self, x, y, alpha=1.0, beta=0.0):
        if x.dtype.itemsize == 4:
            check(_lib.rsv_spmv_f32(self.handle, alpha, _ptr(x), beta, _ptr(y)), "rsv_spmv_f32")
        else:
            check(_lib.rsv_spmv(self.handle, alpha, _ptr(x), beta, _ptr(y)), "rsv_spmv")
        return y

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.rsv_mat_destroy(h)
            self.handle = None


class Vector:
    """An rsv_vec handle: owned device memory (``Vector.create``) or a borrowed
    CUDA tensor (``Vector.wrap``; the tensor must outlive the handle)."""

    def __init__(self, handle, keep=None):
        self.handle = handle
        self._keep = keep
        ptr, n, prec = ctypes.c_void_p(), _I64(), ctypes.c_int()
        check(_lib.rsv_vec_info(handle, ctypes.byref(ptr), ctypes.byref(n), ctypes.byref(prec)), "rsv_vec_info")
        self.data_ptr, self.n, self.precision = ptr.value, n.value, prec.value

    @classmethod
    def create(cls, nx, ny, nz, precision="fp64", stream=None):
        g, h = ctypes.c_void_p(), ctypes.c_void_p()
        check(_lib.rsv_grid_create(nx, ny, nz, ctypes.byref(g)), "rsv_grid_create")
        try:
            prec = {"fp64": RSV_PREC_FP64, "mixed": RSV_PREC_MIXED}[precision]
            check(_lib.rsv_vec_create(g, prec, _stream_ptr(stream), ctypes.byref(h)), "rsv_vec_create")
        finally:
            _lib.rsv_grid_destroy(g)
        return cls(h)

    @classmethod
    def wrap(cls, t):
        """Borrow a contiguous CUDA float64 (FP64) or float32 (FP32) tensor."""
        assert t.is_cuda and t.is_contiguous()
        prec = RSV_PREC_FP64 if t.element_size() == 8 else RSV_PREC_MIXED
        h = ctypes.c_void_p()
        check(_lib.rsv_vec_wrap(ctypes.c_void_p(t.data_ptr()), t.numel(), prec, ctypes.byref(h)), "rsv_vec_wrap")
        return cls(h, keep=t)

    @classmethod
    def of(cls, v):
        return v if isinstance(v, Vector) else cls.wrap(v)

    def set(self, src, stream=None):
        on_dev = int(hasattr(src, "is_cuda") and src.is_cuda)
        if not on_dev:
            src = np.ascontiguousarray(src, dtype=np.float64)
        check(_lib.rsv_vec_set(self.handle, _ptr(src), on_dev, _stream_ptr(stream)), "rsv_vec_set")

    def get(self, dst=None, stream=None):
        if dst is None:
            dst = np.zeros(self.n)
        on_dev = int(hasattr(dst, "is_cuda") and dst.is_cuda)
        check(_lib.rsv_vec_get(self.handle, _ptr(dst), on_dev, _stream_ptr(stream)), "rsv_vec_get")
        return dst

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.rsv_vec_destroy(h)
            self.handle = None


class Solver:
    """Krylov solver + preconditioner bound to a Matrix (which must outlive it)."""

    def __init__(self, A: Matrix, **params):
        self.A = A
        self.params = solver_params(**params)
        h = ctypes.c_void_p()
        check(_lib.rsv_solver_create(A.handle, ctypes.byref(self.params), ctypes.byref(h)), "rsv_solver_create")
        self.handle = h

    def setup(self, pc="bilu0", **pcp):
        st = _lib.rsv_precond_setup(self.handle, PC_TYPES[pc] if isinstance(pc, str) else pc,
                                    ctypes.byref(pc_params(**pcp)))
        check(st, "rsv_precond_setup")

    def set_accumulation(self, acc):
        """Accumulation blocks [nb,3,3] (host numpy or CUDA tensor) for decoupling="timpes"; None drops them."""
        if acc is None:
            check(_lib.rsv_precond_set_accumulation(self.handle, None, 0), "rsv_precond_set_accumulation")
            return
        on_dev = int(hasattr(acc, "is_cuda") and acc.is_cuda)
        if not on_dev:
            acc = np.ascontiguousarray(acc, dtype=np.float64)
        check(_lib.rsv_precond_set_accumulation(self.handle, _ptr(acc), on_dev), "rsv_precond_set_accumulation")

    def apply(self, r, z):
        if r.dtype.itemsize == 4:
            check(_lib.rsv_precond_apply_f32(self.handle, _ptr(r), _ptr(z)), "rsv_precond_apply_f32")
        else:
            check(_lib.rsv_precond_apply(self.handle, _ptr(r), _ptr(z)), "rsv_precond_apply")
        return z

    def dinv(self):
        out = np.zeros((self.A.nb, 3, 3))
        check(_lib.rsv_precond_get_dinv(self.handle, _ptr(out)), "rsv_precond_get_dinv")
        return out

    def cpr_info(self, with_arrays=True):
        """(levels [(nx, ny, nz)...], QI weights [nb,3], [per-level stencil [n_l,7]])."""
        nl = ctypes.c_int()
        dims = (ctypes.c_int * 24)()
        check(_lib.rsv_cpr_info(self.handle, ctypes.byref(nl), dims, None, None), "rsv_cpr_info")
        levels = [(dims[3 * l], dims[3 * l + 1], dims[3 * l + 2]) for l in range(nl.value)]
        if not with_arrays:
            return levels, None, None
        total = sum(a * b_ * c for a, b_, c in levels)
        w = np.zeros((self.A.nb, 3))
        a7 = np.zeros((total, 7))
        check(_lib.rsv_cpr_info(self.handle, None, None, _ptr(w), _ptr(a7)), "rsv_cpr_info")
        out, off = [], 0
        for a, b_, c in levels:
            out.append(a7[off:off + a * b_ * c])
            off += a * b_ * c
        return levels, w, out

    def amg_info(self):
        """[(points, nonzeros)] per level of the algebraic pressure hierarchy, finest first."""
        nl = ctypes.c_int()
        sizes = np.zeros(32, dtype=np.int64)
        check(_lib.rsv_amg_info(self.handle, ctypes.byref(nl), _ptr(sizes)), "rsv_amg_info")
        return [(int(sizes[2 * l]), int(sizes[2 * l + 1])) for l in range(nl.value)]

    def vcycle(self, b, x):
        check(_lib.rsv_cpr_vcycle(self.handle, _ptr(b), _ptr(x)), "rsv_cpr_vcycle")
        return x

    def solve(self, b, x, raise_on_error=False):
        """b, x: float64 [3*nb], both host numpy, both CUDA tensors, or both :class:`Vector`.
        Device data goes through rsv_solve on vector handles (tensors are wrapped, not
        copied); host arrays through rsv_solve_ptr, which copies them in and out.
        Returns (status, info dict)."""
        info = rsv_solve_info()
        if isinstance(b, Vector) or (hasattr(b, "is_cuda") and b.is_cuda):
            bv, xv = Vector.of(b), Vector.of(x)
            st = _lib.rsv_solve(self.handle, bv.handle, xv.handle, ctypes.byref(info))
        else:
            st = _lib.rsv_solve_ptr(self.handle, _ptr(b), _ptr(x), 0, ctypes.byref(info))
        if raise_on_error:
            check(st, "rsv_solve")
        return st, info.as_dict()

    def set_learned(self, unet, lnk, stall_window=0, stall_drop=0.10):
        """Make ``unet`` (a Unet on this matrix's grid) the pressure stage of "cpr_learned"; lnk: ln k per cell.

        Fall back to the V-cycle when the residual falls by less than stall_drop over stall_window
        iterations (stall_window <= 0: 10% over 5)."""
        on_dev = int(hasattr(lnk, "is_cuda") and lnk.is_cuda)
        if not on_dev:
            lnk = np.ascontiguousarray(lnk, dtype=np.float64)
        self._unet = unet   # the solver does not own the network: keep it alive
        check(_lib.rsv_solver_set_learned(self.handle, unet.handle, _ptr(lnk), on_dev, int(stall_window),
                                          float(stall_drop)), "rsv_solver_set_learned")

    def record_pressure(self, buf, max_samples):
        """Record the restricted right-hand sides of FP64 CPR applications into buf (device [max][nb]); None stops."""
        check(_lib.rsv_solver_record_pressure(self.handle, _ptr(buf) if buf is not None else None,
                                              int(max_samples)), "rsv_solver_record_pressure")

    def recorded(self):
        c = ctypes.c_int()
        check(_lib.rsv_solver_recorded(self.handle, ctypes.byref(c)), "rsv_solver_recorded")
        return c.value

    def solve_batched(self, b, x):
        """Independent per-grid solves of a batch matrix. Returns (status, [info dict per grid])."""
        infos = (rsv_solve_info * self.A.nsys)()
        if isinstance(b, Vector) or (hasattr(b, "is_cuda") and b.is_cuda):
            bv, xv = Vector.of(b), Vector.of(x)  # keep the handles alive across the call
            st = _lib.rsv_solve_batched(self.handle, bv.handle, xv.handle, infos)
        else:
            st = _lib.rsv_solve_batched_ptr(self.handle, _ptr(b), _ptr(x), 0, infos)
        return st, [i.as_dict() for i in infos]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.rsv_solver_destroy(h)
            self.handle = None


class Unet:
    """The learned pressure stage's network (rsv_unet.h) on an nx*ny*nz grid."""

    def __init__(self, nx, ny, nz, base=32, levels=4, stream=None):
        self.dims = (nx, ny, nz)
        self.base, self.levels = base, levels
        h = ctypes.c_void_p()
        check(_lib.rsv_unet_create(_stream_ptr(stream), nx, ny, nz, base, levels, ctypes.byref(h)), "rsv_unet_create")
        self.handle = h
        n = ctypes.c_int64()
        check(_lib.rsv_unet_num_params(h, ctypes.byref(n)))
        self.nparam = n.value

    def set_params(self, p):
        on_dev = int(hasattr(p, "is_cuda") and p.is_cuda)
        if not on_dev:
            p = np.ascontiguousarray(p, dtype=np.float32)
        assert (p.numel() if on_dev else p.size) == self.nparam
        check(_lib.rsv_unet_set_params(self.handle, _ptr(p), on_dev), "rsv_unet_set_params")

    def params(self):
        out = np.zeros(self.nparam, dtype=np.float32)
        check(_lib.rsv_unet_get_params(self.handle, _ptr(out), 0), "rsv_unet_get_params")
        return out

    def grads(self):
        out = np.zeros(self.nparam, dtype=np.float32)
        check(_lib.rsv_unet_get_grads(self.handle, _ptr(out), 0), "rsv_unet_get_grads")
        return out

    def save(self, path):
        """Parameters, Adam moments and step count (rsv_unet_save)."""
        check(_lib.rsv_unet_save(self.handle, os.fsencode(path)), "rsv_unet_save")

    def load(self, path):
        check(_lib.rsv_unet_load(self.handle, os.fsencode(path)), "rsv_unet_load")

    def apply(self, rp, lnk, corr):
        """corr = s * U(rp / s, lnk); CUDA float64 tensors of nx*ny*nz values."""
        check(_lib.rsv_unet_apply(self.handle, _ptr(rp), _ptr(lnk), _ptr(corr)), "rsv_unet_apply")
        return corr

    def train_step(self, rp, lnk, target, lr):
        loss = ctypes.c_double()
        check(_lib.rsv_unet_train_step(self.handle, _ptr(rp), _ptr(lnk), _ptr(target), float(lr),
                                       ctypes.byref(loss)), "rsv_unet_train_step")
        return loss.value

    def train_batch(self, rps, lnks, targets, lr):
        """len(rps) training steps (CUDA float64 tensors), one synchronisation; returns the losses."""
        n = len(rps)
        arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        losses = np.zeros(n)
        check(_lib.rsv_unet_train_batch(self.handle, n, arr(rps), arr(lnks), arr(targets), float(lr),
                                        _ptr(losses)), "rsv_unet_train_batch")
        return losses

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.rsv_unet_destroy(h)
            self.handle = None
