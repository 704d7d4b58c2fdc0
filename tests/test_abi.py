"""The C ABI library loads and exports every entry point the header declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("rsv.h", "rsv_unet.h")]


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"RSV_API\s+[\w\s\*]*?\b(rsv_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from tests.helpers import build_library
    path = build_library()
    return ctypes.CDLL(path), path


# The boundary's calls: grid, BSR matrix, vectors, solver, preconditioner setup,
# solve (single and batched), the learned stage's checkpoints, destroy calls.
BOUNDARY = ("rsv_grid_create", "rsv_grid_destroy", "rsv_mat_create_bsr", "rsv_mat_get_pattern", "rsv_mat_set_values",
            "rsv_mat_destroy", "rsv_vec_create", "rsv_vec_wrap", "rsv_vec_set", "rsv_vec_get", "rsv_vec_destroy",
            "rsv_solver_create", "rsv_solver_destroy", "rsv_precond_setup", "rsv_solve", "rsv_solve_batched",
            "rsv_unet_load", "rsv_unet_save", "rsv_status_string", "rsv_spmv")


def test_header_declares_entry_points():
    names = declared_functions()
    for must in BOUNDARY + ("rsv_mat_create", "rsv_solve_ptr", "rsv_solve_batched_ptr"):
        assert must in names, must


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(rsv_\w+)", out))
    assert exported == set(declared_functions())


def test_binding_covers_exports(lib):
    import paper_1602_05901_gb300 as rsv
    assert set(rsv.EXPORTS) == set(declared_functions())


def test_host_side_argument_checks_without_gpu(lib):
    import paper_1602_05901_gb300 as rsv
    g = ctypes.c_void_p()
    assert rsv.rsv_grid_create(0, 4, 4, ctypes.byref(g)) == rsv.RSV_EINVAL
    assert rsv.rsv_grid_create(4, 4, 4, None) == rsv.RSV_EINVAL
    assert rsv.rsv_grid_create(2000, 2000, 2000, ctypes.byref(g)) == rsv.RSV_EINVAL
    assert rsv.rsv_grid_create(3, 2, 1, ctypes.byref(g)) == rsv.RSV_OK
    rsv.rsv_grid_destroy(g)
    assert rsv.rsv_mat_create(None, None, ctypes.byref(g)) == rsv.RSV_EINVAL
    assert rsv.rsv_solver_create(None, None, ctypes.byref(g)) == rsv.RSV_EINVAL
    assert rsv.rsv_precond_setup(None, 1, None) == rsv.RSV_EINVAL
    assert rsv.rsv_solve(None, None, None, None) == rsv.RSV_EINVAL
    assert rsv.rsv_solve_ptr(None, None, None, 0, None) == rsv.RSV_EINVAL
    assert rsv.rsv_solve_batched(None, None, None, None) == rsv.RSV_EINVAL
    # the BSR matrix: block size 3 only, FP64 or mixed storage (checked before any device call)
    assert rsv.rsv_grid_create(3, 2, 1, ctypes.byref(g)) == rsv.RSV_OK
    m = ctypes.c_void_p()
    assert rsv.rsv_mat_create_bsr(g, 4, rsv.RSV_PREC_FP64, None, ctypes.byref(m)) == rsv.RSV_ENOTSUP
    assert rsv.rsv_mat_create_bsr(g, 3, 7, None, ctypes.byref(m)) == rsv.RSV_EINVAL
    assert rsv.rsv_mat_create_bsr(None, 3, rsv.RSV_PREC_FP64, None, ctypes.byref(m)) == rsv.RSV_EINVAL
    v = ctypes.c_void_p()
    assert rsv.rsv_vec_create(g, 7, None, ctypes.byref(v)) == rsv.RSV_EINVAL
    assert rsv.rsv_vec_create(None, rsv.RSV_PREC_FP64, None, ctypes.byref(v)) == rsv.RSV_EINVAL
    rsv.rsv_grid_destroy(g)
    assert rsv.rsv_vec_wrap(None, 10, rsv.RSV_PREC_FP64, ctypes.byref(v)) == rsv.RSV_EINVAL
    assert rsv.rsv_vec_wrap(None, -1, rsv.RSV_PREC_FP64, ctypes.byref(v)) == rsv.RSV_EINVAL
    assert rsv.rsv_vec_set(None, None, 0, None) == rsv.RSV_EINVAL
    assert rsv.rsv_vec_get(None, None, 0, None) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_save(None, b"/nonexistent") == rsv.RSV_EINVAL
    assert rsv.rsv_unet_load(None, b"/nonexistent") == rsv.RSV_EINVAL
    assert rsv.status_string(rsv.RSV_ENOCONV) == "not converged within maxit"
    p = rsv.solver_params()
    assert (p.restart, p.rtol, p.maxit, p.btol) == (30, 1e-8, 2000, 1e-30)


def test_unet_and_conv_argument_checks_without_gpu(lib):
    import paper_1602_05901_gb300 as rsv
    h = ctypes.c_void_p()
    # nx / 2^(levels-1) must be a multiple of 8; base a multiple of 32; 1 <= levels <= 5
    assert rsv.rsv_unet_create(None, 60, 16, 8, 32, 3, ctypes.byref(h)) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_create(None, 64, 16, 8, 16, 3, ctypes.byref(h)) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_create(None, 64, 16, 8, 32, 6, ctypes.byref(h)) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_create(None, 64, 15, 8, 32, 3, ctypes.byref(h)) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_create(None, 64, 16, 8, 32, 3, None) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_apply(None, None, None, None) == rsv.RSV_EINVAL
    assert rsv.rsv_unet_train_step(None, None, None, None, 1e-3, None) == rsv.RSV_EINVAL


def _header_enum(name):
    """{member: value} of a `typedef enum {...} name;` in include/rsv.h."""
    text = open(HEADERS[0]).read()
    body = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return {m: int(v) for m, v in re.findall(r"(RSV_\w+)\s*=\s*(\d+)", body)}


def _header_struct_fields(name):
    text = open(HEADERS[0]).read()
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"\b(\w+)\s*;", body)


def test_binding_constants_and_structs_match_the_header(lib):
    """The binding's preconditioner and status codes and its ctypes mirror of
    rsv_pc_params follow the header (field order and count: the struct is passed by pointer)."""
    import paper_1602_05901_gb300 as rsv
    pcs = _header_enum("rsv_pc_type")
    assert pcs == {n: getattr(rsv, n) for n in pcs}
    assert set(rsv.PC_TYPES.values()) == set(pcs.values())
    statuses = _header_enum("rsv_status")
    assert all(getattr(rsv, n) == v for n, v in statuses.items())
    fields = _header_struct_fields("rsv_pc_params")
    assert fields == [f for f, _ in rsv.rsv_pc_params._fields_]
    p = rsv.pc_params()
    assert (p.gmg_max_levels, p.gmg_max_coarse, p.gmg_sweeps, p.decoupling) == (6, 512, 2, 0)
    assert rsv.pc_params(decoupling="abf").decoupling == 1
