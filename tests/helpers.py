"""Small dense helpers shared by the tests (brute-force references) and the library build hook."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_library():
    """Build librsv.so (loads the build script by path: the package import needs the library)."""
    spec = importlib.util.spec_from_file_location("rsv_build", os.path.join(ROOT, "paper_1602_05901_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def bsr_to_dense(row_ptr, col_idx, vals):
    nb = len(row_ptr) - 1
    A = np.zeros((3 * nb, 3 * nb))
    for r in range(nb):
        for p in range(row_ptr[r], row_ptr[r + 1]):
            c = col_idx[p]
            A[3 * r:3 * r + 3, 3 * c:3 * c + 3] = vals[p]
    return A


def stencil_to_dense(nx, ny, nz, a7):
    """Dense matrix of a seven-point stencil (slots -z,-y,-x,centre,+x,+y,+z)."""
    n = nx * ny * nz
    A = np.zeros((n, n))
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    for c in range(n):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        for s, (di, dj, dk) in enumerate(offs):
            ii, jj, kk = i + di, j + dj, k + dk
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                A[c, nx * ny * kk + nx * jj + ii] += a7[c, s]
    return A


def kron_bsr(nx, ny, nz, m_block, acc_block, trans=lambda c, o: 1.0):
    """BSR matrix sum_faces T (e_i - e_j) e_i^T (x) M + I (x) acc on the seven-point pattern."""
    import synth
    rp, ci = synth.seven_point_pattern(nx, ny, nz)
    nb = nx * ny * nz
    vals = np.zeros((len(ci), 3, 3))
    for r in range(nb):
        diag = np.array(acc_block, dtype=float).copy()
        dpos = None
        for p in range(rp[r], rp[r + 1]):
            c = ci[p]
            if c == r:
                dpos = p
                continue
            t = trans(r, c)
            vals[p] = -t * np.asarray(m_block)
            diag = diag + t * np.asarray(m_block)
        vals[dpos] = diag
    return rp, ci, vals


def per_entry_ratio(got, ref, floor=1e-3):
    """Largest per-entry error, each relative to its own reference magnitude:
    max_i |got_i - ref_i| / (|ref_i| + floor * rms(ref)).

    The floor (a fixed fraction of the RMS entry) keeps entries that are near
    zero from dominating; a wrong value in a handful of entries still shows at
    full size instead of being diluted by the vector's length as in a norm."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    rms = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    scale = np.abs(ref) + floor * rms
    scale[scale == 0] = 1.0
    return float(np.max(np.abs(got - ref) / scale)) if ref.size else 0.0


def report_ratio(name, value, bound):
    """Print an observed per-entry error beside its bound (pytest -s shows it)."""
    print(f"PER_ENTRY {name} {value:.3e} bound {bound:.1e}")
    return value
