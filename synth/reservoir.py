"""Seeded, counter-based generator of reservoir Jacobians (inputs only).

The paper treats structured hexahedral grids whose cells are numbered
bottom-up, C(i,j,k) = nx*ny*k + nx*j + i (Section "Grid", equation for the
default index), with six face neighbours for interior cells and three to five
on the boundary.  It supports finite-volume discretisations but prints no
flux formula, so the Jacobian here follows a black-oil-like synthetic recipe:

* permeability k per cell (log-normal, layered or channelised), in mD;
* two-point transmissibility on unit cells, harmonic average of the two
  cells' permeabilities taken as plain numbers: T_ij = 2 k_i k_j / (k_i + k_j);
* per directed connection i->j an independent 3x3 mobility-like matrix M_ij
  whose off-diagonal entries are uniform(0.1, 1) draws and whose diagonal
  entries are a uniform(0.1, 1) draw plus the sum of their row's three draws,
  so M_ij is row-diagonally dominant and its eigenvalues have positive real
  part; off-diagonal block A_ij = -T_ij M_ij.  (With all nine entries i.i.d.
  the mean of M_ij is rank one, the two secondary unknowns see a diffusion of
  random sign, and the Jacobian is indefinite: Krylov solvers with any of the
  preconditioners here stagnate near relative residual 1.);
* diagonal block A_ii = diag(a_i) * PV/dt + sum_j T_ij M_ij with
  a_i[e] ~ uniform(1, 5) and PV/dt = 0.2 (porosity 0.2, unit volume, unit
  time step), so every block row sums to diag(a_i) * PV/dt (no-flow boundary);
* right-hand side b ~ N(0, 1) per unknown plus +/-1e3 well sources on the
  pressure equation (unknown 3c+0) of selected cells.

Unknowns are point-interleaved: unknown 3c+e, e=0 pressure, e=1,2 secondary.

Random numbers come from a counter-based generator: splitmix64 applied to a
key derived from (seed, stream) plus a per-value counter, giving 53-bit
uniforms; normals by the Box-Muller transform.  Every value is a pure function
of (seed, stream, index), so the arrays do not depend on generation order,
chunking or platform integer semantics.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem", "make_problem", "perm_lognormal", "perm_layered", "perm_channelized",
    "assemble_jacobian", "accumulation_blocks", "seven_point_pattern", "nnzb_of", "uniform01", "std_normal",
    "WORKLOADS", "workload", "batch_sizes",
]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
PV_OVER_DT = 0.2          # porosity 0.2 x unit cell volume / unit time step
WELL_RATE = 1.0e3

# random streams (one per independent quantity)
S_LNK, S_LAYER, S_ACC, S_RHS, S_CHAN, S_WELL, S_MOB0 = 1, 2, 3, 4, 5, 6, 10


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea & Flood 2014) on a uint64 array, wrapping."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    k = np.array([(seed & 0xFFFFFFFF) | ((stream & 0xFFFFFFFF) << 32)], dtype=np.uint64)
    return _splitmix64(_splitmix64(k))[0]


def uniform01(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of splitmix64(key(seed, stream) + idx)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _splitmix64(idx + _key(seed, stream))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def std_normal(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Standard normals by Box-Muller from the uniform pair at counters 2*idx, 2*idx+1."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = uniform01(seed, stream, idx * np.uint64(2))
    u2 = uniform01(seed, stream, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- grid

def nnzb_of(nx: int, ny: int, nz: int) -> int:
    """Block non-zeros of the seven-point pattern: diagonal plus two per interior face."""
    return nx * ny * nz + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))


def seven_point_pattern(nx: int, ny: int, nz: int):
    """BSR pattern of the seven-point stencil in bottom-up cell order.

    Returns (row_ptr int32 [nb+1], col_idx int32 [nnzb]) with each row's
    columns ascending: -z, -y, -x, self, +x, +y, +z (missing faces skipped).
    """
    nb = nx * ny * nz
    c = np.arange(nb, dtype=np.int64)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    offs = [(-nx * ny, k > 0), (-nx, j > 0), (-1, i > 0), (0, np.ones(nb, bool)),
            (1, i < nx - 1), (nx, j < ny - 1), (nx * ny, k < nz - 1)]
    present = np.stack([m for _, m in offs], axis=1)            # [nb, 7]
    cols = c[:, None] + np.array([o for o, _ in offs], dtype=np.int64)[None, :]
    counts = present.sum(axis=1)
    row_ptr = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols[present]
    assert row_ptr[-1] == nnzb_of(nx, ny, nz)
    return row_ptr.astype(np.int32), col_idx.astype(np.int32)


# ------------------------------------------------------------------ permeability

def perm_lognormal(nx, ny, nz, seed, sigma=1.0, mean_md=100.0):
    """ln k ~ N(ln mean, sigma^2), independent per cell."""
    nb = nx * ny * nz
    return math.log(mean_md) + sigma * std_normal(seed, S_LNK, np.arange(nb))


def perm_layered(nx, ny, nz, seed, layer_sigma=1.5, within_sigma=0.5, mean_md=100.0):
    """Per-layer mean ln k ~ N(ln mean, layer_sigma^2); within a layer sigma = within_sigma."""
    nb = nx * ny * nz
    mu = math.log(mean_md) + layer_sigma * std_normal(seed, S_LAYER, np.arange(nz))
    k = np.arange(nb) // (nx * ny)
    return mu[k] + within_sigma * std_normal(seed, S_LNK, np.arange(nb))


def perm_channelized(nx, ny, nz, seed, sigma=2.0, nchannels=5, width=8, height=4,
                     factor=100.0, mean_md=100.0):
    """Log-normal field plus x-aligned high-permeability streaks (k multiplied by factor).

    Each streak spans the full x length, `width` cells in y and `height` in z,
    from a seeded corner; overlapping streaks multiply once per cell.
    """
    lnk = perm_lognormal(nx, ny, nz, seed, sigma, mean_md).reshape(nz, ny, nx)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    u = uniform01(seed, S_CHAN, np.arange(2 * nchannels))
    for s in range(nchannels):
        j0 = int(u[2 * s] * max(ny - width + 1, 1))
        k0 = int(u[2 * s + 1] * max(nz - height + 1, 1))
        mask[k0:k0 + height, j0:j0 + width, :] = True
    lnk[mask] += math.log(factor)
    return lnk.reshape(-1)


# ---------------------------------------------------------------------- Jacobian

def accumulation_blocks(nb, seed, pv_over_dt=PV_OVER_DT):
    """The accumulation (time-derivative) part of every cell's diagonal block,
    diag(a_c) * PV/dt with a_c[e] ~ uniform(1, 5): float64 [nb, 3, 3]."""
    a = 1.0 + 4.0 * uniform01(seed, S_ACC, np.arange(3 * nb)).reshape(nb, 3)
    acc = np.zeros((nb, 3, 3), dtype=np.float64)
    acc[:, [0, 1, 2], [0, 1, 2]] = a * pv_over_dt
    return acc


def assemble_jacobian(nx, ny, nz, lnk, seed, pv_over_dt=PV_OVER_DT):
    """Assemble the 3x3-block Jacobian in BSR form (values float64 [nnzb, 3, 3], row-major blocks).

    Mobility matrix of the connection from cell c to its neighbour in face
    direction d (0:-z 1:-y 2:-x 3:+x 4:+y 5:+z) draws counters 9*c + 3*e + f of
    stream S_MOB0 + d, so M_ij and M_ji are independent.
    """
    nb = nx * ny * nz
    row_ptr, col_idx = seven_point_pattern(nx, ny, nz)
    kd = np.exp(np.asarray(lnk, dtype=np.float64))
    vals = np.zeros((int(row_ptr[-1]), 3, 3), dtype=np.float64)
    c = np.arange(nb, dtype=np.int64)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    diag = accumulation_blocks(nb, seed, pv_over_dt)
    dirs = [(-nx * ny, k > 0), (-nx, j > 0), (-1, i > 0), (1, i < nx - 1), (nx, j < ny - 1),
            (nx * ny, k < nz - 1)]
    # position of each neighbour in the row: columns are ascending, so count present
    # entries before it (the diagonal sits after the three lower neighbours)
    present = np.stack([m for _, m in dirs], axis=1)
    slot_of = np.zeros((nb, 6), dtype=np.int64)
    run = np.zeros(nb, dtype=np.int64)
    for d in range(6):
        if d == 3:
            diag_slot = run.copy()
            run += 1
        slot_of[:, d] = run
        run += present[:, d]
    for d, (off, m) in enumerate(dirs):
        src = c[m]
        dst = src + off
        t = 2.0 * kd[src] * kd[dst] / (kd[src] + kd[dst])
        cnt = (9 * src)[:, None] + np.arange(9, dtype=np.int64)[None, :]
        mob = (0.1 + 0.9 * uniform01(seed, S_MOB0 + d, cnt.reshape(-1))).reshape(-1, 3, 3)
        mob[:, [0, 1, 2], [0, 1, 2]] += mob.sum(axis=2)
        blk = -t[:, None, None] * mob
        vals[row_ptr[src] + slot_of[src, d]] = blk
        diag[src] -= blk
    vals[row_ptr[:-1] + diag_slot] = diag
    return row_ptr, col_idx, vals


# ------------------------------------------------------------------- workloads

@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    row_ptr: np.ndarray   # int32 [nb+1]
    col_idx: np.ndarray   # int32 [nnzb]
    vals: np.ndarray      # float64 [nnzb, 3, 3]
    b: np.ndarray         # float64 [3*nb]
    lnk: np.ndarray       # float64 [nb]
    seed: int = 0
    pv_over_dt: float = PV_OVER_DT

    def accumulation(self):
        """Accumulation blocks [nb, 3, 3] of the assembled Jacobian (the input of true-IMPES)."""
        return accumulation_blocks(self.nb, self.seed, self.pv_over_dt)

    @property
    def nb(self):
        return self.nx * self.ny * self.nz

    @property
    def n(self):
        return 3 * self.nb

    @property
    def nnzb(self):
        return int(self.row_ptr[-1])


def _rhs(nb, seed, wells):
    b = std_normal(seed, S_RHS, np.arange(3 * nb))
    for cell, sign in wells:
        b[3 * cell] += sign * WELL_RATE
    return b


def corner_wells(nx, ny, nz):
    """Producer/injector pair at the two opposite corner cells."""
    return [(0, +1.0), (nx * ny * nz - 1, -1.0)]


def seeded_wells(nx, ny, nz, seed, count=16):
    """`count` distinct seeded cells with alternating source sign."""
    nb = nx * ny * nz
    cells, t = [], 0
    while len(cells) < count:
        cand = int(uniform01(seed, S_WELL, np.array([t]))[0] * nb)
        t += 1
        if cand not in cells:
            cells.append(cand)
    return [(cnum, 1.0 if s % 2 == 0 else -1.0) for s, cnum in enumerate(cells)]


def make_problem(nx, ny, nz, seed, perm="lognormal", sigma=1.0, wells="corner",
                 pv_over_dt=PV_OVER_DT):
    if perm == "lognormal":
        lnk = perm_lognormal(nx, ny, nz, seed, sigma)
    elif perm == "layered":
        lnk = perm_layered(nx, ny, nz, seed)
    elif perm == "channelized":
        lnk = perm_channelized(nx, ny, nz, seed, sigma=sigma)
    else:
        raise ValueError(f"unknown permeability recipe {perm!r}")
    row_ptr, col_idx, vals = assemble_jacobian(nx, ny, nz, lnk, seed, pv_over_dt)
    w = corner_wells(nx, ny, nz) if wells == "corner" else seeded_wells(nx, ny, nz, seed)
    return Problem(nx, ny, nz, row_ptr, col_idx, vals, _rhs(nx * ny * nz, seed, w), lnk, seed, pv_over_dt)


# Named workloads (grid, permeability recipe, seed, wells).
WORKLOADS = {
    "tiny_20x20x10": dict(nx=20, ny=20, nz=10, seed=0, perm="lognormal", sigma=1.0, wells="corner"),
    "mid_100x100x50": dict(nx=100, ny=100, nz=50, seed=1, perm="layered", wells="corner"),
    "large_256x256x128": dict(nx=256, ny=256, nz=128, seed=2, perm="channelized", sigma=2.0,
                              wells="seeded"),
    "learned_128x128x64": dict(nx=128, ny=128, nz=64, seed=10000, perm="channelized", sigma=2.0,
                               wells="seeded"),
}


def workload(name, **override):
    cfg = dict(WORKLOADS[name])
    cfg.update(override)
    return make_problem(**cfg)


def batch_sizes(count=64, seed=3):
    """Uneven ensemble grid sizes: nx, ny ~ U{16..96}, nz ~ U{16..48}, independently."""
    u = uniform01(seed, S_LNK, np.arange(3 * count)).reshape(count, 3)
    nx = 16 + (u[:, 0] * 81).astype(int)
    ny = 16 + (u[:, 1] * 81).astype(int)
    nz = 16 + (u[:, 2] * 33).astype(int)
    return [(int(a), int(b), int(c)) for a, b, c in zip(nx, ny, nz)]


S_NET = 20  # stream of the network's initial weights


def unet_init(base=32, levels=4, seed=0, cin=2):
    """Initial parameters of the learned stage's U-Net as one float32 array.

    He-normal weights (standard deviation sqrt(2 / fan_in)) and zero biases,
    drawn from the counter-based generator, laid out per layer as weight then
    bias in the order enc1a, enc1b, ..., encLb, dec(L-1)a, dec(L-1)b, ...,
    dec1a, dec1b, head (3x3x3 weights [co][27][ci], head [1][base]).
    """
    ch = [base << l for l in range(levels)]
    shapes = []
    prev = cin
    for l in range(levels):
        shapes += [(ch[l], prev, 27), (ch[l], ch[l], 27)]
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        shapes += [(ch[l], ch[l + 1] + ch[l], 27), (ch[l], ch[l], 27)]
    shapes.append((1, ch[0], 1))
    parts = []
    off = 0
    for co, ci, taps in shapes:
        nw = co * ci * taps
        w = std_normal(seed, S_NET, np.arange(off, off + nw)) * np.sqrt(2.0 / (taps * ci))
        if taps == 1:
            w = w * 0.1  # a small head: the untrained stage starts near zero
        parts += [w, np.zeros(co)]
        off += nw
    return np.concatenate(parts).astype(np.float32)
