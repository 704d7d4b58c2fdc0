"""Invariants of the synthetic Jacobian generator (inputs for both sides)."""
import numpy as np
import pytest

import synth
from synth import reservoir as R


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 1), (4, 3, 2), (5, 1, 1), (7, 6, 5)])
def test_pattern_counts_and_order(dims):
    rp, ci = synth.seven_point_pattern(*dims)
    nx, ny, nz = dims
    assert rp[-1] == synth.nnzb_of(*dims) == len(ci)
    for r in range(nx * ny * nz):
        cols = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(cols) > 0) and r in cols
        i, j, k = r % nx, (r // nx) % ny, r // (nx * ny)
        expect = 1 + (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1)
        assert len(cols) == expect


def test_nnzb_matches_table():
    # block counts for the 20x20x10, 100x100x50 and 256x256x128 grids
    assert synth.nnzb_of(20, 20, 10) == 26400
    assert synth.nnzb_of(100, 100, 50) == 3460000
    assert synth.nnzb_of(256, 256, 128) == 58458112


def test_block_row_sums_equal_accumulation():
    """Each block row sums to diag(a_i) PV/dt: fluxes cancel (no-flow boundary)."""
    p = synth.make_problem(6, 5, 4, seed=3)
    sums = np.zeros((p.nb, 3, 3))
    rows = np.repeat(np.arange(p.nb), np.diff(p.row_ptr))
    np.add.at(sums, rows, p.vals)
    off = sums.copy()
    off[:, [0, 1, 2], [0, 1, 2]] = 0
    assert np.abs(off).max() < 1e-12 * np.abs(p.vals).max()
    acc = sums[:, [0, 1, 2], [0, 1, 2]] / R.PV_OVER_DT
    assert acc.min() >= 1.0 and acc.max() <= 5.0


def test_transmissibility_harmonic_and_symmetric():
    nx, ny, nz = 4, 3, 2
    lnk = np.log(np.arange(1, nx * ny * nz + 1, dtype=float))
    rp, ci, vals = R.assemble_jacobian(nx, ny, nz, lnk, seed=9)
    k = np.exp(lnk)
    for r in range(nx * ny * nz):
        for q in range(rp[r], rp[r + 1]):
            c = ci[q]
            if c == r:
                continue
            t = 2 * k[r] * k[c] / (k[r] + k[c])
            m = -vals[q] / t
            # off-diagonal mobility entries in [0.1, 1), diagonal = draw + row sum of draws
            offd = m[~np.eye(3, dtype=bool)]
            assert offd.min() >= 0.1 - 1e-12 and offd.max() < 1.0 + 1e-12
            assert np.all(np.diag(m) > m.sum(axis=1) - np.diag(m))  # row dominant


def test_equal_permeability_gives_t_equal_k():
    nx, ny, nz = 3, 2, 2
    lnk = np.full(nx * ny * nz, np.log(250.0))
    rp, ci, vals = R.assemble_jacobian(nx, ny, nz, lnk, seed=1)
    # each off-diagonal block is -250 * M with M entries >= 0.1: recover T from the
    # block's smallest off-diagonal-of-M entry bound
    for q in range(len(ci)):
        blk = vals[q]
        if np.any(blk < 0):
            m = -blk / 250.0
            assert m[~np.eye(3, dtype=bool)].min() >= 0.1 - 1e-12


def test_rng_is_counter_based_and_uniform():
    a = synth.uniform01(7, 3, np.arange(100000))
    b = synth.uniform01(7, 3, np.arange(50000, 100000))
    assert np.array_equal(a[50000:], b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.005 and abs(a.var() - 1 / 12) < 0.002
    z = synth.std_normal(7, 4, np.arange(200000))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_wells_and_rhs():
    p = synth.make_problem(5, 4, 3, seed=0)
    assert p.b[0] > 500 and p.b[3 * (p.nb - 1)] < -500
    q = synth.make_problem(8, 8, 8, seed=2, wells="seeded")
    big = np.flatnonzero(np.abs(q.b) > 200)
    assert len(big) == 16 and np.all(big % 3 == 0)


def test_batch_sizes_range():
    sizes = synth.batch_sizes()
    assert len(sizes) == 64
    for nx, ny, nz in sizes:
        assert 16 <= nx <= 96 and 16 <= ny <= 96 and 16 <= nz <= 48
