"""The seeded generators: structure of the synthetic Jacobians (sorted columns, diagonal
present, symmetric pattern, wells after the cells) and the SPE10-shaped counts."""
import numpy as np

from synthetic import (box_jacobian, grid_small, grid_spe10, newton_sequence, perturb_values,
                       random_rhs)


def _pattern_ok(a):
    rp, ci = a.row_ptr, a.col_idx
    assert rp[0] == 0 and rp[-1] == len(ci)
    for i in range(a.nb):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and i in row


def test_small_grid_shape():
    a = grid_small()
    assert (a.nb, a.b, a.nnzb) == (2048, 3, 13312)
    _pattern_ok(a)
    assert np.array_equal(grid_small().values, a.values)  # seeded


def test_spe10_counts_formula():
    # 60x220x85 cells + 4 wells: nnzb = cells + 2*faces + 2*4*85
    nx, ny, nz = 60, 220, 85
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert nx * ny * nz + 4 == 1122004
    assert nx * ny * nz + 4 + 2 * faces + 2 * 4 * nz == 7780684
    a = grid_spe10(nx=6, ny=7, nz=5)
    faces = 5 * 7 * 5 + 6 * 6 * 5 + 6 * 7 * 4
    assert a.nnzb == 6 * 7 * 5 + 4 + 2 * faces + 2 * 4 * 5
    _pattern_ok(a)
    rows = np.repeat(np.arange(a.nb), np.diff(a.row_ptr))
    st = set(zip(rows.tolist(), a.col_idx.tolist()))
    assert all((j, i) in st for i, j in st)


def test_perturbation_and_rhs():
    a = box_jacobian(5, 4, 3, 4, 3, n_wells=2)
    v = perturb_values(a, 1)
    rows = np.repeat(np.arange(a.nb), np.diff(a.row_ptr))
    off = rows != a.col_idx
    r = v[off] / a.values[off]
    ok = a.values[off] != 0
    assert np.all((r[ok] >= 0.95) & (r[ok] <= 1.05))
    # block row sums (the accumulation terms) are unchanged
    s0 = np.zeros((a.nb, a.b, a.b))
    s1 = np.zeros((a.nb, a.b, a.b))
    np.add.at(s0, rows, a.values)
    np.add.at(s1, rows, v)
    assert np.allclose(s0, s1, rtol=1e-12, atol=1e-9)
    rhs = random_rhs(a, 2).reshape(a.nb, a.b)
    assert np.all(rhs[a.n_cells:, 1:] == 0.0)


def test_newton_sequence_drift():
    a = box_jacobian(5, 4, 3, 4, 3, n_wells=2)
    seq = newton_sequence(a, 3, 2, seed=9, rel_newton=0.02, rel_step=0.2)
    assert len(seq) == 6
    again = newton_sequence(a, 3, 2, seed=9, rel_newton=0.02, rel_step=0.2)
    assert all(np.array_equal(x, y) for x, y in zip(seq, again))
    rows = np.repeat(np.arange(a.nb), np.diff(a.row_ptr))
    off = rows != a.col_idx
    prev = a.values
    for k, v in enumerate(seq):
        rel = 0.2 if k % 2 == 0 else 0.02
        ok = prev[off] != 0
        r = v[off][ok] / prev[off][ok]
        assert np.all((r >= 1 - rel) & (r <= 1 + rel))  # each step perturbs the previous one
        s0 = np.zeros((a.nb, a.b, a.b))
        s1 = np.zeros((a.nb, a.b, a.b))
        np.add.at(s0, rows, a.values)
        np.add.at(s1, rows, v)
        assert np.allclose(s0, s1, rtol=1e-12, atol=1e-9)  # accumulation terms kept
        prev = v
    # the drift accumulates: the last Jacobian is further from the first than the second is
    d1 = np.abs(seq[1][off] - seq[0][off]).sum()
    d5 = np.abs(seq[5][off] - seq[0][off]).sum()
    assert d5 > d1
