"""Pins for the oracle's elimination of the well unknowns (Eq. Jacobian-system: reservoir
rows first, well rows last): the Schur complement A_RR - A_RW A_WW^-1 A_WR against a dense
computation, the reduced right-hand side and the recovered well unknowns against a dense
solve of the full system, and the rejected layouts."""
import numpy as np
import pytest

import oracle
from synthetic import box_jacobian, random_rhs


def _dense(a):
    return a.to_scipy().toarray()


@pytest.mark.parametrize("dims,b,wells", [((5, 4, 6), 3, 2), ((4, 4, 9), 4, 1), ((6, 3, 4), 2, 3)])
def test_schur_complement_and_recovery(dims, b, wells):
    a = box_jacobian(*dims, b, 7, n_wells=wells)
    W = oracle.Wells(a, wells)
    nr = a.nb - wells
    A = _dense(a)
    R, Wr = slice(0, nr * b), slice(nr * b, a.nb * b)
    S = A[R, R] - A[R, Wr] @ np.linalg.solve(A[Wr, Wr], A[Wr, R])
    rp, ci, v = W.reduced()
    Sg = np.zeros((nr * b, nr * b))
    for i in range(nr):
        for p in range(rp[i], rp[i + 1]):
            Sg[i * b:(i + 1) * b, ci[p] * b:(ci[p] + 1) * b] = v[p * b * b:(p + 1) * b * b].reshape(b, b)
    assert np.allclose(Sg, S, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    # pattern: A_RR's blocks and every pair of cells on one well
    rows = np.repeat(np.arange(a.nb), np.diff(a.row_ptr))
    want = {(i, j) for i, j in zip(rows, a.col_idx) if i < nr and j < nr}
    for w in range(wells):
        perf = [j for j in a.col_idx[a.row_ptr[nr + w]:a.row_ptr[nr + w + 1]] if j < nr]
        want |= {(c, d) for c in perf for d in perf}
    got = {(i, int(ci[p])) for i in range(nr) for p in range(rp[i], rp[i + 1])}
    assert got == want
    # reduced solve + recovery = full solve
    g = random_rhs(a, 3)
    g[nr * b:] = np.random.default_rng(3).normal(size=wells * b)
    x = np.linalg.solve(A, g)
    xs = np.linalg.solve(S, W.reduce_rhs(g))
    assert np.allclose(W.recover(g, xs), x, rtol=1e-10, atol=1e-10 * np.abs(x).max())
    # new values: the same relations hold
    v2 = a.values * (1.0 + 0.01 * np.random.default_rng(4).normal(size=a.values.shape))
    W.update_values(v2)
    a2 = a.__class__(**{**a.__dict__, "values": v2})
    A2 = _dense(a2)
    S2 = A2[R, R] - A2[R, Wr] @ np.linalg.solve(A2[Wr, Wr], A2[Wr, R])
    rp, ci, v = W.reduced()
    Sg2 = np.zeros_like(S2)
    for i in range(nr):
        for p in range(rp[i], rp[i + 1]):
            Sg2[i * b:(i + 1) * b, ci[p] * b:(ci[p] + 1) * b] = v[p * b * b:(p + 1) * b * b].reshape(b, b)
    assert np.allclose(Sg2, S2, rtol=1e-12, atol=1e-12 * np.abs(S2).max())


def _tiny(pairs, nb):
    """b = 1 matrix with the given symmetric off-diagonal pairs, diagonally dominant."""
    from synthetic import BSRMatrix
    rows = [[i] for i in range(nb)]
    for i, j in pairs:
        rows[i].append(j)
        rows[j].append(i)
    rp, ci, v = [0], [], []
    for i in range(nb):
        for j in sorted(rows[i]):
            ci.append(j)
            v.append(10.0 if j == i else -1.0)
        rp.append(len(ci))
    return BSRMatrix(nb=nb, b=1, row_ptr=np.array(rp, np.int32), col_idx=np.array(ci, np.int32),
                     values=np.array(v).reshape(-1, 1, 1))


def test_rejected_layouts():
    chain = [(0, 1), (1, 2)]
    oracle.Wells(_tiny(chain + [(1, 3), (2, 4)], 5), 2)               # one well per cell: fine
    with pytest.raises(oracle.OracleError):
        oracle.Wells(_tiny(chain + [(1, 3), (1, 4)], 5), 2)           # cell 1 on two wells
    with pytest.raises(oracle.OracleError):
        oracle.Wells(_tiny(chain + [(1, 3), (2, 4), (3, 4)], 5), 2)   # wells coupled
    a = box_jacobian(4, 4, 3, 2, 1, n_wells=2)
    with pytest.raises(oracle.OracleError):
        oracle.Wells(a, a.nb)                                          # no reservoir rows
