"""Pins for the oracle's PGS-MC (Algorithm 4.3) and block ILU(0) (stage R of Eq. MSP).

* A forward multi-colour sweep from x = 0 solves (D + L) x = b in colour order, and a
  backward sweep solves (D + U) x_new = b - L x_old: both checked against SciPy's
  triangular solver.
* g = n (one colour per vertex) is the classical GS (Section 4.1).
* The vertices of one colour are independent: a vectorised Jacobi update per colour
  class reproduces the sequential sweep.
* ILU(0) of a block tridiagonal chain in natural order has no fill, so it is the exact
  LU; in red-black order on a 7-point grid the black pivots have the closed form
  A_bb - sum_r A_br A_rr^-1 A_rb (only the Schur diagonal survives ILU(0)).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle
from synthetic import box_jacobian, chain_bsr, poisson3d_bsr, random_rhs


def _colour_ordered_csr(a_csr, rp, ci):
    n = a_csr.shape[0]
    colour, g = oracle.vertices_grouping(n, rp, ci)
    perm = np.lexsort((np.arange(n), colour))
    ap = a_csr[perm][:, perm].tocsr()
    ap.sort_indices()
    cptr = np.zeros(g + 1, np.int32)
    np.cumsum(np.bincount(colour, minlength=g + 1)[1:], out=cptr[1:])
    return ap, cptr


def _scalar_pressure_like(seed, dims=(9, 7, 5)):
    a = box_jacobian(*dims, 1, seed, layered=True, kz_ratio=0.1, n_wells=2)
    m = a.to_scipy().tocsr()
    return m, a


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_forward_sweep_is_lower_triangular_solve(seed):
    m, a = _scalar_pressure_like(seed)
    ap, cptr = _colour_ordered_csr(m, a.row_ptr, a.col_idx)
    b = np.random.default_rng(seed).normal(size=m.shape[0])
    x = oracle.pgs_mc(ap.indptr, ap.indices, ap.data, cptr, b, np.zeros_like(b), True)
    ref = spl.spsolve_triangular(sp.tril(ap).tocsr(), b, lower=True)
    assert np.allclose(x, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("seed", [4, 5])
def test_backward_sweep_is_upper_triangular_solve(seed):
    m, a = _scalar_pressure_like(seed)
    ap, cptr = _colour_ordered_csr(m, a.row_ptr, a.col_idx)
    rng = np.random.default_rng(seed)
    b, x0 = rng.normal(size=m.shape[0]), rng.normal(size=m.shape[0])
    x = oracle.pgs_mc(ap.indptr, ap.indices, ap.data, cptr, b, x0, False)
    rhs = b - sp.tril(ap, k=-1) @ x0
    ref = spl.spsolve_triangular(sp.triu(ap).tocsr(), rhs, lower=False)
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_one_colour_per_vertex_is_classical_gs():
    m, a = _scalar_pressure_like(7, (6, 5, 4))
    n = m.shape[0]
    m = m.tocsr()
    m.sort_indices()
    cptr = np.arange(n + 1, dtype=np.int32)
    b = np.random.default_rng(0).normal(size=n)
    x = oracle.pgs_mc(m.indptr, m.indices, m.data, cptr, b, np.zeros(n), True)
    ref = spl.spsolve_triangular(sp.tril(m).tocsr(), b, lower=True)
    assert np.allclose(x, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("seed", [8, 9])
def test_colour_classes_update_independently(seed):
    m, a = _scalar_pressure_like(seed)
    ap, cptr = _colour_ordered_csr(m, a.row_ptr, a.col_idx)
    rng = np.random.default_rng(seed)
    b, x0 = rng.normal(size=m.shape[0]), rng.normal(size=m.shape[0])
    x = oracle.pgs_mc(ap.indptr, ap.indices, ap.data, cptr, b, x0, True)
    d = ap.diagonal()
    off = (ap - sp.diags(d)).tocsr()
    y = x0.copy()
    for c in range(len(cptr) - 1):
        s = slice(cptr[c], cptr[c + 1])
        y[s] = (b[s] - off[s] @ y) / d[s]  # whole colour class at once
    assert np.allclose(x, y, rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_bilu_exact_on_chain_in_natural_order():
    a = chain_bsr(40, 3, 11)
    o = oracle.Oracle(a, precond=oracle.PREC_R_ONLY, bilu_order=1)
    g = np.random.default_rng(1).normal(size=a.n)
    w = o.apply_precond(g)
    ref = np.linalg.solve(a.to_dense(), g)
    assert np.allclose(w, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    x, info = o.solve(g, tol=1e-10)
    assert info["iterations"] == 1


def test_bilu_red_black_closed_form():
    a = box_jacobian(6, 5, 4, 2, 13)  # no wells: red-black colouring
    o = oracle.Oracle(a, precond=oracle.PREC_R_ONLY)
    colour, g = o.colour0()
    assert g == 2
    perm = np.lexsort((np.arange(a.nb), colour))
    piv = o.bilu_pivots()  # colour order
    blocks = {}
    for i in range(a.nb):
        for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
            blocks[(i, int(a.col_idx[p]))] = a.values[p]
    for k, i in enumerate(perm):
        if colour[i] == 1:
            ref = blocks[(i, i)]
        else:
            ref = blocks[(i, i)].copy()
            for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
                r = int(a.col_idx[p])
                if r != i:
                    ref = ref - blocks[(i, r)] @ np.linalg.solve(blocks[(r, r)], blocks[(r, i)])
        assert np.allclose(piv[k], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), k


def _concentration_split(a, perm, iperm):
    """Block lower (diagonal included) and strictly upper parts of Pi_N^T A Pi_N in colour
    order, dense."""
    bn = a.b - 1
    L = np.zeros((a.nb * bn, a.nb * bn))
    U = np.zeros_like(L)
    for i in range(a.nb):
        for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
            j = int(a.col_idx[p])
            M = L if iperm[j] <= iperm[i] else U
            M[iperm[i] * bn:(iperm[i] + 1) * bn, iperm[j] * bn:(iperm[j] + 1) * bn] = \
                a.values[p][1:, 1:]
    return L, U


@pytest.mark.parametrize("sweeps", [3, 6])
def test_stage_n_sweeps_are_the_block_gs_iteration(sweeps):
    """k forward sweeps from zero are k steps of the block Gauss-Seidel splitting
    (D + L_A) x_{s+1} = r - U_A x_s of Pi_N^T A Pi_N in colour order."""
    a = box_jacobian(5, 4, 3, 3, 17, n_wells=1)
    o = oracle.Oracle(a, precond=oracle.PREC_N_ONLY, bgs_sweeps=sweeps)
    colour, g = o.colour0()
    perm = np.lexsort((np.arange(a.nb), colour))
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(a.nb)
    gvec = random_rhs(a, 2)
    w = o.apply_precond(gvec).reshape(a.nb, a.b)
    assert np.all(w[:, 0] == 0.0)
    L, U = _concentration_split(a, perm, iperm)
    rhs = gvec.reshape(a.nb, a.b)[perm][:, 1:].reshape(-1)
    x = np.zeros_like(rhs)
    for _ in range(sweeps):
        x = np.linalg.solve(L, rhs - U @ x)
    ref = x.reshape(a.nb, a.b - 1)
    assert np.allclose(w[perm][:, 1:], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_stage_n_is_block_gs_on_concentration_subsystem():
    """Stage N with one forward sweep from zero solves the block lower-triangular part
    of Pi_N^T A Pi_N (colour order) exactly; the pressure slot is untouched."""
    a = box_jacobian(5, 4, 3, 3, 17, n_wells=1)
    o = oracle.Oracle(a, precond=oracle.PREC_N_ONLY, bgs_sweeps=1)
    colour, g = o.colour0()
    perm = np.lexsort((np.arange(a.nb), colour))
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(a.nb)
    gvec = random_rhs(a, 2)
    w = o.apply_precond(gvec).reshape(a.nb, a.b)
    assert np.all(w[:, 0] == 0.0)
    bn = a.b - 1
    L = np.zeros((a.nb * bn, a.nb * bn))
    for i in range(a.nb):
        for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
            j = int(a.col_idx[p])
            if iperm[j] <= iperm[i]:
                L[iperm[i] * bn:(iperm[i] + 1) * bn, iperm[j] * bn:(iperm[j] + 1) * bn] = \
                    a.values[p][1:, 1:]
    rhs = gvec.reshape(a.nb, a.b)[perm][:, 1:].reshape(-1)
    ref = np.linalg.solve(L, rhs).reshape(a.nb, bn)
    assert np.allclose(w[perm][:, 1:], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


# ---- the smoothers the paper compares PGS-MC with (Section 5.1.1, Table 2)

@pytest.mark.parametrize("seed", [1, 2])
def test_jacobi_sweep_closed_form(seed):
    """PJAC-NO: x1 = D^-1 (b - (A - D) x0); from zero it is D^-1 b."""
    m, a = _scalar_pressure_like(seed)
    rng = np.random.default_rng(seed)
    b, x0 = rng.normal(size=m.shape[0]), rng.normal(size=m.shape[0])
    d = m.diagonal()
    x = oracle.jacobi_sweep(m.indptr, m.indices, m.data, b, x0)
    ref = (b - (m @ x0 - d * x0)) / d
    assert np.allclose(x, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    x = oracle.jacobi_sweep(m.indptr, m.indices, m.data, b, np.zeros_like(b))
    assert np.allclose(x, b / d, rtol=1e-15, atol=0)


@pytest.mark.parametrize("seed,forward", [(1, True), (2, False), (3, True)])
def test_pgs_no_sweep_is_block_jacobi_of_triangular_solves(seed, forward):
    """PGS-NO: every chunk of 16 rows solves its lower (forward) or upper (backward)
    triangle with the rest of its rows and the other chunks at their old values."""
    m, a = _scalar_pressure_like(seed)
    n = m.shape[0]
    rng = np.random.default_rng(seed)
    b, x0 = rng.normal(size=n), rng.normal(size=n)
    x = oracle.pgs_no_sweep(m.indptr, m.indices, m.data, b, x0, forward)
    c = oracle.PGS_NO_CHUNK
    ref = np.empty(n)
    for c0 in range(0, n, c):
        c1 = min(c0 + c, n)
        blk = m[c0:c1, c0:c1].tocsr()
        rhs = b[c0:c1] - (m[c0:c1] @ x0 - blk @ x0[c0:c1])     # other chunks, old values
        tri = sp.tril(blk) if forward else sp.triu(blk)
        rhs = rhs - (blk - tri) @ x0[c0:c1]                      # own rows not yet swept
        ref[c0:c1] = spl.spsolve_triangular(tri.tocsr(), rhs, lower=forward)
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_pgs_no_on_one_chunk_is_gauss_seidel_and_on_diagonal_is_jacobi():
    m, a = _scalar_pressure_like(4, dims=(4, 2, 2))   # 16 cells + 2 wells: one chunk + 2 rows
    n = m.shape[0]
    b = np.random.default_rng(4).normal(size=n)
    x = oracle.pgs_no_sweep(m.indptr, m.indices, m.data, b, np.zeros(n), True)
    sub = m[:16, :16].tocsr()
    ref = spl.spsolve_triangular(sp.tril(sub).tocsr(), b[:16], lower=True)
    assert np.allclose(x[:16], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    dg = sp.diags(np.arange(1.0, 41.0)).tocsr()
    bd = np.ones(40)
    assert np.allclose(oracle.pgs_no_sweep(dg.indptr, dg.indices, dg.data, bd, np.zeros(40)),
                       bd / np.arange(1.0, 41.0))


@pytest.mark.parametrize("smoother", [1, 2])
def test_alternative_smoothers_solve(smoother):
    """MSP-GMRES with PJAC-NO or PGS-NO in the AMG still solves to tolerance; the coarse
    levels are kept in natural order as one class."""
    a = box_jacobian(9, 7, 6, 3, 11, layered=True, kz_ratio=0.1, n_wells=1)
    o = oracle.Oracle(a, coarse_max=40, smoother=smoother)
    for l in range(1, o.num_levels - 1):
        assert o.level(l)["ncolours"] == 1
    x, info = o.solve(random_rhs(a, 2))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-6
