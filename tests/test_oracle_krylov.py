"""Pins for the oracle's MSP (Algorithm 3.1 against the product form of Eq. MSP), the
FGMRES(30) solve (Section 5 settings, tolerance 1e-6), and the adaptive setup of
Section 3.2."""
import numpy as np
import pytest

import oracle
from synthetic import (box_jacobian, diagonal_bsr, grid_small, grid_spe10, perturb_values,
                       poisson3d_bsr, random_rhs)


def _dense(a):
    return a.to_dense()


@pytest.mark.parametrize("case", [
    dict(dims=(4, 3, 2), b=2, wells=0), dict(dims=(4, 4, 3), b=3, wells=1),
    dict(dims=(5, 4, 4), b=4, wells=2), dict(dims=(6, 6, 4), b=4, wells=0),
])
def test_msp_equals_product_form(case):
    """I - B A = (I - R A)(I - Pi_P B_P Pi_P^T A)(I - Pi_N B_N Pi_N^T A): Algorithm 3.1 is
    checked against the three single-stage operators composed as in Eq. MSP."""
    a = box_jacobian(*case["dims"], case["b"], 31, layered=True, kz_ratio=0.1,
                     n_wells=case["wells"])
    A = _dense(a)
    kw = dict(coarse_max=8)
    full = oracle.Oracle(a, **kw)
    stN = oracle.Oracle(a, precond=oracle.PREC_N_ONLY, **kw)
    stP = oracle.Oracle(a, precond=oracle.PREC_P_ONLY, **kw)
    stR = oracle.Oracle(a, precond=oracle.PREC_R_ONLY, **kw)
    v = np.random.default_rng(0).normal(size=a.n)
    lhs = v - full.apply_precond(A @ v)
    e = v - stN.apply_precond(A @ v)
    e = e - stP.apply_precond(A @ e)
    e = e - stR.apply_precond(A @ e)
    assert np.allclose(lhs, e, rtol=1e-10, atol=1e-10 * np.abs(e).max())


@pytest.mark.parametrize("b,wells", [(3, 1), (4, 2)])
def test_stage_p_with_exact_coarse_solve_is_the_decoupled_pressure_inverse(b, wells):
    """Stage P alone with one AMG level (coarse_max >= n, a direct solve) is
    Pi_P A_P^-1 Pi_P^T: restriction r_P[i] = omega_i . r_i with omega_i^T = e_0^T D_i^-1,
    A_P[i,j] = omega_i . A_ij e_0, and the correction added to unknown 0 of every block."""
    a = box_jacobian(4, 3, 3, b, 61, layered=True, kz_ratio=0.1, n_wells=wells)
    o = oracle.Oracle(a, precond=oracle.PREC_P_ONLY, coarse_max=10**6)
    nb = a.nb
    rows = np.repeat(np.arange(nb), np.diff(a.row_ptr))
    diag = {i: a.values[p] for p, (i, j) in enumerate(zip(rows, a.col_idx)) if i == j}
    omega = np.array([np.linalg.inv(diag[i])[0] for i in range(nb)])
    AP = np.zeros((nb, nb))
    for p, (i, j) in enumerate(zip(rows, a.col_idx)):
        AP[i, j] = omega[i] @ a.values[p][:, 0]
    r = np.random.default_rng(7).normal(size=a.n)
    e = np.linalg.solve(AP, np.einsum("ik,ik->i", omega, r.reshape(nb, b)))
    want = np.zeros((nb, b))
    want[:, 0] = e
    got = o.apply_precond(r)
    assert np.allclose(got, want.reshape(-1), rtol=1e-10, atol=1e-10 * np.abs(e).max())
    o.close()


@pytest.mark.parametrize("case", [
    dict(dims=(2, 2, 2), b=2, wells=0), dict(dims=(3, 3, 2), b=3, wells=1),
    dict(dims=(4, 4, 3), b=4, wells=1), dict(dims=(6, 6, 4), b=4, wells=2),
    dict(dims=(6, 5, 4), b=3, wells=0),
])
def test_solution_matches_dense_lu(case):
    a = box_jacobian(*case["dims"], case["b"], 41, layered=True, kz_ratio=0.1,
                     n_wells=case["wells"])
    rhs = random_rhs(a, 5)
    A = _dense(a)
    xs = np.linalg.solve(A, rhs)
    o = oracle.Oracle(a, coarse_max=10)
    x, info = o.solve(rhs, tol=1e-6)
    assert info["status"] == 0
    assert np.linalg.norm(rhs - A @ x) / np.linalg.norm(rhs) <= 1e-6 * (1 + 1e-9)
    assert info["rel_residual"] == pytest.approx(np.linalg.norm(rhs - A @ x) /
                                                 np.linalg.norm(rhs), rel=1e-6)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= cond * 1e-6


@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_krylov_finite_termination(k):
    """GMRES on a diagonal matrix with k distinct eigenvalues terminates in k steps."""
    rng = np.random.default_rng(k)
    eig = np.linspace(1.0, 3.0, k)
    d = eig[rng.integers(0, k, size=200)]
    d[:k] = eig
    a = diagonal_bsr(d)
    o = oracle.Oracle(a, precond=oracle.PREC_NONE, coarse_max=1000)
    x, info = o.solve(rng.normal(size=200), tol=1e-10)
    assert info["iterations"] == k


def test_zero_rhs_gives_zero_solution():
    a = grid_small()
    o = oracle.Oracle(a, coarse_max=200)
    x, info = o.solve(np.zeros(a.n))
    assert info["iterations"] == 0 and np.all(x == 0) and info["status"] == 0


def test_restart_and_max_it():
    a = grid_spe10(nx=10, ny=12, nz=5)
    rhs = random_rhs(a, 9)
    o = oracle.Oracle(a, precond=oracle.PREC_NONE, restart=5, max_it=23, coarse_max=200)
    x, info = o.solve(rhs, tol=1e-12)
    assert info["status"] == oracle.ORC_NOT_CONVERGED and info["iterations"] == 23


def test_nonfinite_rhs_rejected():
    a = grid_small()
    o = oracle.Oracle(a, coarse_max=200)
    rhs = random_rhs(a, 1)
    rhs[7] = np.nan
    x, info = o.solve(rhs)
    assert info["status"] == -4


def test_small_grid_converges():
    a = grid_small()
    o = oracle.Oracle(a)
    x, info = o.solve(random_rhs(a, 1))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-6


def _sequence(mu, nsolves=6, seed=51):
    a = grid_spe10(nx=10, ny=12, nz=5)
    o = oracle.Oracle(a, mu=mu, coarse_max=100)
    its, setups = [], []
    for k in range(nsolves):
        if k > 0:
            o.update_values(perturb_values(a, seed + k))
        x, info = o.solve(random_rhs(a, seed + 100 + k))
        its.append(info["iterations"])
        setups.append(info["setup_performed"])
    return its, setups, o.setup_calls


def test_adaptive_setup_trace():
    """Section 3.2: the first solve uses a freshly generated B; solve iota regenerates iff
    It^(iota-1) > mu.  mu = 0 is the plain MSP (a setup for every solve)."""
    its, setups, calls = _sequence(0)
    assert setups == [1] * 6 and calls == 6
    its, setups, calls = _sequence(10 ** 6)
    assert setups == [1, 0, 0, 0, 0, 0] and calls == 1
    mu = 25
    its, setups, calls = _sequence(mu)
    expect = [1] + [1 if its[k - 1] > mu else 0 for k in range(1, 6)]
    assert setups == expect and calls == sum(expect)


def test_adaptive_setup_boundary():
    """It^(iota-1) equal to mu keeps B; one more than mu regenerates it (the rule is a
    strict inequality).  The first solve's count does not depend on mu."""
    its, _, _ = _sequence(10 ** 6, nsolves=2)
    first = its[0]
    _, setups, calls = _sequence(first, nsolves=2)
    assert setups == [1, 0] and calls == 1
    _, setups, calls = _sequence(first - 1, nsolves=2)
    assert setups == [1, 1] and calls == 2


def test_reuse_keeps_stage_operators_but_uses_current_matrix():
    """On reuse (Section 3.2) the residual steps of Algorithm 3.1 use the
    current A while B_N, B_P and R stay those of the last setup."""
    a = grid_spe10(nx=6, ny=5, nz=4)
    o = oracle.Oracle(a, mu=10 ** 6, coarse_max=20)
    g = random_rhs(a, 3)
    w_old = o.apply_precond(g)
    a2 = a.copy()
    a2.values = perturb_values(a, 7)
    o.update_values(a2.values)
    w_new = o.apply_precond(g)
    fresh = oracle.Oracle(a2, coarse_max=20)
    w_fresh = fresh.apply_precond(g)
    assert not np.allclose(w_new, w_old)
    assert not np.allclose(w_new, w_fresh)
    # the stage-R-only operator is unchanged by the value update (frozen factors)
    r_only = oracle.Oracle(a, precond=oracle.PREC_R_ONLY, coarse_max=20)
    w1 = r_only.apply_precond(g)
    r_only.update_values(a2.values)
    assert np.array_equal(r_only.apply_precond(g), w1)
