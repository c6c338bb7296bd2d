"""Pins for the oracle's pressure stage: pairwise aggregation (the oracle's reading of the
NPAIR citation in Section 5), the Galerkin coarse operators, and UA-AMG convergence on the
3-D Poisson problem; plus the pressure matrix of the decoupled restriction."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from synthetic import box_jacobian, grid_small, grid_spe10, poisson3d_bsr, random_rhs


def _level_csr(L):
    n = L["n"]
    return sp.csr_matrix((L["values"], L["col_idx"], L["row_ptr"]), shape=(n, n))


def _brute_pairwise(A, beta, seed):
    """Tiny-input restatement of one matching pass with dense arrays."""
    n = A.shape[0]
    S = ((A != 0) | (A.T != 0)) & ~np.eye(n, dtype=bool)
    s = -(A + A.T) / 2.0
    cand = []
    for i in range(n):
        js = np.nonzero(S[i])[0]
        if len(js) and s[i, js].max() > 0:
            cand.append([j for j in js if s[i, j] >= beta * s[i, js].max()])
        else:
            cand.append([])
    order = sorted(range(n), key=lambda i: (oracle.splitmix64(i ^ seed), i))
    partner = [-1] * n
    marked = [False] * n
    for i in order:
        if marked[i]:
            continue
        free = [j for j in cand[i] if not marked[j]]
        marked[i] = True
        if free:
            j = max(free, key=lambda j: (s[i, j], -j))
            marked[j] = True
            partner[i], partner[j] = j, i
    reps = sorted({min(i, partner[i]) if partner[i] >= 0 else i for i in range(n)})
    rank = {r: k for k, r in enumerate(reps)}
    return np.array([rank[min(i, partner[i]) if partner[i] >= 0 else i] for i in range(n)])


def test_splitmix64_reference_values():
    # SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference generator) seeded with 0
    # outputs 0xE220A8397B1DCDAF then 0x6E789E6AA1B965F4; the oracle's function is that
    # output applied to the state x (x + golden gamma, then the mix).
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def _golden_pairwise():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "pairwise_hand_traces.json")
    with open(path) as f:
        return json.load(f)


def test_splitmix64_published_outputs():
    ref = _golden_pairwise()["splitmix64_reference"]
    for x, y in zip(ref["inputs"], ref["outputs"]):
        assert oracle.splitmix64(int(x, 16)) == int(y, 16)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_pairwise_hand_traces(k):
    """One matching pass on a 7-node graph traced by hand (tests/golden): exact-threshold
    candidates, a negative strength, a tie, an asymmetric pair whose row-only strength
    would choose differently, taken candidates and singletons."""
    d = _golden_pairwise()
    gr, case = d["graph"], d["cases"][k]
    n = gr["n"]
    ent = {(i, i): gr["diagonal"] for i in range(n)}
    for i, j, v in gr["entries"]:
        ent[(i, j)] = v
    keys = sorted(ent)
    rp = np.zeros(n + 1, np.int32)
    for i, _ in keys:
        rp[i + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    ci = np.array([j for _, j in keys], np.int32)
    v = np.array([ent[key] for key in keys])
    order = sorted(range(n), key=lambda i: (oracle.splitmix64(i ^ case["seed"]), i))
    assert order == case["visit_order"]  # the premise of the trace
    agg, nc = oracle.pairwise(rp, ci, v, 0.25, case["seed"])
    assert nc == case["nagg"]
    assert agg.tolist() == case["agg"]
    assert [sorted(np.nonzero(agg == c)[0].tolist()) for c in range(nc)] == case["aggregates"]


@pytest.mark.parametrize("seed", range(6))
def test_pairwise_matches_brute_force(seed):
    a = box_jacobian(5, 4, 3, 1, 100 + seed, layered=True, n_wells=1)
    A = a.to_dense()
    rp, ci = a.row_ptr, a.col_idx
    agg, nc = oracle.pairwise(rp, ci, a.values.reshape(-1), 0.25, seed)
    ref = _brute_pairwise(A, 0.25, seed)
    assert nc == ref.max() + 1
    assert np.array_equal(agg, ref)


def _check_hierarchy(o):
    for l in range(o.num_levels - 1):
        F, Cc = o.level(l), o.level(l + 1)
        agg = F["agg"]
        nc = Cc["n"]
        # partition of the fine level onto 0..nc-1, aggregates of at most 2^npass = 4
        assert agg.min() == 0 and agg.max() == nc - 1
        sizes = np.bincount(agg, minlength=nc)
        assert sizes.min() >= 1 and sizes.max() <= 4
        # every aggregate is connected in the fine adjacency graph
        Af = _level_csr(F)
        Sg = ((abs(Af) + abs(Af.T)) != 0).tocsr()
        for I in np.nonzero(sizes > 1)[0][:400]:
            mem = set(np.nonzero(agg == I)[0].tolist())
            start = next(iter(mem))
            seen, stack = {start}, [start]
            while stack:
                u = stack.pop()
                for v in Sg.indices[Sg.indptr[u]:Sg.indptr[u + 1]]:
                    if v in mem and v not in seen:
                        seen.add(v)
                        stack.append(v)
            assert seen == mem
        # Galerkin: A_c = P^T A P, brute force with a dense P
        P = sp.csr_matrix((np.ones(F["n"]), (np.arange(F["n"]), agg)), shape=(F["n"], nc))
        Ac = (P.T @ Af @ P).toarray()
        got = _level_csr(Cc).toarray()
        assert np.allclose(got, Ac, rtol=1e-13, atol=1e-13 * np.abs(Ac).max())
        # coloured levels: colour classes are independent sets, in contiguous order
        if Cc["ncolours"]:
            cp = Cc["cptr"]
            col = np.repeat(np.arange(len(cp) - 1), np.diff(cp))
            Cm = _level_csr(Cc).tocoo()
            off = Cm.row != Cm.col
            assert not np.any(col[Cm.row[off]] == col[Cm.col[off]])


def test_hierarchy_on_poisson():
    a = poisson3d_bsr(16, 16, 16)
    o = oracle.Oracle(a, coarse_max=100)
    assert o.num_levels >= 3
    _check_hierarchy(o)


def test_hierarchy_on_compositional_grid():
    a = grid_spe10(nx=12, ny=15, nz=6)
    o = oracle.Oracle(a, coarse_max=60)
    assert o.num_levels >= 3
    _check_hierarchy(o)


def test_pressure_matrix_is_decoupled_restriction():
    """A_P[i,j] = omega_i^T A_ij e_0 with omega_i^T = e_0^T D_i^-1 (quasi-IMPES weights, the
    reading taken of the unspecified Pi_P^T in Eq. MSP); without decoupling it is
    A_ij[0,0]."""
    a = box_jacobian(4, 3, 3, 3, 21, n_wells=1)
    for dec in (1, 0):
        o = oracle.Oracle(a, decoupling=dec)
        colour, g = o.colour0()
        perm = np.lexsort((np.arange(a.nb), colour))
        iperm = np.empty_like(perm)
        iperm[perm] = np.arange(a.nb)
        L0 = _level_csr(o.level(0)).toarray()
        ref = np.zeros((a.nb, a.nb))
        for i in range(a.nb):
            d = [p for p in range(a.row_ptr[i], a.row_ptr[i + 1]) if a.col_idx[p] == i][0]
            w = np.linalg.inv(a.values[d])[0] if dec else np.eye(a.b)[0]
            for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
                ref[iperm[i], iperm[a.col_idx[p]]] = w @ a.values[p][:, 0]
        assert np.allclose(L0, ref, rtol=1e-12, atol=1e-14)


def _two_grid_rate(n_side, levels):
    a = poisson3d_bsr(n_side, n_side, n_side)
    o = oracle.Oracle(a, precond=oracle.PREC_P_ONLY, max_levels=levels, coarse_max=1,
                      coarse_hard_max=100000)
    A = a.to_scipy().tocsr()
    rng = np.random.default_rng(0)
    x_true = rng.normal(size=a.n)
    b = A @ x_true
    x = np.zeros(a.n)
    errs = []
    for _ in range(8):
        x = x + o.apply_precond(b - A @ x)
        errs.append(np.linalg.norm(x - x_true))
    return (errs[-1] / errs[2]) ** (1 / 5)


def test_two_grid_contracts_on_poisson():
    rate = _two_grid_rate(10, 2)
    assert rate < 0.9


def test_vcycle_contracts_on_poisson():
    assert _two_grid_rate(12, 5) < 0.95


def test_vcycle_fgmres_iterations_grow_slowly():
    its = []
    for n in (16, 32):
        a = poisson3d_bsr(n, n, n)
        o = oracle.Oracle(a, precond=oracle.PREC_P_ONLY, coarse_max=50)
        rhs = np.random.default_rng(3).normal(size=a.n)
        x, info = o.solve(rhs, tol=1e-6)
        assert info["status"] == 0
        A = a.to_scipy()
        assert np.linalg.norm(rhs - A @ x) / np.linalg.norm(rhs) <= 1e-6 * 1.0001
        its.append(info["iterations"])
    assert its[1] <= 2 * its[0] and its[1] < 60, its


def test_exact_coarse_solve_gives_one_iteration():
    """Section 3.2: one iteration means B is the exact inverse.  Block size 1 with the
    coarsest level holding the whole problem makes stage P an exact solve."""
    a = poisson3d_bsr(8, 7, 6)
    o = oracle.Oracle(a, coarse_max=10000)
    assert o.num_levels == 1
    x, info = o.solve(np.random.default_rng(4).normal(size=a.n), tol=1e-8)
    assert info["iterations"] == 1 and info["status"] == 0


def test_levels_shrink_and_stop_at_coarse_max():
    a = grid_small()
    o = oracle.Oracle(a, coarse_max=150)
    ns = [o.level(l)["n"] for l in range(o.num_levels)]
    assert ns[0] == a.nb and ns[-1] <= 150 and all(ns[k + 1] < ns[k] for k in range(len(ns) - 1))
    assert all(ns[k] > 150 for k in range(len(ns) - 1))
