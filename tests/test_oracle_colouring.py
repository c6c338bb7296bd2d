"""Pins for the oracle's colouring (Algorithm 4.1 VerticesSplitting, Algorithm 4.2
VerticesGrouping, Section 4.2) against hand traces, the colouring principles (i)-(iii)
of Section 4.1, the red-black special case, and a second, literal implementation."""
import json
import os

import numpy as np
import pytest

from conftest import csr_from_edges
from synthetic import box_jacobian, grid_spe10, poisson3d_bsr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "alg41_hand_traces.json")


def _adj_sets(n, rp, ci):
    s = [set() for _ in range(n)]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = int(ci[p])
            if j != i:
                s[i].add(j)
                s[j].add(i)
    return s


def literal_grouping(n, rp, ci):
    """Second implementation of Algorithms 4.1/4.2 written from the pseudo-code with
    Python sets and a full scan for every pick (quadratic; tiny graphs only)."""
    S = _adj_sets(n, rp, ci)
    deg = [len(S[i]) for i in range(n)]
    colour = [0] * n
    V = set(range(n))
    g = 0
    while V:
        g += 1
        W, Wbar, What = set(), set(), set()
        while V:
            pool = What if What else V
            vi = min(pool, key=lambda v: (-deg[v], v))
            if not (S[vi] & W):
                W.add(vi)
                V.discard(vi)
                What.discard(vi)
                Wbar |= (S[vi] & V)
                V -= S[vi]
                second = set()
                for k in S[vi]:
                    second |= S[k]
                second -= S[vi] | {vi}
                What |= (second & V)
            else:
                Wbar.add(vi)
                V.discard(vi)
                What.discard(vi)
        for v in W:
            colour[v] = g
        V = Wbar
    return np.asarray(colour), g


def check_valid(n, rp, ci, colour, g):
    # (i)+(ii): every vertex has exactly one colour in 1..g, every colour is used
    assert colour.min() >= 1 and colour.max() == g
    assert set(np.unique(colour)) == set(range(1, g + 1))
    # (iii): no edge inside a colour class
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            if j != i:
                assert colour[i] != colour[j], (i, j)


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_traces(oracle_lib, case):
    rp, ci = csr_from_edges(case["n"], case["edges"])
    colour, g = oracle_lib.vertices_grouping(case["n"], rp, ci)
    assert g == case["g"]
    assert colour.tolist() == case["colour"]


@pytest.mark.parametrize("dims", [(5, 4, 3), (16, 16, 8), (7, 1, 1), (6, 9, 1)])
def test_red_black_on_seven_point_grid(oracle_lib, dims):
    """Without wells the 7-point grid graph is bipartite and every vertex the frontier
    offers lies at distance 2 from a chosen one, so pass 1 takes exactly the parity
    class of the first max-degree vertex: g = 2 (the red-black case, Section 4.1)."""
    a = poisson3d_bsr(*dims)
    colour, g = oracle_lib.vertices_grouping(a.nb, a.row_ptr, a.col_idx)
    nx, ny, nz = dims
    i = np.arange(a.nb)
    parity = (i % nx + (i // nx) % ny + i // (nx * ny)) % 2
    deg = np.diff(a.row_ptr) - 1
    first = int(np.argmax(deg))  # max degree, smallest index
    assert g == 2
    assert np.array_equal(colour == 1, parity == parity[first])


@pytest.mark.parametrize("seed", range(12))
def test_matches_literal_implementation(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    m = int(rng.integers(n, 4 * n))
    edges = {tuple(sorted(e)) for e in rng.integers(0, n, size=(m, 2)) if e[0] != e[1]}
    rp, ci = csr_from_edges(n, sorted(edges))
    colour, g = oracle_lib.vertices_grouping(n, rp, ci)
    ref, gref = literal_grouping(n, rp, ci)
    assert g == gref
    assert np.array_equal(colour, ref)
    check_valid(n, rp, ci, colour, g)


def test_literal_implementation_on_grid_with_wells(oracle_lib):
    a = grid_spe10(nx=6, ny=5, nz=4)
    colour, g = oracle_lib.vertices_grouping(a.nb, a.row_ptr, a.col_idx)
    ref, gref = literal_grouping(a.nb, a.row_ptr, a.col_idx)
    assert g == gref and np.array_equal(colour, ref)
    check_valid(a.nb, a.row_ptr, a.col_idx, colour, g)
    assert g > 2  # wells break the bipartite structure


def test_nonsymmetric_pattern_is_symmetrised(oracle_lib):
    # edge stored in one direction only still separates the two vertices
    n = 3
    rp = np.array([0, 2, 3, 4], np.int32)
    ci = np.array([0, 2, 1, 2], np.int32)  # row 0 holds (0,2); row 2 holds only (2,2)
    colour, g = oracle_lib.vertices_grouping(n, rp, ci)
    assert colour[0] != colour[2]


def test_valid_on_larger_grid_with_wells(oracle_lib):
    a = box_jacobian(30, 20, 10, 2, 5, layered=True, kz_ratio=0.1, n_wells=4)
    colour, g = oracle_lib.vertices_grouping(a.nb, a.row_ptr, a.col_idx)
    check_valid(a.nb, a.row_ptr, a.col_idx, colour, g)


# ---- greedy colouring in Jones-Plassmann priority order (an alternative to Alg 4.1/4.2)

def _splitmix64(x):
    """SplitMix64 output function (Vigna), written from its published definition."""
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


JP_SEED = 0x4A6F6E6573504C


def brute_force_jp(n, rp, ci):
    """First-fit greedy in priority order (degree descending, then the high word of
    SplitMix64(v ^ seed), then index) with Python sets: the colouring the parallel
    Jones-Plassmann rounds must reproduce."""
    S = _adj_sets(n, rp, ci)
    order = sorted(range(n), key=lambda v: (-len(S[v]), _splitmix64(v ^ JP_SEED) >> 32, v))
    colour = [0] * n
    for v in order:
        used = {colour[u] for u in S[v]}
        c = 1
        while c in used:
            c += 1
        colour[v] = c
    return colour


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return csr_from_edges(n, edges)


@pytest.mark.parametrize("seed", range(6))
def test_jp_matches_brute_force(oracle_lib, seed):
    n = 40 + 7 * seed
    rp, ci = _random_graph(n, 0.12, seed)
    c, g = oracle_lib.jp_colouring(n, rp, ci)
    ref = brute_force_jp(n, rp, ci)
    assert list(c) == ref and g == max(ref)


def test_jp_colouring_properties(oracle_lib):
    a = box_jacobian(9, 8, 6, 3, 2, n_wells=2)
    n = a.nb
    c, g = oracle_lib.jp_colouring(n, a.row_ptr, a.col_idx)
    S = _adj_sets(n, a.row_ptr, a.col_idx)
    assert all(c[v] != c[u] for v in range(n) for u in S[v])          # proper
    assert g <= max(len(s) for s in S) + 1
    for v in range(n):                                                # first fit (Grundy)
        around = {int(c[u]) for u in S[v]}
        assert all(k in around for k in range(1, int(c[v])))


def test_jp_complete_graph_and_star(oracle_lib):
    n = 9
    rp, ci = csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    c, g = oracle_lib.jp_colouring(n, rp, ci)
    assert g == n and sorted(c) == list(range(1, n + 1))
    rp, ci = csr_from_edges(n, [(0, j) for j in range(1, n)])           # star: centre first
    c, g = oracle_lib.jp_colouring(n, rp, ci)
    assert g == 2 and c[0] == 1 and all(x == 2 for x in c[1:])
