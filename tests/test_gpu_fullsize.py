"""Parity at the full SPE10-shaped size (60x220x85 cells + 4 wells, 4x4 blocks, FP64), in
the configuration the benchmark times: integer setup outputs and level matrices
bit-exact against the oracle, one MSP application (Algorithm 3.1) within 1e-10, SpMV
elementwise, and the solve's true residual (recomputed with SciPy) <= 1e-6.  The
oracle's full solve (about 140 iterations) is too slow for a test; the iteration count
is compared at smaller sizes in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from synthetic import grid_spe10, random_rhs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_08594_gb300 as msp  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def full():
    a = grid_spe10()
    rp = torch.from_numpy(a.row_ptr).to(DEV)
    ci = torch.from_numpy(a.col_idx).to(DEV)
    v = torch.from_numpy(a.values.reshape(-1)).to(DEV)
    g = msp.Solver(a.nb, a.b, rp, ci, v)
    o = oracle.Oracle(a)
    yield a, g, o
    g.close()
    o.close()


def test_full_size_setup_bit_exact(full):
    a, g, o = full
    cg, ng = g.colour0()
    co, no = o.colour0()
    assert ng == no and np.array_equal(cg, co)
    assert g.num_levels == o.num_levels
    for l in range(o.num_levels):
        lg, lo = g.level(l), o.level(l)
        for key in ("n", "nnz", "ncolours"):
            assert lg[key] == lo[key], (l, key)
        for key in ("perm", "cptr", "agg", "row_ptr", "col_idx", "values"):
            assert np.array_equal(lg[key], lo[key]), (l, key)


def test_full_size_msp_application(full):
    a, g, o = full
    x = random_rhs(a, 21)
    w = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    g.apply_precond(torch.from_numpy(x).to(DEV), w)
    ref = o.apply_precond(x)
    err = np.abs(w.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, err


def test_full_size_spmv_sampled_rows(full):
    a, g, o = full
    x = np.random.default_rng(3).normal(size=a.n)
    y = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    g.spmv(torch.from_numpy(x).to(DEV), y)
    y = y.cpu().numpy()
    rows = np.random.default_rng(4).choice(a.nb, size=2000, replace=False)
    rows = np.concatenate([rows, np.arange(a.n_cells, a.nb)])  # every well row
    b = a.b
    for i in rows:
        ref = np.zeros(b)
        for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
            j = a.col_idx[p]
            ref += a.values[p] @ x[j * b:(j + 1) * b]
        assert np.allclose(y[i * b:(i + 1) * b], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_full_size_solve_residual(full):
    a, g, o = full
    rhs = random_rhs(a, 22)
    x = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    info = g.solve(torch.from_numpy(rhs).to(DEV), x, 1e-6)
    assert info["status"] == 0
    r = rhs - a.to_scipy() @ x.cpu().numpy()
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6 * 1.001
