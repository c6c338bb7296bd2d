"""The batched solve (msp_set_instances / msp_solve_batch) on the GPU against the oracle:
several instances of one block size stacked block-diagonally, set up once, each solved by
its own FGMRES in the same launches.  Per instance: the iteration count within one of the
oracle's FGMRES on the stack with the right-hand side restricted to that instance (the
preconditioner of a stack is block diagonal, so that is the instance's own solve), and the
true residual <= tol.  Also: a zero right-hand side, the FP32 preconditioner, repeated
solves bit-identical, new values with the adaptive rule, rejected couplings and offsets."""
import numpy as np
import pytest

import oracle
from synthetic import BSRMatrix, box_jacobian, perturb_values, random_rhs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_08594_gb300 as msp  # noqa: E402

DEV = torch.device("cuda:0")
CFG = dict(coarse_max=80, mu=10**6)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _instances(b=4):
    return [box_jacobian(9, 7, 5, b, 21, layered=True, kz_ratio=0.1, n_wells=1),
            box_jacobian(6, 6, 4, b, 22),
            box_jacobian(12, 5, 3, b, 23, layered=True, kz_ratio=0.1, n_wells=2),
            box_jacobian(4, 3, 3, b, 24),
            box_jacobian(10, 10, 2, b, 25, n_wells=1)]


def _stack(ms):
    nb, b, rp, ci, v, off = msp.stack_block_diagonal(ms)
    S = BSRMatrix(nb=nb, b=b, row_ptr=rp, col_idx=ci, values=v.reshape(-1, b, b))
    return S, off


def _rhs(ms, off, b, seed):
    return np.concatenate([random_rhs(m, seed + k) for k, m in enumerate(ms)])


@pytest.fixture(scope="module")
def batch():
    ms = _instances()
    S, off = _stack(ms)
    g = msp.BatchSolver(S.nb, S.b, _t(S.row_ptr), _t(S.col_idx), _t(S.values.reshape(-1)), off,
                        **CFG)
    o = oracle.Oracle(S, **CFG)
    yield ms, S, off, g, o
    g.close()
    o.close()


def test_each_instance_matches_the_oracle(batch):
    ms, S, off, g, o = batch
    b = S.b
    rhs = _rhs(ms, off, b, 40)
    x = torch.zeros(S.nb * b, dtype=torch.float64, device=DEV)
    infos = g.solve_batch(_t(rhs), x, 1e-6)
    x = x.cpu().numpy()
    A = S.to_scipy()
    for k in range(len(ms)):
        lo, hi = off[k] * b, off[k + 1] * b
        assert infos[k]["status"] == 0, (k, infos[k])
        gk = np.zeros_like(rhs)
        gk[lo:hi] = rhs[lo:hi]
        xo, oinfo = o.solve(gk, 1e-6)
        assert abs(infos[k]["iterations"] - oinfo["iterations"]) <= 1, (k, infos[k], oinfo)
        xk = np.zeros_like(x)
        xk[lo:hi] = x[lo:hi]
        r = gk - A @ xk
        assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(gk) * 1.001, k
        assert abs(infos[k]["rel_residual"] - np.linalg.norm(r) / np.linalg.norm(gk)) < 1e-9


def test_repeat_is_bit_identical_and_zero_rhs(batch):
    ms, S, off, g, o = batch
    b = S.b
    rhs = _rhs(ms, off, b, 50)
    rhs[off[1] * b:off[2] * b] = 0.0  # instance 1: zero right-hand side
    x1 = torch.zeros(S.nb * b, dtype=torch.float64, device=DEV)
    x2 = torch.zeros(S.nb * b, dtype=torch.float64, device=DEV)
    i1 = g.solve_batch(_t(rhs), x1, 1e-6)
    i2 = g.solve_batch(_t(rhs), x2, 1e-6)
    assert torch.equal(x1, x2)
    assert [i["iterations"] for i in i1] == [i["iterations"] for i in i2]
    assert i1[1]["status"] == 0 and i1[1]["iterations"] == 0
    assert torch.count_nonzero(x1[off[1] * b:off[2] * b]) == 0


def test_batch_agrees_with_the_whole_stack_solve(batch):
    ms, S, off, g, o = batch
    b = S.b
    rhs = _rhs(ms, off, b, 60)
    xb = torch.zeros(S.nb * b, dtype=torch.float64, device=DEV)
    infos = g.solve_batch(_t(rhs), xb, 1e-6)
    for k in (0, 2):
        lo, hi = off[k] * b, off[k + 1] * b
        gk = np.zeros_like(rhs)
        gk[lo:hi] = rhs[lo:hi]
        xs = torch.zeros(S.nb * b, dtype=torch.float64, device=DEV)
        info = g.solve(_t(gk), xs, 1e-6)
        assert abs(info["iterations"] - infos[k]["iterations"]) <= 1
        assert torch.count_nonzero(xs[:lo]) == 0 and torch.count_nonzero(xs[hi:]) == 0


def test_fp32_and_new_values():
    ms = _instances(b=3)
    S, off = _stack(ms)
    g = msp.BatchSolver(S.nb, S.b, _t(S.row_ptr), _t(S.col_idx), _t(S.values.reshape(-1)), off,
                        coarse_max=80, mu=20, precision=msp.MSP_PRECISION_FP32)
    rhs = _rhs(ms, off, S.b, 70)
    for step in range(3):
        if step:
            v = perturb_values(S, 80 + step)
            g.update_values(_t(v.reshape(-1)))
            S = BSRMatrix(nb=S.nb, b=S.b, row_ptr=S.row_ptr, col_idx=S.col_idx, values=v)
        x = torch.zeros(S.nb * S.b, dtype=torch.float64, device=DEV)
        infos = g.solve_batch(_t(rhs), x, 1e-6)
        xx = x.cpu().numpy()
        A = S.to_scipy()
        for k in range(len(ms)):
            lo, hi = off[k] * S.b, off[k + 1] * S.b
            gk = np.zeros_like(rhs)
            gk[lo:hi] = rhs[lo:hi]
            xk = np.zeros_like(xx)
            xk[lo:hi] = xx[lo:hi]
            assert infos[k]["status"] == 0
            assert np.linalg.norm(gk - A @ xk) <= 1e-6 * np.linalg.norm(gk) * 1.001
    g.close()


def test_instances_with_long_well_rows():
    """Wells perforating 20-24 layers: rows of more than 16 blocks, walked by a thread block
    each in the level-0 kernels, in several instances at once, with instances leaving the
    active set at different steps."""
    ms = [box_jacobian(5, 4, 24, 4, 41, layered=True, kz_ratio=0.1, n_wells=2),
          box_jacobian(6, 5, 20, 4, 42, n_wells=1),
          box_jacobian(7, 3, 22, 4, 43, layered=True, kz_ratio=0.1, n_wells=3)]
    S, off = _stack(ms)
    assert int((np.diff(S.row_ptr) > 16).sum()) == 6
    g = msp.BatchSolver(S.nb, S.b, _t(S.row_ptr), _t(S.col_idx), _t(S.values.reshape(-1)), off,
                        **CFG)
    o = oracle.Oracle(S, **CFG)
    rhs = _rhs(ms, off, S.b, 90)
    x = torch.zeros(S.nb * S.b, dtype=torch.float64, device=DEV)
    infos = g.solve_batch(_t(rhs), x, 1e-6)
    xx = x.cpu().numpy()
    A = S.to_scipy()
    for k in range(len(ms)):
        lo, hi = off[k] * S.b, off[k + 1] * S.b
        gk = np.zeros_like(rhs)
        gk[lo:hi] = rhs[lo:hi]
        _, oinfo = o.solve(gk, 1e-6)
        assert infos[k]["status"] == 0, (k, infos[k])
        assert abs(infos[k]["iterations"] - oinfo["iterations"]) <= 1, (k, infos[k], oinfo)
        xk = np.zeros_like(xx)
        xk[lo:hi] = xx[lo:hi]
        assert np.linalg.norm(gk - A @ xk) <= 1e-6 * np.linalg.norm(gk) * 1.001, k
    g.close()
    o.close()


def test_rejected_instances():
    ms = _instances()[:2]
    S, off = _stack(ms)
    s = msp.Solver(S.nb, S.b, _t(S.row_ptr), _t(S.col_idx), _t(S.values.reshape(-1)), **CFG)
    with pytest.raises(msp.MspError) as e:
        msp.msp_set_instances(s.h, [0, 10, 5, S.nb])  # not increasing
    assert e.value.status == msp._native.MSP_ERR_ARG
    with pytest.raises(msp.MspError) as e:
        msp.msp_set_instances(s.h, [0, off[1] + 3, S.nb])  # cuts through instance 0's couplings
    assert e.value.status == msp._native.MSP_ERR_PATTERN
    with pytest.raises(msp.MspError):
        msp.msp_solve_batch(s.h, 2, _t(np.ones(S.nb * S.b)),
                            torch.zeros(S.nb * S.b, dtype=torch.float64, device=DEV))
    s.close()
