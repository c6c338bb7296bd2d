"""Host-side checks of the batched form: the block-diagonal stacking, and the property the
batched solve rests on, pinned with the oracle — on a block-diagonal matrix the
multi-stage preconditioner (Algorithm 3.1 with the colouring, aggregation, stage operators
and coarsest solve set up on the whole stack) is block diagonal: a vector supported on one
instance is mapped to a vector supported on that instance, exactly, and the FGMRES of the
stack with a right-hand side supported on one instance never leaves it."""
import numpy as np

import oracle
import paper_2208_08594_gb300 as msp
from synthetic import BSRMatrix, box_jacobian, random_rhs


def _instances():
    return [box_jacobian(5, 4, 3, 3, 11), box_jacobian(4, 4, 4, 3, 12, n_wells=1),
            box_jacobian(6, 3, 2, 3, 13, layered=True, kz_ratio=0.1)]


def test_stack_block_diagonal_matches_dense():
    import scipy.sparse as sp
    ms = _instances()
    nb, b, rp, ci, v, off = msp.stack_block_diagonal(ms)
    assert nb == sum(m.nb for m in ms) and b == 3
    assert list(off) == [0, ms[0].nb, ms[0].nb + ms[1].nb, nb]
    S = BSRMatrix(nb=nb, b=b, row_ptr=rp, col_idx=ci, values=v.reshape(-1, b, b))
    D = sp.block_diag([m.to_scipy() for m in ms]).toarray()
    assert np.array_equal(S.to_scipy().toarray(), D)


def test_preconditioner_of_a_stack_is_block_diagonal():
    ms = _instances()
    nb, b, rp, ci, v, off = msp.stack_block_diagonal(ms)
    S = BSRMatrix(nb=nb, b=b, row_ptr=rp, col_idx=ci, values=v.reshape(-1, b, b))
    o = oracle.Oracle(S, coarse_max=20, mu=10**6)
    rng = np.random.default_rng(5)
    for k in range(len(ms)):
        lo, hi = off[k] * b, off[k + 1] * b
        g = np.zeros(nb * b)
        g[lo:hi] = rng.normal(size=hi - lo)
        w = o.apply_precond(g)
        assert np.all(w[:lo] == 0.0) and np.all(w[hi:] == 0.0)
        assert np.any(w[lo:hi] != 0.0)
        x, info = o.solve(g, 1e-8)
        assert info["status"] == 0
        assert np.all(x[:lo] == 0.0) and np.all(x[hi:] == 0.0)
        r = g - S.to_scipy() @ x
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(g) * 1.001
    o.close()


def test_stack_rejects_mixed_block_sizes():
    import pytest
    with pytest.raises(ValueError):
        msp.stack_block_diagonal([box_jacobian(3, 3, 2, 3, 1), box_jacobian(3, 3, 2, 4, 2)])


def test_colour_classes_of_a_stack_are_instance_major():
    """The batched Krylov kernels cut the colour-ordered vector into (colour, instance)
    segments: within every level-0 colour class (rows in original order, Algorithm 4.3
    step 3) the rows of one instance must be contiguous and the instances in order.  The
    colouring here is the oracle's, which the library's equals bit for bit."""
    ms = _instances() + [box_jacobian(3, 3, 3, 3, 14, n_wells=1)]
    nb, b, rp, ci, v, off = msp.stack_block_diagonal(ms)
    S = BSRMatrix(nb=nb, b=b, row_ptr=rp, col_idx=ci, values=v.reshape(-1, b, b))
    o = oracle.Oracle(S, coarse_max=20, mu=10**6)
    colour, g = o.colour0()
    perm = np.lexsort((np.arange(nb), colour))  # colour order, original order inside
    inst = np.searchsorted(off, perm, side="right") - 1
    cls = colour[perm]
    segments = 0
    for c in np.unique(cls):
        ids = inst[cls == c]
        assert np.all(np.diff(ids) >= 0), c
        segments += len(np.unique(ids))
    assert segments <= g * len(ms)
    # every instance appears in at least one class, and a class never mixes rows of two
    # instances inside one segment
    assert set(np.unique(inst)) == set(range(len(ms)))
    o.close()
