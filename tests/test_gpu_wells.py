"""Parity of the CUDA elimination of the well unknowns (Schur complement of A_WW in the
Jacobian with implicit wells, Eq. Jacobian-system) with the oracle, through the C ABI:

* the reduced pattern bit-exact, its values, A_WW^-1 products, the reduced right-hand
  side and the recovered well unknowns bit-exact (both sides form every b x b product in
  the same order without fused multiply-add), also after new values;
* FGMRES + MSP on the reduced system: iteration count within +-1 of the oracle's, and
  the true residual of the FULL system <= tol * ||g_S|| (the well rows are satisfied up
  to rounding by the recovery);
* the rejected layouts (a cell on two wells, wells coupled to each other, no cell rows);
* the full SPE10-shaped size (60x220x85 + 4 wells): pattern, values and vectors
  bit-exact, and the solve's full-system residual.
"""
import numpy as np
import pytest

import oracle
from synthetic import BSRMatrix, box_jacobian, grid_spe10, random_rhs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_08594_gb300 as msp  # noqa: E402

DEV = torch.device("cuda:0")


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def _rhs_with_wells(a, seed):
    g = random_rhs(a, seed)
    g[a.n_cells * a.b:] = np.random.default_rng(seed + 1).normal(size=a.n_wells * a.b)
    return g


def _tiny(pairs, nb):
    """b = 1 matrix with the given symmetric off-diagonal pairs, diagonally dominant."""
    rows = [[i] for i in range(nb)]
    for i, j in pairs:
        rows[i].append(j)
        rows[j].append(i)
    rp, ci, v = [0], [], []
    for i in range(nb):
        for j in sorted(rows[i]):
            ci.append(j)
            v.append(10.0 if j == i else -1.0 - 0.1 * (i + j))
        rp.append(len(ci))
    return BSRMatrix(nb=nb, b=1, row_ptr=np.array(rp, np.int32), col_idx=np.array(ci, np.int32),
                     values=np.array(v).reshape(-1, 1, 1), n_cells=nb - 2, n_wells=2)


CASES = {
    "b3_two_wells": lambda: box_jacobian(5, 4, 6, 3, 7, n_wells=2),
    "b4_one_well": lambda: box_jacobian(4, 4, 9, 4, 7, n_wells=1),
    "b2_three_wells": lambda: box_jacobian(6, 3, 4, 2, 7, n_wells=3),
    "spe10_like_b4": lambda: grid_spe10(nx=23, ny=17, nz=9),
    "lone_well_b1": lambda: _tiny([(0, 1), (1, 2), (1, 3)], 5),  # well 4 perforates nothing
}


def _check_bit_exact(a, W, O, seed):
    rp, ci, v = W.reduced()
    orp, oci, ov = O.reduced()
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(ci.cpu().numpy(), oci)
    assert np.array_equal(_bits(v.cpu().numpy()), _bits(ov))
    g = _rhs_with_wells(a, seed)
    gs = torch.empty(W.nr * a.b, dtype=torch.float64, device=DEV)
    W.reduce_rhs(_t(g), gs)
    ogs = O.reduce_rhs(g)
    assert np.array_equal(_bits(gs.cpu().numpy()), _bits(ogs))
    xs = np.random.default_rng(seed + 2).normal(size=W.nr * a.b)
    x = torch.empty(a.nb * a.b, dtype=torch.float64, device=DEV)
    W.recover(_t(g), _t(xs), x)
    assert np.array_equal(_bits(x.cpu().numpy()), _bits(O.recover(g, xs)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_reduction_bit_exact(name):
    a = CASES[name]()
    rp, ci, v = _t(a.row_ptr), _t(a.col_idx), _t(a.values.reshape(-1))
    W = msp.Wells(a.nb, a.b, a.n_wells, rp, ci, v)
    O = oracle.Wells(a, a.n_wells)
    _check_bit_exact(a, W, O, 11)
    v2 = a.values * (1.0 + 0.02 * np.random.default_rng(5).normal(size=a.values.shape))
    W.update_values(_t(v2.reshape(-1)))
    O.update_values(v2)
    _check_bit_exact(a, W, O, 12)
    W.close()
    O.close()


def test_recover_in_place():
    a = CASES["b3_two_wells"]()
    W = msp.Wells(a.nb, a.b, a.n_wells, _t(a.row_ptr), _t(a.col_idx), _t(a.values.reshape(-1)))
    O = oracle.Wells(a, a.n_wells)
    g = _rhs_with_wells(a, 3)
    xs = np.random.default_rng(4).normal(size=W.nr * a.b)
    buf = torch.zeros(a.nb * a.b, dtype=torch.float64, device=DEV)
    buf[:W.nr * a.b] = _t(xs)
    W.recover(_t(g), buf, buf)
    assert np.array_equal(_bits(buf.cpu().numpy()), _bits(O.recover(g, xs)))


@pytest.mark.parametrize("name,cfg", [("spe10_like_b4", dict(coarse_max=120)),
                                      ("b3_two_wells", dict(coarse_max=30))])
def test_eliminated_solve_matches_oracle(name, cfg):
    a = CASES[name]()
    S = msp.WellEliminatedSolver(a.nb, a.b, a.n_wells, _t(a.row_ptr), _t(a.col_idx),
                                 _t(a.values.reshape(-1)), **cfg)
    O = oracle.Wells(a, a.n_wells)
    orp, oci, ov = O.reduced()
    red = BSRMatrix(nb=O.nr, b=a.b, row_ptr=orp, col_idx=oci, values=ov.reshape(-1, a.b, a.b),
                    n_cells=O.nr)
    ref = oracle.Oracle(red, **cfg)
    g = _rhs_with_wells(a, 31)
    x = torch.zeros(a.nb * a.b, dtype=torch.float64, device=DEV)
    info = S.solve(_t(g), x, 1e-6)
    gs = O.reduce_rhs(g)
    _, oinfo = ref.solve(gs, 1e-6)
    assert info["status"] == 0
    assert abs(info["iterations"] - oinfo["iterations"]) <= 1
    r = g - a.to_scipy() @ x.cpu().numpy()
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(gs) * 1.001
    ref.close()
    S.close()
    O.close()


def test_rejected_layouts():
    chain = [(0, 1), (1, 2)]

    def make(a):
        return msp.Wells(a.nb, a.b, 2, _t(a.row_ptr), _t(a.col_idx), _t(a.values.reshape(-1)))

    make(_tiny(chain + [(1, 3), (2, 4)], 5)).close()               # one well per cell: fine
    for pairs in (chain + [(1, 3), (1, 4)],                        # cell 1 on two wells
                  chain + [(1, 3), (2, 4), (3, 4)]):               # wells coupled
        with pytest.raises(msp.MspError) as e:
            make(_tiny(pairs, 5))
        assert e.value.status == msp._native.MSP_ERR_ARG
    a = _tiny(chain, 5)
    with pytest.raises(msp.MspError):
        msp.Wells(a.nb, a.b, a.nb, _t(a.row_ptr), _t(a.col_idx), _t(a.values.reshape(-1)))


@pytest.mark.slow
def test_full_size_reduction_and_solve():
    a = grid_spe10()
    rp, ci, v = _t(a.row_ptr), _t(a.col_idx), _t(a.values.reshape(-1))
    S = msp.WellEliminatedSolver(a.nb, a.b, a.n_wells, rp, ci, v)
    O = oracle.Wells(a, a.n_wells)
    _check_bit_exact(a, S.wells, O, 41)
    S.update_values(v)  # back to the original values after the check's own inputs
    g = random_rhs(a, 42)
    x = torch.zeros(a.nb * a.b, dtype=torch.float64, device=DEV)
    info = S.solve(_t(g), x, 1e-6)
    assert info["status"] == 0
    r = g - a.to_scipy() @ x.cpu().numpy()
    gs = O.reduce_rhs(g)
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(gs) * 1.001
    S.close()
    O.close()


def _compact_wells(a):
    """The one-unknown form of a matrix whose wells are identity-padded block rows: the
    cell matrix A_RR, the perforated cells of every well (ascending), A_RW (column 0 of
    the cell-well blocks), A_WR (row 0 of the well-cell blocks) and A_WW (entry (0, 0) of
    the well's diagonal block)."""
    nr, nw, b = a.n_cells, a.n_wells, a.b
    rp, ci, v = [0], [], []
    arw_of = {}
    for c in range(nr):
        for p in range(a.row_ptr[c], a.row_ptr[c + 1]):
            j = int(a.col_idx[p])
            if j < nr:
                ci.append(j)
                v.append(a.values[p])
            else:
                arw_of[c] = a.values[p][:, 0].copy()
        rp.append(len(ci))
    wptr, cells, arw, awr, aww = [0], [], [], [], []
    for w in range(nw):
        i = nr + w
        for p in range(a.row_ptr[i], a.row_ptr[i + 1]):
            j = int(a.col_idx[p])
            if j < nr:
                cells.append(j)
                awr.append(a.values[p][0, :].copy())
                arw.append(arw_of[j])
            elif j == i:
                aww.append(a.values[p][0, 0])
        wptr.append(len(cells))
    return (np.array(rp, np.int32), np.array(ci, np.int32), np.array(v).reshape(-1, b, b),
            np.array(wptr, np.int32), np.array(cells, np.int32),
            np.array(arw).reshape(-1, b), np.array(awr).reshape(-1, b), np.array(aww))


def _padded(nr, b, rp, ci, v, wptr, cells, arw, awr, aww):
    """The same system with every well padded to a b x b block row: A_RW in column 0,
    A_WR in row 0, A_WW at (0, 0) of an identity block (Eq. Jacobian-system with the
    well's extra unknowns decoupled)."""
    nw = len(aww)
    perf = {int(c): k for k, c in enumerate(cells)}
    well = {int(c): w for w in range(nw) for c in cells[wptr[w]:wptr[w + 1]]}
    prp, pci, pv = [0], [], []
    for c in range(nr):
        for p in range(rp[c], rp[c + 1]):
            pci.append(int(ci[p]))
            pv.append(v[p])
        if c in perf:
            blk = np.zeros((b, b))
            blk[:, 0] = arw[perf[c]]
            pci.append(nr + well[c])
            pv.append(blk)
        prp.append(len(pci))
    for w in range(nw):
        for k in range(wptr[w], wptr[w + 1]):
            blk = np.zeros((b, b))
            blk[0, :] = awr[k]
            pci.append(int(cells[k]))
            pv.append(blk)
        d = np.eye(b)
        d[0, 0] = aww[w]
        pci.append(nr + w)
        pv.append(d)
        prp.append(len(pci))
    return BSRMatrix(nb=nr + nw, b=b, row_ptr=np.array(prp, np.int32),
                     col_idx=np.array(pci, np.int32), values=np.array(pv).reshape(-1, b, b),
                     n_cells=nr, n_wells=nw)


@pytest.mark.parametrize("name", ["b3_two_wells", "spe10_like_b4", "b2_three_wells"])
def test_one_unknown_wells_match_the_oracle(name):
    """msp_wells_setup_scalar: the compact form (A_RR, perforations, A_RW, A_WR, scalar
    A_WW) gives the reduced matrix, right-hand side and recovered unknowns of the oracle's
    elimination of the padded system bit for bit, and A_S equals the scalar Schur
    complement A_RR - A_RW A_WR / A_WW."""
    a = CASES[name]()
    nr, nw, b = a.n_cells, a.n_wells, a.b
    rp, ci, v, wptr, cells, arw, awr, aww = _compact_wells(a)
    W = msp.ScalarWells(nr, b, nw, _t(rp), _t(ci), _t(v.reshape(-1)), _t(wptr), _t(cells),
                        _t(arw.reshape(-1)), _t(awr.reshape(-1)), _t(aww))
    ap = _padded(nr, b, rp, ci, v, wptr, cells, arw, awr, aww)
    O = oracle.Wells(ap, nw)
    srp, sci, sv = W.reduced()
    orp, oci, ov = O.reduced()
    assert np.array_equal(srp.cpu().numpy(), orp) and np.array_equal(sci.cpu().numpy(), oci)
    assert np.array_equal(_bits(sv.cpu().numpy()), _bits(ov))
    # closed form of the scalar Schur complement
    dense = np.zeros((nr * b, nr * b))
    for c in range(nr):
        for p in range(rp[c], rp[c + 1]):
            dense[c * b:(c + 1) * b, ci[p] * b:(ci[p] + 1) * b] = v[p]
    for w in range(nw):
        for k in range(wptr[w], wptr[w + 1]):
            for k2 in range(wptr[w], wptr[w + 1]):
                c, c2 = cells[k], cells[k2]
                dense[c * b:(c + 1) * b, c2 * b:(c2 + 1) * b] -= np.outer(arw[k], awr[k2]) / aww[w]
    got = np.zeros_like(dense)
    svh = sv.cpu().numpy().reshape(-1, b, b)
    for c in range(nr):
        for p in range(orp[c], orp[c + 1]):
            got[c * b:(c + 1) * b, oci[p] * b:(oci[p] + 1) * b] = svh[p]
    assert np.allclose(got, dense, rtol=1e-13, atol=1e-13 * np.abs(dense).max())
    # right-hand side and recovery through the padded layout
    rng = np.random.default_rng(5)
    gr, gw = rng.normal(size=nr * b), rng.normal(size=nw)
    g = torch.empty((nr + nw) * b, dtype=torch.float64, device=DEV)
    W.pack_rhs(_t(gr), _t(gw), g)
    gpad = np.concatenate([gr, np.concatenate([[gw[w]] + [0.0] * (b - 1) for w in range(nw)])])
    assert np.array_equal(g.cpu().numpy(), gpad)
    gs = torch.empty(nr * b, dtype=torch.float64, device=DEV)
    W.reduce_rhs(g, gs)
    assert np.array_equal(_bits(gs.cpu().numpy()), _bits(O.reduce_rhs(gpad)))
    xs = rng.normal(size=nr * b)
    x = torch.empty((nr + nw) * b, dtype=torch.float64, device=DEV)
    W.recover(g, _t(xs), x)
    ox = O.recover(gpad, xs)
    assert np.array_equal(_bits(x.cpu().numpy()), _bits(ox))
    xr = torch.empty(nr * b, dtype=torch.float64, device=DEV)
    xw = torch.empty(nw, dtype=torch.float64, device=DEV)
    W.unpack(x, xr, xw)
    assert np.array_equal(xr.cpu().numpy(), xs)
    assert np.array_equal(xw.cpu().numpy(), ox.reshape(-1, b)[nr:, 0])
    # x_W = (g_W - A_WR x_R) / A_WW
    for w in range(nw):
        ref = gw[w] - sum(awr[k] @ xs[cells[k] * b:(cells[k] + 1) * b]
                          for k in range(wptr[w], wptr[w + 1]))
        assert np.isclose(xw[w].item(), ref / aww[w], rtol=1e-12)
    # new values
    v2 = v * 1.01
    W.update_values(_t(v2.reshape(-1)), _t(arw.reshape(-1) * 0.9), _t(awr.reshape(-1)), _t(aww * 1.1))
    O2 = oracle.Wells(_padded(nr, b, rp, ci, v2, wptr, cells, arw * 0.9, awr, aww * 1.1), nw)
    assert np.array_equal(_bits(W.reduced()[2].cpu().numpy()), _bits(O2.reduced()[2]))
    W.close()
    O.close()
    O2.close()


def test_one_unknown_wells_rejected_layouts():
    a = CASES["b3_two_wells"]()
    nr, nw, b = a.n_cells, a.n_wells, a.b
    rp, ci, v, wptr, cells, arw, awr, aww = _compact_wells(a)
    bad = cells.copy()
    bad[1], bad[0] = bad[0], bad[1]  # not ascending within the well
    with pytest.raises(msp.MspError) as e:
        msp.ScalarWells(nr, b, nw, _t(rp), _t(ci), _t(v.reshape(-1)), _t(wptr), _t(bad),
                        _t(arw.reshape(-1)), _t(awr.reshape(-1)), _t(aww))
    assert e.value.status == -1
    twice = cells.copy()
    twice[wptr[1]] = cells[0]  # a cell perforated by two wells
    twice[wptr[1]:wptr[2]] = np.sort(twice[wptr[1]:wptr[2]])
    with pytest.raises(msp.MspError) as e:
        msp.ScalarWells(nr, b, nw, _t(rp), _t(ci), _t(v.reshape(-1)), _t(wptr), _t(twice),
                        _t(arw.reshape(-1)), _t(awr.reshape(-1)), _t(aww))
    assert e.value.status == -1
