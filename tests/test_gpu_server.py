"""The request loop (msp_server_*) on the GPU: several systems of different sizes and block
sizes, each a Newton-like sequence (same pattern, values perturbed by up to 5 % per step),
solved (a) each alone, one request at a time, and (b) all in one mix with four concurrent
slots.  Every solution of the mix equals the one computed alone bit for bit (each system
runs the same deterministic kernels on its own buffers), and equals the single-handle
API's (Solver: setup, then update_values + solve per step); every solve reaches the
tolerance; a budget that holds only some of the systems forces releases and still gives
converged results; the handle footprint stays below the admission estimate."""
import numpy as np
import pytest

from synthetic import box_jacobian, perturb_values, random_rhs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_08594_gb300 as msp  # noqa: E402

SYSTEMS = [  # (nx, ny, nz, b, wells)
    (12, 10, 6, 4, 1), (20, 9, 5, 3, 0), (8, 8, 12, 6, 2), (16, 14, 7, 2, 1), (10, 6, 9, 5, 0),
    (24, 11, 4, 4, 1),
]
STEPS = 3


@pytest.fixture(scope="module")
def streams():
    out = []
    for key, (nx, ny, nz, b, w) in enumerate(SYSTEMS):
        a = box_jacobian(nx, ny, nz, b, 100 + key, layered=True, kz_ratio=0.1, n_wells=w)
        vals, cur = [], a
        for k in range(STEPS):
            v = np.ascontiguousarray(perturb_values(cur, 300 + 10 * key + k).reshape(-1))
            vals.append(v)
            cur = a.__class__(**{**a.__dict__, "values": v.reshape(a.values.shape)})
        rhs = [np.ascontiguousarray(random_rhs(a, 500 + 10 * key + k)) for k in range(STEPS)]
        out.append((a, vals, rhs))
    return out


def _submit_all(server, streams, order):
    tickets, xs = {}, {}
    for key, k in order:
        a, vals, rhs = streams[key]
        x = np.zeros(a.nb * a.b)
        xs[(key, k)] = x
        tickets[(key, k)] = server.submit(key, a.nb, a.b, rhs[k], x, values=vals[k],
                                          row_ptr=a.row_ptr, col_idx=a.col_idx, rel_tol=1e-6)
    return tickets, xs


def _cfg():
    return dict(coarse_max=60, mu=8)


def test_mix_equals_alone(streams):
    alone = {}
    S = msp.Server(slots=1, **_cfg())
    for key in range(len(streams)):
        for k in range(STEPS):
            t, xs = _submit_all(S, streams, [(key, k)])
            r = S.wait(t[(key, k)], 120.0)
            assert r is not None and r["status"] == 0, r
            alone[(key, k)] = (xs[(key, k)].copy(), r)
    S.close()

    order = [(key, k) for k in range(STEPS) for key in range(len(streams))]
    S = msp.Server(slots=4, **_cfg())
    tickets, xs = _submit_all(S, streams, order)
    res = {kk: S.wait(t, 300.0) for kk, t in tickets.items()}
    st = S.stats()
    S.close()
    assert st["completed"] == len(order) and st["evictions"] == 0
    slots_used = {r["slot"] for r in res.values()}
    assert len(slots_used) > 1
    for kk, r in res.items():
        assert r["status"] == 0, (kk, r)
        assert r["setup"] == (1 if kk[1] == 0 else 0)
        x_alone, r_alone = alone[kk]
        assert r["info"]["iterations"] == r_alone["info"]["iterations"], kk
        assert r["info"]["setup_performed"] == r_alone["info"]["setup_performed"], kk
        assert np.array_equal(xs[kk].view(np.int64), x_alone.view(np.int64)), kk
        a, vals, rhs = streams[kk[0]]
        A = a.__class__(**{**a.__dict__, "values": vals[kk[1]].reshape(a.values.shape)})
        rr = rhs[kk[1]] - A.to_scipy() @ xs[kk]
        assert np.linalg.norm(rr) <= 1e-6 * np.linalg.norm(rhs[kk[1]]) * 1.001

    # the single-handle API gives the same solutions
    dev = torch.device("cuda:0")
    for key in (0, 2):
        a, vals, rhs = streams[key]
        s = msp.Solver(a.nb, a.b, torch.from_numpy(a.row_ptr).to(dev),
                       torch.from_numpy(a.col_idx).to(dev), torch.from_numpy(vals[0]).to(dev),
                       **_cfg())
        for k in range(STEPS):
            if k:
                s.update_values(torch.from_numpy(vals[k]).to(dev))
            x = torch.zeros(a.nb * a.b, dtype=torch.float64, device=dev)
            s.solve(torch.from_numpy(rhs[k]).to(dev), x, 1e-6)
            assert np.array_equal(x.cpu().numpy().view(np.int64), xs[(key, k)].view(np.int64))
        s.close()


def test_budget_forces_releases(streams):
    cfg = msp.msp_config_default(**_cfg())
    est = [msp.msp_estimate_device_bytes(a.nb, a.b, a.nnzb, cfg) for a, _, _ in streams]
    # a new system is charged its estimate until it is set up, so with 1.3 x the largest
    # estimate every admission beyond the first few has to release an idle system
    budget = int(1.3 * max(est))
    S = msp.Server(slots=3, hbm_budget=budget, **_cfg())
    order = [(key, k) for k in range(STEPS) for key in range(len(streams))]
    tickets, xs = _submit_all(S, streams, order)
    res = {kk: S.wait(t, 300.0) for kk, t in tickets.items()}
    st = S.stats()
    S.close()
    assert st["evictions"] > 0 and st["peak_charged_bytes"] <= budget
    for kk, r in res.items():
        assert r["status"] == 0, (kk, r)
        a, vals, rhs = streams[kk[0]]
        A = a.__class__(**{**a.__dict__, "values": vals[kk[1]].reshape(a.values.shape)})
        rr = rhs[kk[1]] - A.to_scipy() @ xs[kk]
        assert np.linalg.norm(rr) <= 1e-6 * np.linalg.norm(rhs[kk[1]]) * 1.001


def test_footprint_within_estimate(streams):
    dev = torch.device("cuda:0")
    cfg = msp.msp_config_default(**_cfg())
    for a, vals, rhs in streams[:3]:
        s = msp.Solver(a.nb, a.b, torch.from_numpy(a.row_ptr).to(dev),
                       torch.from_numpy(a.col_idx).to(dev), torch.from_numpy(vals[0]).to(dev),
                       **_cfg())
        x = np.zeros(a.nb * a.b)
        s.update_values_host(vals[1])
        s.solve_host(rhs[0], x)
        used = msp.msp_device_bytes(s.h)
        est = msp.msp_estimate_device_bytes(a.nb, a.b, a.nnzb, cfg)
        assert 0 < used <= est, (used, est)
        s.close()
