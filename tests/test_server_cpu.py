"""Host-side checks of the request loop (msp_server_*) without a GPU: a recording executor
replaces the CUDA solver, so the scheduling itself is tested — per-key order and mutual
exclusion, overlap across keys, the device-memory budget with least-recently-used
release of idle systems, submit-order admission of requests that wait for memory,
release and new-pattern requests, rejection of a system larger than the budget."""
import threading
import time

import numpy as np
import pytest

from paper_2208_08594_gb300 import _native

NB, B, NNZB = 1000, 4, 7000


class Recorder:
    """Executor that sleeps for a request and logs (event, key, slot, t, setup)."""

    def __init__(self, run_s=0.02, bytes_of=None):
        self.run_s = run_s
        self.bytes_of = bytes_of or (lambda key: EST)
        self.log = []
        self.alive = {}  # key -> bytes of the systems the executor holds
        self.max_alive = 0
        self.active = set()
        self.max_active = 0
        self.overlap_same_key = False
        self.mu = threading.Lock()
        self.fn = _native.MSP_SERVER_EXEC_FN(self._exec)

    def _exec(self, user, op, req, slot, setup, bytes_out):
        key = req.contents.key
        if op == _native.MSP_EXEC_RELEASE:
            with self.mu:
                self.alive.pop(key, None)
                self.log.append(("release", key, slot, time.monotonic(), 0))
            return 0
        with self.mu:
            if key in self.active:
                self.overlap_same_key = True
            self.active.add(key)
            self.max_active = max(self.max_active, len(self.active))
            if setup:
                self.alive[key] = self.bytes_of(key)
            self.max_alive = max(self.max_alive, sum(self.alive.values()))
            self.log.append(("start", key, slot, time.monotonic(), setup))
        time.sleep(self.run_s)
        with self.mu:
            self.active.discard(key)
            self.log.append(("end", key, slot, time.monotonic(), setup))
        bytes_out[0] = self.bytes_of(key)
        return 0


EST = None


@pytest.fixture(scope="module", autouse=True)
def _estimate():
    global EST
    EST = _native.msp_estimate_device_bytes(NB, B, NNZB)
    assert EST > NNZB * B * B * 8


def _request(key, flags=0, nb=NB, nnzb=NNZB):
    rp = np.zeros(nb + 1, np.int32)
    ci = np.zeros(nnzb, np.int32)
    v = np.zeros(nnzb * B * B)
    g = np.zeros(nb * B)
    x = np.zeros(nb * B)
    req = _native.MspRequest()
    req.key, req.nb, req.b, req.nnzb = key, nb, B, nnzb
    req.h_row_ptr, req.h_col_idx, req.h_values = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
    req.h_rhs, req.h_x, req.rel_tol, req.flags = g.ctypes.data, x.ctypes.data, 1e-6, flags
    return req, (rp, ci, v, g, x)


def _run(slots, budget, keys_flags, rec):
    S = _native.msp_server_create(slots, budget, None, 0, rec.fn)
    keep, tickets = [], []
    for key, flags in keys_flags:
        req, arrays = _request(key, flags)
        keep.append(arrays)
        tickets.append(_native.msp_server_submit(S, req))
    results = [_native.msp_server_wait(S, t, 30.0) for t in tickets]
    stats = _native.msp_server_get_stats(S)
    rec.before_free = list(rec.log)
    _native.msp_server_free(S)  # releases the systems still resident
    return results, stats


def test_per_key_order_and_overlap_across_keys():
    rec = Recorder()
    order = [(k % 4, 0) for k in range(16)]  # 4 keys x 4 Newton steps, interleaved
    results, stats = _run(4, 100 * EST, order, rec)
    assert all(r is not None and r["status"] == 0 for r in results)
    assert not rec.overlap_same_key
    assert rec.max_active > 1  # different keys ran at the same time
    starts = [(k, t) for e, k, s, t, _ in rec.log if e == "start"]
    for key in range(4):
        ts = [t for k, t in starts if k == key]
        assert ts == sorted(ts) and len(ts) == 4
    # the first request of a key sets it up, the later ones reuse it
    for key in range(4):
        mine = [r for r in results if r["key"] == key]
        assert [r["setup"] for r in mine] == [1, 0, 0, 0]
    assert stats["completed"] == 16 and stats["resident_systems"] == 4
    assert stats["evictions"] == 0


def test_budget_and_lru_release():
    rec = Recorder(run_s=0.01)
    # room for two systems; keys 0, 1, 0, then 2 must release key 1 (least recently used)
    results, stats = _run(1, int(2.5 * EST), [(0, 0), (1, 0), (0, 0), (2, 0)], rec)
    assert all(r["status"] == 0 for r in results)
    rel = [k for e, k, *_ in rec.before_free if e == "release"]
    assert rel == [1]
    assert sorted(k for e, k, *_ in rec.log[len(rec.before_free):]) == [0, 2]
    assert rec.max_alive <= 2.5 * EST
    assert stats["evictions"] == 1 and stats["peak_charged_bytes"] <= 2.5 * EST


def test_memory_waiters_keep_their_order():
    rec = Recorder(run_s=0.03)
    # budget for one system at a time, several slots: the new keys start in submit order
    keys = [(k, 0) for k in range(5)]
    results, stats = _run(4, int(1.5 * EST), keys, rec)
    assert all(r["status"] == 0 for r in results)
    starts = [k for e, k, *_ in rec.log if e == "start"]
    assert starts == list(range(5))
    assert rec.max_active == 1 and rec.max_alive <= 1.5 * EST
    assert stats["evictions"] == 4


def test_release_and_new_pattern():
    rec = Recorder(run_s=0.005)
    R, N = _native.MSP_REQ_RELEASE, _native.MSP_REQ_NEW_PATTERN
    results, stats = _run(2, 100 * EST, [(7, 0), (7, R), (7, 0), (7, N), (7, 0)], rec)
    assert [r["setup"] for r in results] == [1, 0, 1, 1, 0]
    events = [(e, k) for e, k, *_ in rec.before_free if e in ("start", "release")]
    # release after the second request; the new pattern releases the old system first
    assert events == [("start", 7), ("start", 7), ("release", 7), ("start", 7), ("release", 7),
                      ("start", 7), ("start", 7)]
    assert stats["resident_systems"] == 1


def test_replacement_passes_a_memory_waiter():
    """Two resident systems fill the budget and each has a new-pattern request queued
    behind a third key that needs room: the replacements go first (their systems cannot be
    released while they have requests queued), then the third key evicts one of them."""
    rec = Recorder(run_s=0.005)
    N = _native.MSP_REQ_NEW_PATTERN
    results, stats = _run(1, int(2.5 * EST), [(0, 0), (1, 0), (2, 0), (0, N), (1, N)], rec)
    assert all(r is not None and r["status"] == 0 for r in results)
    starts = [k for e, k, *_ in rec.before_free if e == "start"]
    assert starts[:2] == [0, 1] and sorted(starts[2:]) == [0, 1, 2]
    assert starts.index(2, 2) > 2  # key 2 started after a replacement
    assert rec.max_alive <= 2.5 * EST


def test_first_value_update_is_charged_before_it_runs():
    """A system's footprint grows once after its setup: its first update of values from the
    host allocates the staging copy (nnzb * b * b doubles).  Budget 2 x the estimate minus
    half a copy: keys 0 and 1 set up and key 0 updates; key 1's update would take the
    total past the budget, so it is charged the copy first and the idle key 0 is released
    before it runs (without that charge the total would exceed the budget afterwards)."""
    nb, nnzb = 200, 20000
    est = _native.msp_estimate_device_bytes(nb, B, nnzb)
    copy = nnzb * B * B * 8
    assert copy > 0.1 * est
    grown = set()

    class Staging(Recorder):
        def _exec(self, user, op, req, slot, setup, bytes_out):
            st = super()._exec(user, op, req, slot, setup, bytes_out)
            if op != _native.MSP_EXEC_RELEASE:
                key = req.contents.key
                if setup:
                    grown.discard(key)
                else:
                    grown.add(key)
                with self.mu:
                    self.alive[key] = est - 1000 - (0 if key in grown else copy)
                    self.max_alive = max(self.max_alive, sum(self.alive.values()))
                bytes_out[0] = self.alive[key]
            return st

    budget = 2 * est - copy // 2

    def run(keys):
        rec = Staging(run_s=0.005, bytes_of=lambda key: est - 1000 - copy)
        grown.clear()
        S = _native.msp_server_create(1, budget, None, 0, rec.fn)
        keep, tickets = [], []
        for key in keys:
            req, arrays = _request(key, 0, nb=nb, nnzb=nnzb)
            keep.append(arrays)
            tickets.append(_native.msp_server_submit(S, req))
        results = [_native.msp_server_wait(S, t, 30.0) for t in tickets]
        stats = _native.msp_server_get_stats(S)
        released = [k for e, k, *_ in rec.log if e == "release"]
        _native.msp_server_free(S)
        assert all(r["status"] == 0 for r in results)
        assert stats["peak_charged_bytes"] <= budget
        assert rec.max_alive <= budget
        return [r["setup"] for r in results], released

    # key 0 is idle with nothing queued when key 1 updates: it is released
    assert run((0, 1, 0, 1)) == ([1, 1, 0, 0], [0])
    # key 0 has a request queued (with its pattern) and nothing runs: it is released all
    # the same and set up again by that request (which in turn releases the idle key 1)
    assert run((0, 1, 0, 1, 0)) == ([1, 1, 0, 0, 1], [0, 1])


def test_oversized_request_rejected_and_bad_arguments():
    rec = Recorder()
    S = _native.msp_server_create(2, EST // 2, None, 0, rec.fn)
    req, keep = _request(3)
    t = _native.msp_server_submit(S, req)
    r = _native.msp_server_wait(S, t, 5.0)
    assert r["status"] == _native.MSP_ERR_NOMEM and r["slot"] == -1
    assert _native.msp_server_get_stats(S)["rejected"] == 1
    with pytest.raises(_native.MspError):
        _native.msp_server_wait(S, t, 0.0)  # retired ticket
    bad, keep2 = _request(4)
    bad.rel_tol = 0.0
    with pytest.raises(_native.MspError):
        _native.msp_server_submit(S, bad)
    _native.msp_server_free(S)
    with pytest.raises(_native.MspError):
        _native.msp_server_create(0, EST, None, 0, rec.fn)
    assert not rec.log
