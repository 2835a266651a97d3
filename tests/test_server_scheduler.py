"""The request server's scheduler on the host (no GPU): a server made by
trm_server_create_fn runs a Python function per admitted request instead of
a GPU solve, so admission in arrival order, the memory budget, the bound on
concurrent solves, refusals, waits and status propagation are checked with
real threads and the real admission rule."""
import ctypes as ct
import threading
import time

import pytest


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


class Recorder:
    """Stands in for the solver: records when each request (identified by
    opt.seed) runs, how many run at once and their summed footprints."""

    def __init__(self, trm, hold=0.05, fail=()):
        self.trm, self.hold, self.fail = trm, hold, set(fail)
        self.lock = threading.Lock()
        self.live = self.used = self.max_live = self.max_used = 0
        self.start, self.end = {}, {}
        self.cfn = trm.TRM_SERVER_FN(self._run)

    def _run(self, pp, lam, eg, stats, ctx):
        p = ct.cast(pp, ct.POINTER(self.trm.trm_problem)).contents
        idx = int(p.opt.seed)
        fp = self.trm.trm_footprint_bytes(p.nx * p.ny * p.nz, p.m)
        with self.lock:
            self.start[idx] = time.monotonic()
            self.live += 1
            self.used += fp
            self.max_live = max(self.max_live, self.live)
            self.max_used = max(self.max_used, self.used)
        time.sleep(self.hold)
        for j in range(p.m):
            lam[j] = idx + j
        eg[0] = float(idx)
        with self.lock:
            self.live -= 1
            self.used -= fp
            self.end[idx] = time.monotonic()
        return -4 if idx in self.fail else 0


def _server(trm, rec, budget, max_live):
    return trm.trm_server_create_fn(budget, max_live, rec.cfn)


def _submit(trm, srv, n, m, idx):
    opt = trm.trm_default_options(seed=idx)
    return trm.trm_server_submit(srv, (n, n, n), 2, 1.0, None, m, 1e-8, opt)


def test_concurrency_budget_results_and_status(trm):
    rec = Recorder(trm, fail={5})
    sizes = [(12, 8), (16, 16), (20, 24), (14, 12), (18, 40), (16, 8),
             (12, 32), (22, 16), (16, 64), (12, 8)]
    fps = [trm.trm_footprint_bytes(n ** 3, m) for n, m in sizes]
    budget = sum(sorted(fps)[-3:])          # room for about three at a time
    srv = _server(trm, rec, budget, 4)
    try:
        tickets = [_submit(trm, srv, n, m, i)
                   for i, (n, m) in enumerate(sizes)]
        out = [trm.trm_server_wait(srv, t, m)
               for t, (_, m) in zip(tickets, sizes)]
    finally:
        trm.trm_server_destroy(srv)
    assert 2 <= rec.max_live <= 4            # concurrent, never above max_live
    assert rec.max_used <= budget            # never above the memory budget
    for i, ((n, m), (lam, eg, _, status, lat)) in enumerate(zip(sizes, out)):
        assert list(lam) == [float(i + j) for j in range(m)] and eg == i
        assert status == (-4 if i == 5 else 0)
        assert lat >= rec.hold * 0.9


def test_admission_is_in_arrival_order(trm):
    """A request that does not fit waits at the head of the queue, and the
    requests behind it wait too even where they would fit now."""
    rec = Recorder(trm, hold=0.1)
    small = trm.trm_footprint_bytes(12 ** 3, 8)
    big = trm.trm_footprint_bytes(24 ** 3, 64)
    budget = big + small // 2                # big fits alone, not beside small
    srv = _server(trm, rec, budget, 8)
    try:
        ta = _submit(trm, srv, 12, 8, 0)      # runs at once
        time.sleep(0.02)
        tb = _submit(trm, srv, 24, 64, 1)     # waits for 0 to finish
        tc = _submit(trm, srv, 12, 8, 2)      # would fit beside 0, waits for 1
        for t, m in ((ta, 8), (tb, 64), (tc, 8)):
            assert trm.trm_server_wait(srv, t, m)[3] == 0
    finally:
        trm.trm_server_destroy(srv)
    assert rec.start[1] >= rec.end[0]
    assert rec.start[2] >= rec.start[1]
    assert rec.max_used <= budget


def test_refusals(trm):
    rec = Recorder(trm, hold=0.0)
    fp = trm.trm_footprint_bytes(16 ** 3, 16)
    srv = _server(trm, rec, fp, 2)
    try:
        with pytest.raises(trm.TrmError) as e:     # alone above the budget
            _submit(trm, srv, 20, 16, 0)
        assert e.value.status == -2
        with pytest.raises(trm.TrmError) as e:     # m >= N
            _submit(trm, srv, 2, 8, 1)
        assert e.value.status == -1
        t = _submit(trm, srv, 16, 16, 2)
        assert trm.trm_server_wait(srv, t, 16)[3] == 0
        # a ticket is released by its wait
        assert trm.lib.trm_server_wait(srv, t, None, None, None, None) == -1
    finally:
        trm.trm_server_destroy(srv)
    with pytest.raises(trm.TrmError) as e:
        trm.trm_server_create_fn(1 << 30, 2, None)
    assert e.value.status == -1
