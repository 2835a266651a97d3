"""The request server (serving row of the hot-path table): problems of
different sizes solved concurrently give the same bytes as when each is
solved alone on its own handle, and the results are the oracle's."""
import numpy as np
import pytest

import trm_inputs as ti
from oracle import operator as op

from . import gpu_util as gu

pytestmark = pytest.mark.gpu

# (grid edge, order, wells, m, well seed)
MIX = [(12, 2, 4, 8, 1), (16, 4, 8, 16, 2), (20, 2, 12, 24, 3),
       (14, 4, 6, 12, 4), (24, 4, 16, 32, 5), (18, 2, 10, 40, 6),
       (22, 4, 20, 48, 7), (16, 2, 4, 64, 8)]


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


def _problem(n, order, wells, seed):
    shape = (n, n, n)
    return shape, ti.gaussian_wells(shape, wells, seed=seed)


def _opts(trm):
    return trm.trm_default_options(precision=trm.TRM_MIXED, precond=1, seed=3)


def test_mix_equals_solo_and_oracle(trm):
    solo = []
    for n, order, wells, m, seed in MIX:
        shape, V = _problem(n, order, wells, seed)
        opt = _opts(trm)
        opt.stream = gu.stream()
        h = trm.trm_create_stencil(n, n, n, order, 1.0, V, m, 1e-9, opt)
        try:
            lam, eg, st, status = trm.trm_solve(h, n ** 3, m)
        finally:
            trm.trm_destroy(h)
        assert status == 0
        solo.append((lam, eg))
    budget = 4 * sum(trm.trm_footprint_bytes(n ** 3, m) for n, _, _, m, _ in MIX)
    srv = trm.trm_server_create(budget, 6)
    try:
        tickets = []
        for n, order, wells, m, seed in MIX:
            shape, V = _problem(n, order, wells, seed)
            tickets.append(trm.trm_server_submit(srv, shape, order, 1.0, V, m,
                                                 1e-9, _opts(trm)))
        got = [trm.trm_server_wait(srv, t, m) for t, (_, _, _, m, _) in
               zip(tickets, MIX)]
    finally:
        trm.trm_server_destroy(srv)
    for (lam, eg, st, status, lat), (lam0, eg0) in zip(got, solo):
        assert status == 0 and lat > 0
        assert np.array_equal(lam, lam0) and eg == eg0
    # the smallest problem against dense eigenvalues of the oracle's H
    n, order, wells, m, seed = MIX[0]
    shape, V = _problem(n, order, wells, seed)
    ref = op.lowest_eigenvalues(op.grid_hamiltonian(shape, order, 1.0, V), m)
    assert np.max(np.abs(got[0][0] - ref)) < 1e-9


def test_admission_by_footprint(trm):
    """A problem whose footprint exceeds the budget is refused at submission;
    a budget of one solve runs the queue one at a time, in order."""
    n, m = 16, 16
    fp = trm.trm_footprint_bytes(n ** 3, m)
    srv = trm.trm_server_create(fp, 4)
    try:
        with pytest.raises(trm.TrmError) as e:
            trm.trm_server_submit(srv, (24, 24, 24), 2, 1.0, None, 64, 1e-8,
                                  _opts(trm))
        assert e.value.status == -2
        ts = [trm.trm_server_submit(srv, (n, n, n), 2, 1.0, None, m, 1e-8,
                                    _opts(trm)) for _ in range(3)]
        outs = [trm.trm_server_wait(srv, t, m) for t in ts]
    finally:
        trm.trm_server_destroy(srv)
    assert all(o[3] == 0 for o in outs)
    assert outs[0][4] < outs[1][4] < outs[2][4]  # served in order, one at a time
    assert np.array_equal(outs[0][0], outs[2][0])


def test_warm_start_across_related_requests(trm):
    """Next row 2 of the scope table: a request started from the converged
    block of a related one (the same grid, the potential scaled by 1.02)
    needs fewer iterations than a cold start and reaches the same
    eigenvalues (the oracle's dense diagonalisation, 1e-9)."""
    n, order, m = 16, 4, 16
    shape, N = (n, n, n), n ** 3
    V = ti.gaussian_wells(shape, 8, seed=11)
    V2 = 1.02 * V
    srv = trm.trm_server_create(4 * trm.trm_footprint_bytes(N, m), 4)
    try:
        CA = np.zeros((N, m), order="F")
        ta = trm.trm_server_submit(srv, shape, order, 1.0, V, m, 1e-9,
                                   _opts(trm), C_out=CA)
        lam_a, eg_a, st_a, s_a, _ = trm.trm_server_wait(srv, ta, m)
        tc = trm.trm_server_submit(srv, shape, order, 1.0, V2, m, 1e-9,
                                   _opts(trm))
        tw = trm.trm_server_submit(srv, shape, order, 1.0, V2, m, 1e-9,
                                   _opts(trm), C0=CA)
        lam_c, eg_c, st_c, s_c, _ = trm.trm_server_wait(srv, tc, m)
        lam_w, eg_w, st_w, s_w, _ = trm.trm_server_wait(srv, tw, m)
    finally:
        trm.trm_server_destroy(srv)
    assert s_a == 0 and s_c == 0 and s_w == 0
    # C_out holds the converged (orthonormal) block of the first request
    assert np.max(np.abs(CA.T @ CA - np.eye(m))) < 1e-10
    assert st_w["iterations"] < st_c["iterations"], (st_w, st_c)
    ref = op.lowest_eigenvalues(op.grid_hamiltonian(shape, order, 1.0, V2), m)
    assert np.max(np.abs(lam_w - ref)) < 1e-9
    assert np.max(np.abs(lam_c - ref)) < 1e-9
