"""GPU tests of the serving loop (lqcd_serve_*).

Continuous batching: requests of mixed lattice sizes, kappa and precision
arrive while others run, are admitted as slots and HBM budget allow, run
concurrently on per-slot streams and retire independently.  Each served
C(t) must equal the same request solved alone (lqcd_pion_corr) and the FP64
oracle within 1e-8 relative; admission by HBM budget, polling time-outs,
unknown tickets and shutdown with pending work are checked too.
"""
import numpy as np
import pytest

import oracle
from paper_2503_16994_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_16994_gb300 import lqcd
    return lqcd


FIELDS = {
    "a": ((4, 4, 4, 4), 0.3, 1),
    "b": ((6, 6, 6, 8), 0.3, 2),
    "c": ((8, 8, 8, 8), 0.2, 3),
}


def test_served_results_equal_alone_and_oracle(lq):
    U = {k: inputs.gauge_field(d, e, seed=s) for k, (d, e, s) in FIELDS.items()}
    srv = lq.serve_create(device=0, hbm_budget_bytes=0, max_slots=3)
    try:
        gid = {k: lq.serve_gauge(srv, FIELDS[k][0], U[k]) for k in FIELDS}
        plan = [("a", 0.120, 1.0, (0, 0, 0, 0), "fp16"), ("b", 0.125, 1.3, (1, 2, 3, 5), "fp32"),
                ("c", 0.118, 1.5, (3, 0, 7, 2), "fp16"), ("a", 0.125, 1.7, (1, 1, 0, 3), "fp64"),
                ("b", 0.122, 1.0, (0, 5, 2, 7), "fp16"), ("c", 0.121, 1.2, (0, 0, 0, 0), "fp32"),
                ("a", 0.110, 0.0, (3, 3, 3, 3), "fp16"), ("b", 0.126, 1.5, (2, 2, 2, 2), "fp16")]
        tickets = [lq.serve_submit(srv, gid[k], lq.dirac_params(kap, c),
                                   lq.solver_params(tol=1e-10, maxiter=5000, precision=p), src)
                   for k, kap, c, src, p in plan]
        assert len(set(tickets)) == len(tickets)
        stamps = []
        for t, (k, kap, c, src, p) in zip(tickets, plan):
            dims = FIELDS[k][0]
            rc, corr, infos, ts = lq.serve_poll(srv, t, dims[3], timeout_ms=-1)
            assert rc == lq.OK, infos
            assert ts[0] <= ts[1] <= ts[2] <= ts[3]
            stamps.append(ts)
            assert all(i["true_resid"] <= 1e-10 for i in infos)
            ref, *_ = oracle.pion(dims, U[k], kap, c, src, tol=1e-13)
            assert np.all(np.abs(corr - ref) <= 1e-8 * np.abs(ref)), (k, p)
            # the same request alone through the lattice API
            lat = lq.lattice_create(dims)
            try:
                g = lq.gauge_upload(lat, U[k])
                alone, _, _, rc2 = lq.pion_corr(lat, g, lq.dirac_params(kap, c),
                                                lq.solver_params(tol=1e-10, maxiter=5000, precision=p), src, dims=dims)
            finally:
                lq.lattice_destroy(lat)
            assert rc2 == lq.OK
            assert np.all(np.abs(corr - alone) <= 1e-8 * np.abs(alone))
            with pytest.raises(lq.LqcdError) as e:  # polled tickets are forgotten
                lq.serve_poll(srv, t, dims[3], timeout_ms=0)
            assert e.value.code == lq.ENOTFOUND
    finally:
        lq.serve_destroy(srv)
    # continuous batching, from the timestamps {arrive, admit, start, finish}:
    # requests ran at the same time, and a slot freed by a retired request
    # took a queued one while another request was still running
    n = len(stamps)
    assert any(stamps[i][2] < stamps[j][3] and stamps[j][2] < stamps[i][3]
               for i in range(n) for j in range(i + 1, n)), stamps
    assert any(stamps[j][3] <= stamps[i][1] and stamps[k][2] < stamps[i][1] < stamps[k][3]
               for i in range(n) for j in range(n) for k in range(n) if len({i, j, k}) == 3), stamps


def test_admission_by_hbm_budget(lq):
    dims = (8, 8, 8, 8)
    U = inputs.gauge_field(dims, 0.2, seed=4)
    # too small for the gauge field itself
    srv = lq.serve_create(device=0, hbm_budget_bytes=1 << 20, max_slots=1)
    try:
        with pytest.raises(lq.LqcdError) as e:
            lq.serve_gauge(srv, dims, U)
        assert e.value.code == lq.ENOMEM
    finally:
        lq.serve_destroy(srv)
    # room for the field but not for a request's workspace
    srv = lq.serve_create(device=0, hbm_budget_bytes=12 << 20, max_slots=1)
    try:
        g = lq.serve_gauge(srv, dims, U)
        with pytest.raises(lq.LqcdError) as e:
            lq.serve_submit(srv, g, lq.dirac_params(0.12, 1.0), lq.solver_params(precision="fp64"), (0, 0, 0, 0))
        assert e.value.code == lq.ENOMEM and "budget" in str(e.value)
    finally:
        lq.serve_destroy(srv)


def test_poll_busy_timeout_unknown_and_shutdown(lq):
    dims = (16, 16, 16, 16)
    U = inputs.gauge_field(dims, 0.4, seed=6)
    srv = lq.serve_create(device=0, hbm_budget_bytes=0, max_slots=1)
    try:
        g = lq.serve_gauge(srv, dims, U)
        sp = lq.solver_params(tol=1e-10, maxiter=20000, precision="fp64")
        t1 = lq.serve_submit(srv, g, lq.dirac_params(0.130, 1.5), sp, (0, 0, 0, 0))
        t2 = lq.serve_submit(srv, g, lq.dirac_params(0.129, 1.5), sp, (1, 0, 0, 0))
        # one slot: the second request waits behind the first, which takes seconds in FP64
        rc, *_ = lq.serve_poll(srv, t2, 16, timeout_ms=0)
        assert rc == lq.EBUSY
        rc, *_ = lq.serve_poll(srv, t2, 16, timeout_ms=20)
        assert rc == lq.ETIMEOUT
        with pytest.raises(lq.LqcdError) as e:
            lq.serve_poll(srv, 987654321, 16, timeout_ms=0)
        assert e.value.code == lq.ENOTFOUND
        rc, corr, infos, ts = lq.serve_poll(srv, t1, 16, timeout_ms=-1)
        assert rc == lq.OK and np.all(corr > 0)
        # queue more work and stop the server while it runs: destroy must return,
        # and a poll already waiting on a queued request must return too
        import threading
        queued = [lq.serve_submit(srv, g, lq.dirac_params(0.128, 1.5), sp, (k, 1, 0, 0)) for k in range(3)]
        got, entering = [], threading.Event()

        def wait_for_last():
            entering.set()
            got.append(lq.serve_poll(srv, queued[-1], 16, timeout_ms=-1)[0])

        waiter = threading.Thread(target=wait_for_last)
        waiter.start()
        assert entering.wait(timeout=10)
        rc, *_ = lq.serve_poll(srv, queued[-1], 16, timeout_ms=500)  # the waiter is inside its poll by now
        assert rc == lq.ETIMEOUT  # still queued behind the running requests
    finally:
        lq.serve_destroy(srv)
    waiter.join(timeout=60)
    assert not waiter.is_alive()
    assert got == [lq.ETIMEOUT]
