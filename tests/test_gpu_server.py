"""Continuous-batching server: results equal solving each request alone, with joins and leaves
at iteration boundaries while other requests run, and admission by a device-memory budget."""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_08875_gb300 import Server, Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def make_request(dom, K, J, seed):
    g, _ = inputs.smooth_forcing(K, J, seed=seed, domain=dom)
    u0 = inputs.manufactured(K, J, dom)[1] if seed % 2 else np.zeros_like(g[0])
    g = torch.from_numpy(inputs.to_grid(K, dom, g)).pin_memory()
    u0 = torch.from_numpy(inputs.to_grid(K, dom, u0)).pin_memory()
    return dom, K, J, g, u0, torch.zeros(g.shape, dtype=torch.float64).pin_memory()


def alone(dom, K, J, g, u0, precision):
    with Solver(K, J, domain=dom, precision=precision, tol=1e-10) as s:
        u = torch.zeros_like(g)
        its, _ = s.solve_host(g, u0, u)
    return u, its


def wait_all(srv, tickets, timeout=120):
    t0 = time.time()
    out = {}
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                st = srv.poll(t)
                if st["state"] >= Server.DONE:
                    out[t] = st
        assert time.time() - t0 < timeout
        time.sleep(0.002)
    return out


@pytest.mark.parametrize("precision", ["mixed_precond", "fp64"])
def test_server_results_equal_alone(precision):
    shapes = [(0, 4, 3), (0, 5, 4), (1, 4, 4), (0, 4, 3), (2, 3, 3), (0, 5, 4), (0, 4, 3), (1, 4, 4), (0, 6, 3),
              (2, 3, 3)]
    reqs = [make_request(d, K, J, 10 + i) for i, (d, K, J) in enumerate(shapes)]
    srv = Server(slots_per_group=2, memory_budget_gb=40.0, precision=precision, tol=1e-10)
    tickets = []

    def producer():  # staggered arrivals: later requests join groups that are already iterating
        for r in reqs:
            tickets.append(srv.submit(*r))
            time.sleep(0.003)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    res = wait_all(srv, tickets)
    srv.stop()
    for t, r in zip(tickets, reqs):
        assert res[t]["state"] == Server.DONE and res[t]["latency_s"] > 0
        ua, its = alone(*r[:5], precision)
        assert torch.equal(r[5], ua), t
        assert res[t]["iterations"] == its


def test_server_budget_admits_one_group_at_a_time():
    shapes = [(0, 5, 4), (0, 4, 5), (0, 5, 4), (1, 5, 3)]
    reqs = [make_request(d, K, J, 30 + i) for i, (d, K, J) in enumerate(shapes)]
    # a one-slot group of these shapes is budgeted at about 0.07 GB: 0.1 GB holds one at a time,
    # so idle groups are released to admit the next shape
    srv = Server(slots_per_group=1, memory_budget_gb=0.1, tol=1e-10)
    tickets = [srv.submit(*r) for r in reqs]
    res = wait_all(srv, tickets)
    srv.stop()
    for t, r in zip(tickets, reqs):
        assert res[t]["state"] == Server.DONE
        ua, _ = alone(*r[:5], "mixed_precond")
        assert torch.equal(r[5], ua)


def test_server_rejects_a_request_larger_than_the_budget():
    srv = Server(slots_per_group=1, memory_budget_gb=0.05, tol=1e-10)
    r = make_request(0, 7, 5, 3)
    t = srv.submit(*r)
    res = wait_all(srv, [t])
    srv.stop()
    assert res[t]["state"] == Server.FAILED


def test_cancel_and_deadline():
    from paper_2009_08875_gb300 import _lib
    # one group slot and large problems, so that later requests wait in the queue
    big = [make_request(0, 7, 7, 60 + i) for i in range(4)]
    srv = Server(slots_per_group=1, memory_budget_gb=40.0, tol=1e-10)
    t_run = srv.submit(*big[0])
    t_queued = srv.submit(*big[1])
    t_late = srv.submit(*big[2], timeout=1e-6)          # past its deadline before it can start
    srv.cancel(t_queued)
    # cancel the first request once it runs
    t0 = time.time()
    while srv.poll(t_run)["state"] == Server.QUEUED:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    srv.cancel(t_run)
    t_ok = srv.submit(*big[3], timeout=600.0)           # generous deadline: completes
    res = wait_all(srv, [t_run, t_queued, t_late, t_ok])
    srv.stop()
    assert res[t_queued]["state"] == Server.FAILED and res[t_queued]["status"] == _lib.ST_ERR_CANCELLED
    assert res[t_late]["state"] == Server.FAILED and res[t_late]["status"] == _lib.ST_ERR_TIMEOUT
    # the running request leaves at an iteration boundary (or had already finished)
    assert res[t_run]["status"] in (_lib.ST_ERR_CANCELLED, _lib.ST_OK)
    assert res[t_ok]["state"] == Server.DONE and res[t_ok]["status"] == _lib.ST_OK
    u_alone, its = alone(*big[3][:5], "mixed_precond")
    assert torch.equal(big[3][5], u_alone) and res[t_ok]["iterations"] == its


def test_server_rejects_bad_requests_and_stops_empty():
    # invalid shapes and a NaN timeout are rejected at submission; unknown tickets at poll and
    # cancel; a server that never got a request stops cleanly
    import ctypes

    from paper_2009_08875_gb300 import _lib
    lib = _lib.load()
    srv = Server(slots_per_group=1, memory_budget_gb=1.0, tol=1e-10)
    buf = torch.zeros(4, dtype=torch.float64)
    p = buf.data_ptr()
    t = ctypes.c_int64(-1)
    for dom, K, J in ((2, 9, 3), (1, 1, 3), (3, 4, 3), (0, 13, 3), (0, 4, 15), (0, 4, 0)):
        assert lib.st_server_submit_deadline(srv._h, dom, K, J, p, p, p, 0.0, ctypes.byref(t)) == _lib.ST_ERR_ARG
    assert lib.st_server_submit_deadline(srv._h, 0, 4, 3, p, p, p, float("nan"), ctypes.byref(t)) == _lib.ST_ERR_ARG
    assert t.value == -1
    state = ctypes.c_int()
    assert lib.st_server_poll(srv._h, 0, ctypes.byref(state), None, None, None) == _lib.ST_ERR_ARG
    assert lib.st_server_cancel(srv._h, 5) == _lib.ST_ERR_ARG
    srv.stop()
