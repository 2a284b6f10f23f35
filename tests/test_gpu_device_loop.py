"""The device-driven PCG loop (st_config.use_graphs = 2) against the host-driven one.

With use_graphs = 2 a solve is one CUDA graph whose WHILE node repeats the iteration body, and
a stop-test kernel takes the per-problem decisions of Sec. 3.4 (Eq. 3.3) on the device.  The
kernels and their order are those of the host-driven loop (use_graphs = 1: the host reads the
scalars back and tests after every iteration), so solutions, iteration counts, refinement steps
and statuses must be bitwise the same, for every precision, for batches whose problems stop at
different iterations, at maxit, and for a zero right-hand side.  st_batch_run with use_graphs = 2
runs all shape groups as branches of one graph and must give what it gives with host threads.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_08875_gb300 import Batch, Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _forcing(K, J, B, seed, domain=0):
    gs, us = [], []
    for b in range(B):
        g, u0 = inputs.smooth_forcing(K, J, seed=seed + b, domain=domain)
        # problems of different sizes stop at different iterations
        gs.append(inputs.to_grid(K, domain, g) * (10.0 ** b))
        us.append(inputs.to_grid(K, domain, u0))
    return np.stack(gs), np.stack(us)


def _solve(K, J, B, g, u0, domain=0, **cfg):
    # graphs run only on a stream other than the legacy default stream
    with torch.cuda.stream(torch.cuda.Stream()):
        return _solve_on_stream(K, J, B, g, u0, domain, **cfg)


def _solve_on_stream(K, J, B, g, u0, domain=0, **cfg):
    with Solver(K, J, domain=domain, batch=B, **cfg) as s:
        gd = torch.from_numpy(np.ascontiguousarray(g)).cuda().reshape(s.shape)
        ud = torch.from_numpy(np.ascontiguousarray(u0)).cuda().reshape(s.u0_shape)
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(gd, ud, f)
        w = torch.empty_like(f)
        st = _status_of(s, f, w)
        torch.cuda.synchronize()
        infos = [s.problem_info(b) for b in range(B)]
        return st, w.cpu(), infos


def _status_of(s, f, w):
    from paper_2009_08875_gb300 import _lib
    try:
        s.pcg_solve(f, w)
        return _lib.ST_OK
    except _lib.STError as e:
        return e.status


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_precond", "mixed_bf16", "fp64_df"])
@pytest.mark.parametrize("K,J,B,domain", [(4, 3, 1, 0), (5, 4, 3, 0), (5, 3, 2, 1)])
def test_device_loop_equals_host_loop_bitwise(precision, K, J, B, domain):
    g, u0 = _forcing(K, J, B, seed=11 * K + J, domain=domain)
    a = _solve(K, J, B, g, u0, domain, precision=precision, use_graphs=1)
    d = _solve(K, J, B, g, u0, domain, precision=precision, use_graphs=2)
    assert a[0] == d[0]
    assert a[2] == d[2]
    assert torch.equal(a[1], d[1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_loop_maxit_and_zero_problem(precision):
    K, J, B = 4, 3, 3
    g, u0 = _forcing(K, J, B, seed=5)
    g[1] = 0.0
    u0[1] = 0.0  # problem 1: zero right-hand side, never iterates
    for mx in (3, 200):
        a = _solve(K, J, B, g, u0, precision=precision, maxit=mx, use_graphs=1)
        d = _solve(K, J, B, g, u0, precision=precision, maxit=mx, use_graphs=2)
        assert a[0] == d[0], mx
        assert a[2] == d[2], mx
        assert torch.equal(a[1], d[1]), mx
        assert d[2][1]["iterations"] == 0
    assert a[0] == 0 and d[0] == 0


def test_device_loop_reuses_its_graph_and_follows_new_vectors():
    K, J = 4, 3
    g, u0 = _forcing(K, J, 1, seed=3)
    with torch.cuda.stream(torch.cuda.Stream()), Solver(K, J) as s:
        gd = torch.from_numpy(g[0]).cuda()
        ud = torch.from_numpy(u0[0]).cuda()
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(gd, ud, f)
        w1, w2, w3 = (torch.empty_like(f) for _ in range(3))
        n1, _ = s.pcg_solve(f, w1)
        n2, _ = s.pcg_solve(f, w2)      # a new solution vector: the graph is captured again
        n3, _ = s.pcg_solve(f, w2)      # the same vectors: the graph is replayed
        s.pcg_solve(2.0 * f, w3)        # a new right-hand side
        torch.cuda.synchronize()
    assert n1 == n2 == n3
    assert torch.equal(w1, w2)
    assert torch.allclose(w3, 2.0 * w1, rtol=1e-9, atol=0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_precond"])
def test_batch_graph_equals_batch_threads(precision):
    rng = np.random.default_rng(4)
    shapes = [(0, 4, 3), (0, 4, 3), (1, 5, 4), (0, 5, 2), (2, 3, 3), (0, 4, 3)]
    probs = []
    for i, (dom, K, J) in enumerate(shapes):
        g, u0 = inputs.smooth_forcing(K, J, seed=int(rng.integers(1 << 20)), domain=dom)
        probs.append((dom, K, J, torch.from_numpy(inputs.to_grid(K, dom, g)).pin_memory(),
                      torch.from_numpy(inputs.to_grid(K, dom, u0)).pin_memory()))
    outs = {}
    for mode in (1, 2):
        bt = Batch(precision=precision, use_graphs=mode)
        us = []
        for dom, K, J, g, u0 in probs:
            u = torch.full(g.shape, float("nan"), dtype=torch.float64).pin_memory()
            bt.add(dom, K, J, g, u0, u)
            us.append(u)
        st = bt.run()
        outs[mode] = (st, us, [bt.info(i) for i in range(len(probs))])
        bt.close()
    assert outs[1][0] == outs[2][0] == 0
    assert outs[1][2] == outs[2][2]
    for a, b in zip(outs[1][1], outs[2][1]):
        assert torch.equal(a, b)
