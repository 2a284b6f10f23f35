"""Batched handles: B problems of one shape solved in lock step, each with its own scalars.

A problem must give the same bits alone and inside a batch (all kernels act per problem, the
inner-product partition depends only on the problem size, and a finished problem is frozen by
zero step lengths while the others go on).  The ST_MIXED_PRECOND mode (binary64 PCG with a
binary32 preconditioner) must reach the 1e-8 target against the binary64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def forcings(K, J, B, domain=0):
    gs, u0s = [], []
    for b in range(B):
        g, u0 = inputs.smooth_forcing(K, J, seed=100 + b, domain=domain)
        if b % 2 == 1:  # mix in nonzero initial data
            u0 = inputs.manufactured(K, J, domain)[1]
        gs.append(inputs.to_grid(K, domain, g))
        u0s.append(inputs.to_grid(K, domain, u0))
    return np.stack(gs), np.stack(u0s)


def solve(K, J, g, u0, B, precision, domain=0, tol=1e-10):
    with Solver(K, J, domain=domain, batch=B, precision=precision, tol=tol) as s:
        gd = torch.from_numpy(g.reshape(s.shape)).cuda()
        u0d = torch.from_numpy(u0.reshape(s.u0_shape)).cuda()
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(gd, u0d, f)
        w = torch.empty_like(f)
        s.pcg_solve(f, w)
        u = torch.empty_like(f)
        s.synthesize(w, u)
        torch.cuda.synchronize()
        infos = [s.problem_info(b) for b in range(B)]
        return u.cpu().numpy().reshape(B, s.Nt, s.Nx), infos


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_precond"])
def test_batch_equals_alone_bitwise(precision):
    K, J, B = 5, 4, 5
    g, u0 = forcings(K, J, B)
    ub, infos = solve(K, J, g, u0, B, precision)
    for b in (0, 3):
        ua, info_a = solve(K, J, g[b:b + 1], u0[b:b + 1], 1, precision)
        assert np.array_equal(ub[b], ua[0]), (precision, b)
        assert infos[b]["iterations"] == info_a[0]["iterations"]
        assert infos[b]["outer_iterations"] == info_a[0]["outer_iterations"]
    assert all(i["status"] == 0 and i["relres"] <= 1e-10 for i in infos)


def test_batch_problems_match_oracle_lshape():
    K, J, B = 4, 3, 3
    g, u0 = forcings(K, J, B, domain=1)
    ub, _ = solve(K, J, g, u0, B, "fp64", domain=1, tol=1e-12)
    p = schur.Problem(K, J, 1)
    for b in range(B):
        u_ref, _, _ = schur.solve(p, inputs.from_grid(K, 1, g[b]), inputs.from_grid(K, 1, u0[b]), tol=1e-13)
        out = inputs.from_grid(K, 1, ub[b])
        assert np.abs(out - u_ref).max() <= 1e-10 * np.abs(u_ref).max()


def test_mixed_precond_meets_fp64_target():
    K, J = 6, 5
    g, u0 = forcings(K, J, 1)
    u64, i64 = solve(K, J, g, u0, 1, "fp64")
    upc, ipc = solve(K, J, g, u0, 1, "mixed_precond")
    err = np.abs(upc - u64).max() / np.abs(u64).max()
    assert err < 1e-8, err
    # a binary32 preconditioner costs at most a few extra iterations of the flexible PCG
    assert ipc[0]["iterations"] <= i64[0]["iterations"] + 3


def test_batched_operators_equal_single():
    K, J, B = 5, 3, 4
    rng = np.random.default_rng(5)
    with Solver(K, J, batch=B) as s, Solver(K, J) as s1:
        x = torch.from_numpy(rng.standard_normal(s.shape)).cuda()
        for op_b, op_1 in ((s.apply_S, s1.apply_S), (s.apply_KX, s1.apply_KX), (s.synthesize, s1.synthesize),
                           (s.analyze, s1.analyze), (s.apply_S_nodal, s1.apply_S_nodal)):
            yb = torch.empty_like(x)
            op_b(x, yb)
            for b in range(B):
                y1 = torch.empty_like(x[b])
                op_1(x[b].contiguous(), y1)
                torch.cuda.synchronize()
                assert torch.equal(yb[b], y1)


@pytest.mark.parametrize("precision", ["fp64", "mixed_precond"])
def test_multi_shape_runner_equals_alone(precision):
    from paper_2009_08875_gb300 import Batch
    rng = np.random.default_rng(7)
    shapes = [(0, 4, 3), (0, 5, 4), (1, 4, 3), (0, 4, 3), (0, 5, 4), (1, 5, 3), (0, 4, 3), (2, 3, 3), (2, 3, 3)]
    bt = Batch(precision=precision, tol=1e-10)
    probs = []
    for i, (dom, K, J) in enumerate(shapes):
        g, u0 = inputs.smooth_forcing(K, J, seed=int(rng.integers(1 << 30)), domain=dom)
        g = torch.from_numpy(inputs.to_grid(K, dom, g)).pin_memory()
        u0 = torch.from_numpy(inputs.to_grid(K, dom, inputs.manufactured(K, J, dom)[1])).pin_memory()
        u = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
        assert bt.add(dom, K, J, g, u0, u) == i
        probs.append((dom, K, J, g, u0, u))
    assert bt.run() == 0
    assert bt.buckets() == 5
    for i, (dom, K, J, g, u0, u) in enumerate(probs):
        with Solver(K, J, domain=dom, precision=precision, tol=1e-10) as s:
            ua = torch.zeros_like(u)
            its, _ = s.solve_host(g, u0, ua)
        assert torch.equal(u, ua), i
        assert bt.info(i)["iterations"] == its
    bt.close()


def test_empty_batch_and_rejected_shapes():
    # a batch without problems runs no bucket; shapes outside the accepted levels (the cube above
    # K = 8, the L-shape at K = 1, domain 3, K = 13, J = 15, J = 0) are rejected before any copy
    from paper_2009_08875_gb300 import Batch, _lib
    bt = Batch(precision="fp64")
    assert bt.run() == _lib.ST_OK and bt.buckets() == 0
    buf = torch.zeros(4, dtype=torch.float64)
    p = buf.data_ptr()
    lib = _lib.load()
    for dom, K, J in ((2, 9, 3), (1, 1, 3), (3, 4, 3), (0, 13, 3), (0, 4, 15), (0, 4, 0)):
        assert lib.st_batch_add(bt._h, dom, K, J, p, p, p, None) == _lib.ST_ERR_ARG, (dom, K, J)
    assert bt.run() == _lib.ST_OK and bt.buckets() == 0
    bt.close()
