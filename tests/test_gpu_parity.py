"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, row by row of the hot path.

Tolerance.  Both sides evaluate the same formulas in IEEE binary64; only the summation
order and the form of a few updates differ (for example x + r/d against (b - sum)/d in
Gauss-Seidel).  Each output value is the result of a few hundred such operations (two
V-cycles of about 60 flops per point per level plus the stencils), each contributing a
relative rounding error of at most 2^-53 = 1.1e-16 amplified by the operator's mild
conditioning, so operator outputs agree to about 1e-13 relative to their largest entry;
the tests ask for 1e-12.  PCG solutions are compared at 1e-10 relative, the FP64 target.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur, space, time as tm  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_OP = 1e-12
TOL_SOLVE = 1e-10

# (K, J): K = 7 spans 2 x 3 Gauss-Seidel tiles of 90 x 58 points with ragged edges
SIZES = [(1, 1), (2, 2), (3, 4), (5, 3), (7, 4)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


_probs = {}


def oracle_problem(K, J):
    if (K, J) not in _probs:
        _probs[(K, J)] = schur.Problem(K, J)
    return _probs[(K, J)]


@pytest.fixture(scope="module")
def solvers():
    cache = {}

    def get(K, J, **kw):
        key = (K, J, tuple(sorted(kw.items())))
        if key not in cache:
            cache[key] = Solver(K, J, **kw)
        return cache[key]

    yield get
    for s in cache.values():
        s.close()


@pytest.mark.parametrize("K,J", SIZES)
def test_wavelet_synthesis_and_analysis(solvers, K, J):
    p, s = oracle_problem(K, J), solvers(K, J)
    w = inputs.random_state(p.Nt, p.Nx, 11)          # wavelet rows, in-place order
    wt, ut = dev(w), torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.synthesize(wt, ut)
    u_ref = p.synth(p.from_inplace(w))
    assert rel(host(ut), u_ref) < 1e-14
    x = inputs.random_state(p.Nt, p.Nx, 12)
    out = torch.empty_like(wt)
    s.analyze(dev(x), out)
    assert rel(host(out), p.to_inplace(p.analysis(x))) < 1e-14


@pytest.mark.parametrize("K,J", SIZES)
def test_Kx_multigrid(solvers, K, J):
    p, s = oracle_problem(K, J), solvers(K, J)
    ns = 2 * p.Nt
    b = inputs.random_state(ns, p.Nx, 13)
    x = torch.empty((ns, p.Nx), dtype=torch.float64, device="cuda")
    s.apply_Kx(dev(b), x)
    ref = p.Kx.apply(b.T).T
    assert rel(host(x), ref) < TOL_OP


@pytest.mark.parametrize("K,J", SIZES)
def test_S_single_scale_both_routes(solvers, K, J):
    p, s = oracle_problem(K, J), solvers(K, J)
    u = inputs.random_state(p.Nt, p.Nx, 14)
    y = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.apply_S_nodal(dev(u), y)
    yh = host(y)
    assert rel(yh, p.apply_S_route2(u)) < TOL_OP
    assert rel(yh, p.apply_S_route1(u)) < TOL_OP


@pytest.mark.parametrize("K,J", SIZES)
def test_Shat_and_KX(solvers, K, J):
    p, s = oracle_problem(K, J), solvers(K, J)
    w = inputs.random_state(p.Nt, p.Nx, 15)
    q = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.apply_S(dev(w), q)
    ref = p.to_inplace(p.apply_Shat(p.from_inplace(w)))
    assert rel(host(q), ref) < TOL_OP
    z = torch.empty_like(q)
    s.apply_KX(dev(w), z)
    ref = p.to_inplace(p.apply_KX(p.from_inplace(w)))
    assert rel(host(z), ref) < TOL_OP


@pytest.mark.parametrize("K,J", SIZES)
def test_rhs(solvers, K, J):
    p, s = oracle_problem(K, J), solvers(K, J)
    g, u0, _ = inputs.manufactured(K, J)
    f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.rhs(dev(g), dev(u0), f)
    assert rel(host(f), p.to_inplace(p.rhs_hat(g, u0))) < TOL_OP


@pytest.mark.parametrize("K,J", [(3, 4), (5, 3), (4, 5)])
def test_pcg_solution_matches_oracle(solvers, K, J):
    # config-1 shape (K=3, J=4) and two more; oracle solved tighter than the GPU
    p = oracle_problem(K, J)
    s = solvers(K, J, tol=1e-12)
    g, u0, _ = inputs.manufactured(K, J)
    u_ref, w_ref, info = schur.solve(p, g, u0, tol=1e-13)
    f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.rhs(dev(g), dev(u0), f)
    w = torch.empty_like(f)
    its, rr = s.pcg_solve(f, w)
    assert rr <= 1e-12
    assert rel(host(w), p.to_inplace(w_ref)) < TOL_SOLVE
    u = torch.empty_like(f)
    s.synthesize(w, u)
    assert rel(host(u), u_ref) < TOL_SOLVE
    # same iteration count as the oracle at the same tolerance (rounding may shift it by one)
    _, _, info12 = schur.solve(p, g, u0, tol=1e-12)
    assert abs(its - info12["iters"]) <= 1


def test_pcg_iterates_match_oracle_step_by_step(solvers):
    # fixed iteration budgets: the k-th iterate must agree, not only the converged solution
    K, J = 3, 4
    p = oracle_problem(K, J)
    g, u0, _ = inputs.manufactured(K, J)
    fhat = p.rhs_hat(g, u0)
    for k in (1, 2, 5):
        s = solvers(K, J, tol=0.0, maxit=k)
        f = dev(p.to_inplace(fhat))
        w = torch.empty_like(f)
        with pytest.raises(Exception):
            s.pcg_solve(f, w)  # ST_ERR_MAXIT: budget exhausted before tol = 0
        w_ref, info = schur.pcg(p.apply_Shat, p.apply_KX, fhat, tol=0.0, maxit=k)
        assert info["iters"] == k
        assert rel(host(w), p.to_inplace(w_ref)) < 1e-11


def test_zero_rhs_gives_zero_solution(solvers):
    s = solvers(3, 3)
    f = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    w = torch.full_like(f, 7.0)
    its, rr = s.pcg_solve(f, w)
    assert its == 0 and torch.count_nonzero(w).item() == 0


def test_end_to_end_from_host_buffers(solvers):
    K, J = 3, 4
    p = oracle_problem(K, J)
    s = solvers(K, J, tol=1e-12)
    g, u0, _ = inputs.manufactured(K, J)
    u_ref, _, _ = schur.solve(p, g, u0, tol=1e-13)
    gt = torch.from_numpy(g).pin_memory()
    u0t = torch.from_numpy(u0).pin_memory()
    ut = torch.empty(s.shape, dtype=torch.float64).pin_memory()
    its, rr = s.solve_host(gt, u0t, ut)
    assert rel(ut.numpy(), u_ref) < TOL_SOLVE


def test_results_are_bitwise_reproducible(solvers):
    s = solvers(5, 4)
    w = dev(inputs.random_state(s.Nt, s.Nx, 21))
    q1, q2 = torch.empty_like(w), torch.empty_like(w)
    s.apply_S(w, q1)
    s.apply_S(w, q2)
    z1, z2 = torch.empty_like(w), torch.empty_like(w)
    s.apply_KX(w, z1)
    s.apply_KX(w, z2)
    torch.cuda.synchronize()
    assert torch.equal(q1, q2) and torch.equal(z1, z2)


def test_operators_symmetric_positive_at_full_size(solvers):
    # K = 9, J = 9 (N = 1.34e8, the benchmark's size): <S x, y> = <x, S y>, <S x, x> > 0,
    # and the same for K_X, on random vectors (properties that hold at any size)
    s = solvers(9, 9)
    x = dev(inputs.random_state(s.Nt, s.Nx, 31))
    y = dev(inputs.random_state(s.Nt, s.Nx, 32))
    for op in (s.apply_S, s.apply_KX):
        ox, oy = torch.empty_like(x), torch.empty_like(x)
        op(x, ox)
        op(y, oy)
        a = torch.dot(ox.view(-1), y.view(-1)).item()
        b = torch.dot(x.view(-1), oy.view(-1)).item()
        assert abs(a - b) <= 1e-11 * abs(a)
        assert torch.dot(ox.view(-1), x.view(-1)).item() > 0


def test_full_size_sampled_rows_match_oracle(solvers):
    # K = 9, J = 9: rows of S u (row i needs rows i-1..i+1 of u) and of K_X r (row-local)
    # recomputed by the oracle one by one
    K, J = 9, 9
    s = solvers(K, J)
    Nt, Nx = s.Nt, s.Nx
    u = inputs.random_state(Nt, Nx, 41)
    y = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.apply_S_nodal(dev(u), y)
    yh = host(y)
    mesh = space.Mesh(K)
    M, A = space.mass_matrix(mesh), space.stiffness_matrix(mesh)
    Kx = space.Multigrid(K, space.SQUARE, 1.0, 0.0)
    t = tm.time_matrices(J)
    for i in (0, 1, 257, Nt - 1):
        lo, hi = max(i - 1, 0), min(i + 2, Nt)
        UM = (M @ u[lo:hi].T).T
        UA = (A @ u[lo:hi].T).T
        y1 = t["At"][i, lo:hi] @ UM + t["L"].T[i, lo:hi] @ UA
        y2 = t["L"][i, lo:hi] @ UM + t["Mt"][i, lo:hi] @ UA
        row = M @ Kx.apply(y1) + A @ Kx.apply(y2)
        if i == 0:
            row = row + M @ u[0]
        assert rel(yh[i], row) < TOL_OP, i
    r = inputs.random_state(Nt, Nx, 42)
    z = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.apply_KX(dev(r), z)
    zh = host(z)
    for i in (0, 256, 1, Nt - 1):
        lev = 0 if i in (0, Nt - 1) else J - ((i & -i).bit_length() - 1)
        Kl = space.Multigrid(K, space.SQUARE, 0.3, 2.0 ** lev)
        ref = Kl.apply(A @ Kl.apply(r[i]))
        assert rel(zh[i], ref) < TOL_OP, i
    # the benchmark's launch configuration (autotuned kernels and segment lengths) gives bitwise
    # the same operators
    s.autotune()
    y2, z2 = torch.empty_like(y), torch.empty_like(z)
    s.apply_S_nodal(dev(u), y2)
    s.apply_KX(dev(r), z2)
    torch.cuda.synchronize()
    assert torch.equal(y, y2) and torch.equal(z, z2)
    s.set_smoother("tiles")


def _table_5_3():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "table_5_3_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                rows.append((int(a), int(b)))
    return rows


@pytest.mark.parametrize("J", [3, 4, 5, 6])
def test_iteration_counts_match_oracle(J):
    # the paper's stopping rule (Eq. 3.3, eps = 1e-6 absolute) on its 2D workload
    # u = exp(-2 pi^2 t) sin sin, g = 0: the GPU takes as many PCG steps as the oracle
    K = 5
    g, u0, _ = inputs.decaying(K, J)
    p = oracle_problem(K, J)
    _, _, info = schur.solve(p, g, u0, tol=1e-6, tol_mode="abs")
    with Solver(K, J, tol=1e-6, tol_mode=1) as s:
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(dev(g), dev(u0), f)
        w = torch.empty_like(f)
        n, _ = s.pcg_solve(f, w)
    assert abs(n - info["iters"]) <= 1, (J, n, info["iters"])


def _table_5_3_oracle():
    """N_t -> the oracle's multigrid iteration count at K = 9 (tests/golden/table_5_3_oracle.txt,
    written by make_table_5_3_oracle.py from oracle/ only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table_5_3_oracle.txt")
    out = {}
    if os.path.exists(path):
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                out[int(f[0])] = int(f[1])
    return out


@pytest.mark.parametrize("Nt,its", _table_5_3())
def test_table_5_3_iteration_counts(Nt, its):
    # Sec. 5.2, Table 5.3: eps = 1e-6 absolute (Eq. 3.3), u = exp(-2 pi^2 t) sin sin, g = 0, K = 9.
    # Where the oracle's count at K = 9 is stored, the GPU must take it within one iteration (the
    # two differ only in rounding).  Against the paper: with direct inverses the oracle takes the
    # printed counts at N_t = 9 and 17 and one more from N_t = 33 on (test_oracle_schur); with this
    # project's multigrid reading (2 V-cycles of 3 + 3 three-colour sweeps, Sec. 5.1; the paper
    # does not define its smoother) the oracle and the GPU take 3 to 5 more than printed (13, 14
    # at N_t = 9, 17 against 8, 11): the multigrid's error of about 1e-3 spreads the smooth
    # solution over other modes that the absolute 1e-6 rule must then resolve.  Lexicographic,
    # hierarchical (coarse nodes first) and W-cycle smoothers of the same cost change the count by
    # at most one, so the paper's multigrid is closer to an exact solve than its stated settings
    # give; the bound below records that gap.
    K = 9
    J = int(np.log2(Nt - 1))
    g, u0, _ = inputs.decaying(K, J)
    with Solver(K, J, tol=1e-6, tol_mode=1) as s:
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(dev(g), dev(u0), f)
        w = torch.empty_like(f)
        n, _ = s.pcg_solve(f, w)
    oracle = _table_5_3_oracle().get(Nt)
    if oracle is not None:
        assert abs(n - oracle) <= 1, (Nt, n, oracle)
    assert its <= n <= its + 5, (Nt, n, its)
