"""The 3D problem (Sec. 5.2: the unit cube, P1 on Kuhn tetrahedra) on the GPU against the oracle.

Tolerances as in test_gpu_parity: operators 1e-12 of their largest entry (the same binary64
formulas, summation order and the Jacobi-scaled Gauss-Seidel form differ), solutions 1e-10,
mixed-precision solutions 1e-8.  K = 4 has 15^3 points per slice, K = 1 the single-unknown
degenerate case.  The paper's 3D weak-scaling runs (Table 5.5, N_x = 250047, eps = 1e-6,
u = exp(-3 pi^2 t) sin sin sin, tests/golden/table_5_5_iterations.txt) give the iteration counts
checked at the end, within one iteration.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur, space  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CUBE = space.CUBE
TOL_OP = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("c", [0.0, 3.0])
@pytest.mark.parametrize("K,J", [(1, 1), (2, 2), (3, 3), (4, 2)])
def test_cube_operators(K, J, c):
    p = schur.Problem(K, J, CUBE, c=c)
    with Solver(K, J, domain=CUBE, c=c) as s:
        assert s.shape == (p.Nt, p.Nx)
        b = inputs.random_state(2 * p.Nt, p.Nx, 91)
        x = torch.empty((2 * p.Nt, p.Nx), dtype=torch.float64, device="cuda")
        s.apply_Kx(dev(b), x)
        assert rel(host(x), p.Kx.apply(b.T).T) < TOL_OP
        u = inputs.random_state(p.Nt, p.Nx, 92)
        y = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.apply_S_nodal(dev(u), y)
        assert rel(host(y), p.apply_S_route1(u)) < TOL_OP
        w = inputs.random_state(p.Nt, p.Nx, 93)
        s.apply_S(dev(w), y)
        assert rel(host(y), p.to_inplace(p.apply_Shat(p.from_inplace(w)))) < TOL_OP
        s.apply_KX(dev(w), y)
        assert rel(host(y), p.to_inplace(p.apply_KX(p.from_inplace(w)))) < TOL_OP
        g, u0, _ = inputs.manufactured(K, J, CUBE, c=c)
        s.rhs(dev(g), dev(u0), y)
        assert rel(host(y), p.to_inplace(p.rhs_hat(g, u0))) < TOL_OP


@pytest.mark.parametrize("K,J", [(2, 2), (4, 2)])
def test_cube_double_float_operators(K, J):
    # ST_FP64_DF: the cube's multigrid in double-float (about 2^-48 per operation); the tolerance
    # is 32 times the binary64 one (2^5 = 2^-48 / 2^-53), as for the square
    p = schur.Problem(K, J, CUBE)
    with Solver(K, J, domain=CUBE, precision="fp64_df") as s:
        b = inputs.random_state(2 * p.Nt, p.Nx, 94)
        x = torch.empty((2 * p.Nt, p.Nx), dtype=torch.float64, device="cuda")
        s.apply_Kx(dev(b), x)
        assert rel(host(x), p.Kx.apply(b.T).T) < 32 * TOL_OP
        w = inputs.random_state(p.Nt, p.Nx, 95)
        y = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.apply_KX(dev(w), y)
        assert rel(host(y), p.to_inplace(p.apply_KX(p.from_inplace(w)))) < 32 * TOL_OP
        s.apply_S(dev(w), y)
        assert rel(host(y), p.to_inplace(p.apply_Shat(p.from_inplace(w)))) < 32 * TOL_OP


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp64_df", 1e-10), ("mixed", 1e-8),
                                           ("mixed_precond", 1e-8)])
def test_cube_solve(precision, tol):
    K, J = 3, 3
    p = schur.Problem(K, J, CUBE)
    g, u0, _ = inputs.manufactured(K, J, CUBE)
    u_ref, _, _ = schur.solve(p, g, u0, tol=1e-13)
    with Solver(K, J, domain=CUBE, tol=1e-11, precision=precision) as s:
        u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), u)
    assert rel(u.numpy(), u_ref) < tol


def test_cube_iterations_equal_oracle_at_the_papers_rule():
    K, J = 3, 4
    p = schur.Problem(K, J, CUBE)
    g, u0, _ = inputs.decaying(K, J, CUBE)
    _, _, info = schur.solve(p, g, u0, tol=1e-6, tol_mode="abs")
    with Solver(K, J, domain=CUBE, tol=1e-6, tol_mode=1) as s:
        u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        its, _ = s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), u)
    assert its == info["iters"]


def test_cube_nested_matches_oracle():
    K, J, levels, eps = 3, 3, 2, 1e-4
    g, u0, _ = inputs.manufactured(K, J, CUBE)
    _, w_ref, its_ref = schur.nested_solve(K, J, levels, g, u0, eps, domain=CUBE)
    p = schur.Problem(K, J, CUBE)
    with Solver(K, J, domain=CUBE) as s:
        w = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        st, its = s.nested_solve(levels, eps, dev(g), dev(u0), w)
        torch.cuda.synchronize()
    assert st == 0 and its == its_ref
    assert rel(w.cpu().numpy(), p.to_inplace(w_ref)) < 1e-10


def _table_5_5():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "table_5_5_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                rows.append((int(a), int(b)))
    return rows


# Table 5.5 (3D weak scaling) at N_x = 250047 (K = 6), the rows up to N_t = 513: the count must
# be the paper's within one iteration (the paper's smoother ordering is not stated; measured:
# 15, 16, 16, the paper's counts)
@pytest.mark.parametrize("Nt,paper_its", [r for r in _table_5_5() if r[0] <= 513])
def test_cube_table_5_5_iterations(Nt, paper_its):
    K = 6
    J = Nt.bit_length() - 1
    assert 2 ** J + 1 == Nt
    g, u0, _ = inputs.decaying(K, J, CUBE)
    with Solver(K, J, domain=CUBE, tol=1e-6, tol_mode=1, maxit=100) as s:
        u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        its, _ = s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), u)
    assert abs(its - paper_its) <= 1, its
