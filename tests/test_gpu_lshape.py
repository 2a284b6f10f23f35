"""The L-shape (0,1)^2 minus [1/2,1)^2 on the GPU against the oracle (which assembles it by elements).

The library stores the L-shape on the square's (2^K - 1)^2 grid with zeros at the nodes outside
the domain; the oracle numbers only the domain nodes.  Inputs are placed on the grid with
inputs.to_grid and outputs are compared at the domain nodes, and must be exactly zero elsewhere.
Tolerances as in test_gpu_parity (binary64) and test_gpu_mixed (binary32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur, space  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

L = space.LSHAPE
TOL_OP = 1e-12
TOL_SOLVE = 1e-10


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def check(K, out_grid, ref_domain, tol):
    outside = ~inputs.grid_mask(K, L)
    assert np.all(out_grid[..., outside] == 0.0)
    assert rel(inputs.from_grid(K, L, out_grid), ref_domain) < tol


# K = 7 spans several Gauss-Seidel tiles with the re-entrant corner inside one of them
@pytest.mark.parametrize("K,J", [(2, 2), (3, 4), (5, 3), (7, 3)])
def test_lshape_operators(K, J):
    p = schur.Problem(K, J, L)
    with Solver(K, J, domain=L) as s:
        # K_x on 2 N_t slices
        b = inputs.random_state(2 * p.Nt, p.Nx, 61)
        x = torch.empty((2 * p.Nt, s.Nx), dtype=torch.float64, device="cuda")
        s.apply_Kx(dev(inputs.to_grid(K, L, b)), x)
        check(K, host(x), p.Kx.apply(b.T).T, TOL_OP)
        # S in single-scale coordinates, S_hat and K_X in wavelet coordinates
        u = inputs.random_state(p.Nt, p.Nx, 62)
        y = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.apply_S_nodal(dev(inputs.to_grid(K, L, u)), y)
        check(K, host(y), p.apply_S_route1(u), TOL_OP)
        w = inputs.random_state(p.Nt, p.Nx, 63)
        s.apply_S(dev(inputs.to_grid(K, L, w)), y)
        check(K, host(y), p.to_inplace(p.apply_Shat(p.from_inplace(w))), TOL_OP)
        s.apply_KX(dev(inputs.to_grid(K, L, w)), y)
        check(K, host(y), p.to_inplace(p.apply_KX(p.from_inplace(w))), TOL_OP)
        # right-hand side of the manufactured solution u = (1+t^2) sin(2 pi x) sin(2 pi y)
        g, u0, _ = inputs.manufactured(K, J, L)
        s.rhs(dev(inputs.to_grid(K, L, g)), dev(inputs.to_grid(K, L, u0)), y)
        check(K, host(y), p.to_inplace(p.rhs_hat(g, u0)), TOL_OP)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_SOLVE), ("mixed", 1e-8)])
def test_lshape_solve(precision, tol):
    K, J = 5, 4
    p = schur.Problem(K, J, L)
    g, u0, _ = inputs.manufactured(K, J, L)
    u_ref, _, _ = schur.solve(p, g, u0, tol=1e-13)
    with Solver(K, J, domain=L, tol=1e-11, precision=precision) as s:
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(dev(inputs.to_grid(K, L, g)), dev(inputs.to_grid(K, L, u0)), f)
        w = torch.empty_like(f)
        s.pcg_solve(f, w)
        u = torch.empty_like(f)
        s.synthesize(w, u)
        check(K, host(u), u_ref, tol)
