"""The reaction-diffusion equation of Sec. 4 on the GPU against the oracle.

A_x = <D grad, grad> + c M_x (Lemma 4.1) enters the spatial stencils of S, the epilogue, the
middle factor of K_X and every multigrid operator.  Three coefficient sets cover the kernels'
branches: a full anisotropic D with c > 0 (x and y neighbours differ, diagonal couplings in K_x),
a diagonal anisotropic D with c = 0 (x and y neighbours differ, K_x without diagonal couplings),
and an isotropic D = 0.5 Id with c = 3 (K_x with diagonal couplings from the mass term only).
Tolerances as in test_gpu_parity (binary64) and test_gpu_batch (binary32 preconditioner).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur, space  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_OP = 1e-12
TOL_SOLVE = 1e-10

COEFS = {
    "aniso_react": (np.array([[1.3, 0.4], [0.4, 0.7]]), 2.5),
    "diag_aniso": (np.array([[2.0, 0.0], [0.0, 0.25]]), 0.0),
    "iso_react": (np.array([[0.5, 0.0], [0.0, 0.5]]), 3.0),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def check(K, domain, out_grid, ref, tol):
    if domain == space.LSHAPE:
        assert np.all(out_grid[..., ~inputs.grid_mask(K, domain)] == 0.0)
    assert rel(inputs.from_grid(K, domain, out_grid), ref) < tol


# K = 7 spans several Gauss-Seidel tiles and wavefront strips with ragged edges
@pytest.mark.parametrize("name", list(COEFS))
@pytest.mark.parametrize("K,J,domain", [(2, 2, 0), (4, 3, 0), (7, 3, 0), (5, 3, 1)])
def test_operators(name, K, J, domain):
    D, c = COEFS[name]
    p = schur.Problem(K, J, domain, D=D, c=c)
    with Solver(K, J, domain=domain, D=D, c=c) as s:
        b = inputs.random_state(2 * p.Nt, p.Nx, 71)
        x = torch.empty((2 * p.Nt, s.Nx), dtype=torch.float64, device="cuda")
        s.apply_Kx(dev(inputs.to_grid(K, domain, b)), x)
        check(K, domain, host(x), p.Kx.apply(b.T).T, TOL_OP)
        u = inputs.random_state(p.Nt, p.Nx, 72)
        y = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.apply_S_nodal(dev(inputs.to_grid(K, domain, u)), y)
        check(K, domain, host(y), p.apply_S_route1(u), TOL_OP)
        w = inputs.random_state(p.Nt, p.Nx, 73)
        s.apply_S(dev(inputs.to_grid(K, domain, w)), y)
        check(K, domain, host(y), p.to_inplace(p.apply_Shat(p.from_inplace(w))), TOL_OP)
        s.apply_KX(dev(inputs.to_grid(K, domain, w)), y)
        check(K, domain, host(y), p.to_inplace(p.apply_KX(p.from_inplace(w))), TOL_OP)
        g, u0, _ = inputs.manufactured(K, J, domain, D=D, c=c)
        s.rhs(dev(inputs.to_grid(K, domain, g)), dev(inputs.to_grid(K, domain, u0)), y)
        check(K, domain, host(y), p.to_inplace(p.rhs_hat(g, u0)), TOL_OP)


@pytest.mark.parametrize("name", list(COEFS))
@pytest.mark.parametrize("precision,tol", [("fp64", TOL_SOLVE), ("mixed_precond", 1e-8), ("mixed", 1e-8)])
def test_solve(name, precision, tol):
    D, c = COEFS[name]
    K, J = 5, 4
    p = schur.Problem(K, J, D=D, c=c)
    g, u0, _ = inputs.manufactured(K, J, D=D, c=c)
    u_ref, _, _ = schur.solve(p, g, u0, tol=1e-13)
    with Solver(K, J, D=D, c=c, tol=1e-11, precision=precision) as s:
        u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), u)
    assert rel(u.numpy(), u_ref) < tol


def test_smoothers_bitwise_equal_with_anisotropy():
    D, c = COEFS["aniso_react"]
    with Solver(6, 3, D=D, c=c) as s:
        x = dev(np.random.default_rng(9).standard_normal(s.shape))
        out = []
        for kind in ("tiles", "wavefront"):
            s.set_smoother(kind)
            y = torch.empty_like(x)
            s.apply_KX(x, y)
            b = torch.cat([x, x]).contiguous()
            xk = torch.empty_like(b)
            s.apply_Kx(b, xk)
            torch.cuda.synchronize()
            out.append((y, xk))
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_batch_with_coefficients_equals_alone():
    from paper_2009_08875_gb300 import Batch
    D, c = COEFS["aniso_react"]
    bt = Batch(D=D, c=c, tol=1e-10)
    probs = []
    for i, (K, J) in enumerate([(4, 3), (5, 3), (4, 3)]):
        g, u0 = inputs.smooth_forcing(K, J, seed=20 + i)
        g = torch.from_numpy(g).pin_memory()
        u0 = torch.from_numpy(u0).pin_memory()
        u = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
        bt.add(0, K, J, g, u0, u)
        probs.append((K, J, g, u0, u))
    assert bt.run() == 0
    for K, J, g, u0, u in probs:
        with Solver(K, J, D=D, c=c, tol=1e-10) as s:
            ua = torch.zeros_like(u)
            s.solve_host(g, u0, ua)
        assert torch.equal(u, ua)
    bt.close()
