"""st_pcg_solve from a given initial iterate (st_config.initial_guess = 1) against the oracle's PCG
from the same iterate (Sec. 3.4 with w_0 given: r_0 = f_hat - S_hat w_0).

Same tolerances as test_gpu_parity: iterates to 1e-10 of their size, equal iteration counts at
the paper's absolute stopping rule, and zero iterations when the guess already meets it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_guess_matches_oracle_pcg_from_the_same_iterate():
    K, J, eps = 5, 4, 1e-7
    p = schur.Problem(K, J)
    g, u0, _ = inputs.manufactured(K, J)
    fhat = p.rhs_hat(g, u0)
    w0 = np.random.default_rng(4).standard_normal((p.Nt, p.Nx)) * 1e-3
    w_ref, info = schur.pcg(p.apply_Shat, p.apply_KX, fhat, tol=eps, tol_mode="abs", x0=w0)
    with Solver(K, J, tol=eps, tol_mode=1, initial_guess=True) as s:
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(dev(g), dev(u0), f)
        w = dev(p.to_inplace(w0))
        its, _ = s.pcg_solve(f, w)
        torch.cuda.synchronize()
        w = w.cpu().numpy()
    assert its == info["iters"]
    assert np.abs(w - p.to_inplace(w_ref)).max() <= 1e-10 * np.abs(w_ref).max()


def test_converged_guess_takes_no_iteration_and_default_ignores_w():
    K, J = 4, 3
    g, u0, _ = inputs.manufactured(K, J)
    with Solver(K, J, tol=1e-12) as s0:
        f = torch.empty(s0.shape, dtype=torch.float64, device="cuda")
        s0.rhs(dev(g), dev(u0), f)
        w_star = torch.empty_like(f)
        s0.pcg_solve(f, w_star)
        # default: the content of w is ignored
        w_junk = torch.full_like(f, 7.0)
        its_a, _ = s0.pcg_solve(f, w_junk)
        torch.cuda.synchronize()
        assert torch.equal(w_junk, w_star)
    with Solver(K, J, tol=1e-6, tol_mode=1, initial_guess=True) as s:
        w = w_star.clone()
        its, _ = s.pcg_solve(f, w)
        torch.cuda.synchronize()
        assert its == 0 and torch.equal(w, w_star)
