"""Nested iteration (st_nested_solve) on the GPU against the oracle's nested_solve.

Both run the same levels, transfers and stopping rules, so every level takes the same number of
PCG iterations (the stopping test compares sqrt(r^T K_X r) with a tolerance that the residual
crosses by a wide margin in these cases), and the final iterates agree up to binary64 rounding
carried through a few dozen iterations: 1e-10 relative, the FP64 solve target.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("domain,K,J,levels,rate", [(0, 5, 5, 3, 1.0), (0, 6, 4, 4, 2.0), (1, 5, 4, 3, 1.0),
                                                    (0, 4, 4, 1, 1.0), (0, 3, 3, 3, 1.0)])
def test_nested_matches_oracle(domain, K, J, levels, rate):
    eps = 1e-3
    g, u0, _ = inputs.manufactured(K, J, domain)
    _, w_ref, its_ref = schur.nested_solve(K, J, levels, g, u0, eps, rate=rate, domain=domain)
    p = schur.Problem(K, J, domain)
    with Solver(K, J, domain=domain) as s:
        w = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        st, its = s.nested_solve(levels, eps, dev(inputs.to_grid(K, domain, g)),
                                 dev(inputs.to_grid(K, domain, u0)), w, rate=rate)
        torch.cuda.synchronize()
        w = w.cpu().numpy()
    assert st == 0
    assert its == its_ref
    assert rel(inputs.from_grid(K, domain, w), p.to_inplace(w_ref)) < 1e-10


def test_nested_reaction_diffusion():
    D, c = np.array([[1.3, 0.4], [0.4, 0.7]]), 2.5
    K, J, levels, eps = 5, 4, 3, 1e-4
    g, u0, _ = inputs.manufactured(K, J, D=D, c=c)
    _, w_ref, its_ref = schur.nested_solve(K, J, levels, g, u0, eps, D=D, c=c)
    p = schur.Problem(K, J, D=D, c=c)
    with Solver(K, J, D=D, c=c) as s:
        w = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        st, its = s.nested_solve(levels, eps, dev(g), dev(u0), w)
        torch.cuda.synchronize()
    assert st == 0 and its == its_ref
    assert rel(w.cpu().numpy(), p.to_inplace(w_ref)) < 1e-10


def test_nested_batch_equals_alone_and_repeats():
    K, J, levels, B = 5, 4, 3, 3
    gs = [inputs.smooth_forcing(K, J, seed=40 + b)[0] for b in range(B)]
    u0 = np.zeros((B, (2 ** K - 1) ** 2))
    with Solver(K, J, batch=B) as s:
        wb = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        st, itsb = s.nested_solve(levels, 1e-4, dev(np.stack(gs)), dev(u0), wb)
        wb2 = torch.empty_like(wb)
        st2, itsb2 = s.nested_solve(levels, 1e-4, dev(np.stack(gs)), dev(u0), wb2)  # handles reused
        torch.cuda.synchronize()
    assert st == 0 and st2 == 0 and itsb == itsb2 and torch.equal(wb, wb2)
    for b in (0, 2):
        with Solver(K, J) as s:
            wa = torch.empty(s.shape, dtype=torch.float64, device="cuda")
            s.nested_solve(levels, 1e-4, dev(gs[b]), dev(u0[b]), wa)
            torch.cuda.synchronize()
        assert torch.equal(wb[b], wa)


def test_nested_rejects_too_many_levels():
    from paper_2009_08875_gb300 import STError
    with Solver(3, 2) as s:
        w = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        g = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
        u0 = torch.zeros(s.u0_shape, dtype=torch.float64, device="cuda")
        with pytest.raises(STError):
            s.nested_solve(3, 1e-3, g, u0, w)
