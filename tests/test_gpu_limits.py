"""Edge sizes of the boundary: the longest time axis (J = 14, N_t = 16385), the finest space level
(K = 12, N_x = 16 769 025), the smallest problems, and batches at the slice limit.

Against the oracle where it runs in seconds (J = 14 at K = 2), by properties that hold at any size
where it does not (K = 12: symmetry of S_hat and K_X, positivity, and the solve's own residual).
Tolerances as in test_gpu_parity.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur  # noqa: E402
from paper_2009_08875_gb300 import Solver, STError, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_longest_time_axis_matches_oracle():
    K, J = 2, 14
    p = schur.Problem(K, J)
    g, u0, _ = inputs.manufactured(K, J)
    u_ref, _, _ = schur.solve(p, g, u0, tol=1e-13)
    with Solver(K, J, tol=1e-12) as s:
        assert s.shape == (16385, 9)
        u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), u)
    assert rel(u.numpy(), u_ref) < 1e-10


def test_finest_space_level_properties():
    K, J = 12, 1
    with Solver(K, J) as s:
        assert s.shape == (3, (2 ** 12 - 1) ** 2)
        rng = np.random.default_rng(12)
        a = torch.from_numpy(rng.standard_normal(s.shape)).cuda()
        b = torch.from_numpy(rng.standard_normal(s.shape)).cuda()
        Sa, Sb, Ka, Kb = (torch.empty_like(a) for _ in range(4))
        s.apply_S(a, Sa)
        s.apply_S(b, Sb)
        s.apply_KX(a, Ka)
        s.apply_KX(b, Kb)
        torch.cuda.synchronize()
        for A1, A2 in ((Sa, Sb), (Ka, Kb)):
            lhs, rhs = float(torch.sum(b * A1)), float(torch.sum(a * A2))
            assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), float(torch.sum(a * A1)), float(torch.sum(b * A2)))
        assert float(torch.sum(a * Sa)) > 0 and float(torch.sum(a * Ka)) > 0
        # a solve at this size meets its tolerance
        g, u0, _ = inputs.manufactured(K, J)
        f = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.rhs(torch.from_numpy(g).cuda(), torch.from_numpy(u0).cuda(), f)
        w = torch.empty_like(f)
        its, relres = s.pcg_solve(f, w)
        assert relres <= 1e-10 and its < 60


@pytest.mark.parametrize("K,J", [(1, 1), (1, 14), (12, 1)])
def test_smallest_and_extreme_shapes_set_up(K, J):
    with Solver(K, J) as s:
        assert s.shape == (2 ** J + 1, (2 ** K - 1) ** 2)


def test_batch_at_the_slice_limit():
    # 2 B N_t <= 65535: J = 4 (N_t = 17) allows B = 1927; one more is rejected
    J = 4
    B = 65535 // (2 * 17)
    with Solver(2, J, batch=B) as s:
        g = np.stack([inputs.manufactured(2, J)[0]] * B)
        u0 = np.stack([inputs.manufactured(2, J)[1]] * B)
        u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        its, _ = s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), u)
    with Solver(2, J) as s1:
        u1 = torch.zeros(s1.shape, dtype=torch.float64).pin_memory()
        its1, _ = s1.solve_host(torch.from_numpy(g[0]).pin_memory(), torch.from_numpy(u0[0]).pin_memory(), u1)
    assert its == its1 and torch.equal(u[0], u1) and torch.equal(u[B - 1], u1)
    with pytest.raises(STError):
        Solver(2, J, batch=B + 1)
