"""bfloat16-storage multigrid (ST_MIXED_BF16) against the binary64 oracle.

K_X with every multigrid vector stored as bfloat16 (binary32 arithmetic in registers and shared
memory): each store rounds to 8 significant bits, a relative error of at most u = 2^-9.  A
multigrid application stores the iterate a few times per level and cycle, and Gauss-Seidel damps
earlier rounding errors, so K_l A K_l carries an error of a few u: the test allows 16 u in the
max norm (an emulation of the same storage in the oracle's arithmetic, rounding after every
colour step, gave 3.4 u to 5.2 u at K = 3..7).  It must also differ from the binary32 K_X by far
more than binary32 rounding, which shows that the narrow storage is in use.

The solve (binary64 refinement around a binary32 flexible PCG with the bfloat16 preconditioner)
must reach the same 1e-8 target against the oracle as the other mixed modes, with a few more
inner iterations than ST_MIXED_FP32 at most.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import schur  # noqa: E402
from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -9


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("K,J,domain", [(3, 3, 0), (5, 3, 0), (7, 3, 0), (5, 3, 1)])
def test_KX_bf16_within_storage_rounding(K, J, domain):
    p = schur.Problem(K, J, domain)
    r = inputs.random_state(p.Nt, p.Nx, 81)
    z_ref = p.to_inplace(p.apply_KX(p.from_inplace(r)))
    with Solver(K, J, domain=domain) as s:
        rt = torch.from_numpy(inputs.to_grid(K, domain, r)).cuda().float()
        zb = torch.empty_like(rt)
        s.apply_KX_bf16(rt, zb)
        z32 = torch.empty_like(rt)
        s.apply_KX_f32(rt, z32)
        torch.cuda.synchronize()
        zb = inputs.from_grid(K, domain, zb.double().cpu().numpy())
        z32 = inputs.from_grid(K, domain, z32.double().cpu().numpy())
    assert rel(zb, z_ref) < 16 * U_BF16
    assert rel(zb, z32) > 1e-4


@pytest.mark.parametrize("domain", [0, 1])
def test_solve_meets_fp64_target(domain):
    K, J = 5, 4
    p = schur.Problem(K, J, domain)
    g, u0, _ = inputs.manufactured(K, J, domain)
    u_ref, _, _ = schur.solve(p, g, u0, tol=1e-13)
    out = {}
    for precision in ("mixed", "mixed_bf16"):
        with Solver(K, J, domain=domain, tol=1e-11, precision=precision) as s:
            u = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
            gh = torch.from_numpy(inputs.to_grid(K, domain, g)).pin_memory()
            u0h = torch.from_numpy(inputs.to_grid(K, domain, u0)).pin_memory()
            its, _ = s.solve_host(gh, u0h, u)
            out[precision] = (inputs.from_grid(K, domain, u.numpy()), its, s.solve_info())
    ub, its_b, info_b = out["mixed_bf16"]
    assert rel(ub, u_ref) < 1e-8
    assert info_b["outer_iterations"] >= 1
    assert its_b <= out["mixed"][1] + 8


def test_batch_equals_alone_bitwise():
    K, J, B = 5, 4, 3
    gs, u0s = [], []
    for b in range(B):
        g, u0 = inputs.smooth_forcing(K, J, seed=300 + b)
        gs.append(g)
        u0s.append(u0)
    g = np.stack(gs)
    u0 = np.stack(u0s)
    with Solver(K, J, batch=B, precision="mixed_bf16") as s:
        ub = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
        s.solve_host(torch.from_numpy(g).pin_memory(), torch.from_numpy(u0).pin_memory(), ub)
        infos = [s.problem_info(b) for b in range(B)]
    for b in (0, 2):
        with Solver(K, J, precision="mixed_bf16") as s:
            ua = torch.zeros(s.shape, dtype=torch.float64).pin_memory()
            its, _ = s.solve_host(torch.from_numpy(g[b]).pin_memory(), torch.from_numpy(u0[b]).pin_memory(), ua)
        assert torch.equal(ub[b], ua)
        assert infos[b]["iterations"] == its
