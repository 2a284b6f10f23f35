"""The Gauss-Seidel kernels (shared-memory tiles, register wavefront, register tiles, and the
binary32 wide register regions with paired arithmetic) and the autotuner.

All kernels perform the same three-colour sweeps with the same summation order per point, so
every operator that runs the multigrid (K_x, K_X, the binary32 S and K_X, the bfloat16-storage
K_X) must give bitwise the same result with any of them, on the square and on the L-shape, for
one problem and for a batch, the wavefront at any number of rows per segment, and with sweep
counts that are not a multiple of the fused three.  The autotuner only picks among them, so a
solve after st_autotune must give bitwise the solve before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_08875_gb300 import Solver, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def run_ops(s, x):
    out = {}
    y = torch.empty_like(x)
    s.apply_KX(x, y)
    out["KX"] = y.clone()
    x32 = x.float()
    y32 = torch.empty_like(x32)
    s.apply_KX_f32(x32, y32)
    out["KX32"] = y32.clone()
    s.apply_S_f32(x32, y32)
    out["S32"] = y32.clone()
    s.apply_KX_bf16(x32, y32)  # square and L-shape only (not the cube)
    out["KXbf16"] = y32.clone()
    b = torch.cat([x.reshape(-1, s.Nx), x.reshape(-1, s.Nx)]).contiguous()
    xk = torch.empty_like(b)
    s.apply_Kx(b, xk)
    out["Kx"] = xk.clone()
    torch.cuda.synchronize()
    return out


REGISTER_KINDS = ("registers", "registers_8x12", "registers_6x16", "registers_wide")


# K = 3 (one tile / strip), K = 6 and K = 8 (several strips and vertical segments, ragged edges);
# K = 7, 8 and 9 on the square also run the wide binary32 regions on their levels with n >= 96
# (half-warp 96-column regions at n = 127, whole-warp 192-column regions above: two and three
# regions per row, the last clamped against the grid's edge)
@pytest.mark.parametrize("K,J,domain,B", [(3, 3, 0, 1), (6, 4, 0, 1), (8, 2, 0, 1), (6, 3, 1, 1), (5, 3, 0, 3),
                                          (7, 2, 1, 2), (9, 1, 0, 1), (8, 1, 0, 2), (8, 2, 1, 1), (7, 3, 0, 1),
                                          (7, 2, 0, 2)])
def test_tiles_and_wavefront_bitwise_equal(K, J, domain, B):
    with Solver(K, J, domain=domain, batch=B) as s:
        rng = np.random.default_rng(K * 100 + J)
        x = rng.standard_normal(s.shape)
        if domain == 1:
            x = x * inputs.grid_mask(K, 1).reshape(-1)
        x = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        s.set_smoother("tiles")
        a = run_ops(s, x)
        for kind in REGISTER_KINDS:
            s.set_smoother(kind)
            c = run_ops(s, x)
            for name in a:
                assert torch.equal(a[name], c[name]), (name, kind)
        s.set_smoother("wavefront")
        # default segments, then one row per segment, a ragged length, and one segment per strip
        for rows in (0, 1, 5, 73, 1000):
            s.set_wave_rows(rows)
            b = run_ops(s, x)
            for name in a:
                assert torch.equal(a[name], b[name]), (name, rows)


# sweep counts that are not a multiple of three: binary32 launches of one sweep beside fused ones
@pytest.mark.parametrize("K,J,domain,pre,post", [(7, 2, 0, 4, 2), (6, 2, 1, 1, 5), (8, 1, 0, 4, 2), (9, 1, 0, 1, 5)])
def test_register_tiles_with_unfused_sweeps(K, J, domain, pre, post):
    with Solver(K, J, domain=domain, n_pre=pre, n_post=post) as s:
        rng = np.random.default_rng(K + 7 * pre)
        x = rng.standard_normal(s.shape)
        if domain == 1:
            x = x * inputs.grid_mask(K, 1).reshape(-1)
        x = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        s.set_smoother("tiles")
        a = run_ops(s, x)
        for kind in REGISTER_KINDS:
            s.set_smoother(kind)
            c = run_ops(s, x)
            for name in a:
                assert torch.equal(a[name], c[name]), (name, kind)


def test_set_smoother_rejects_unknown_kind():
    from paper_2009_08875_gb300 import _lib
    with Solver(3, 2) as s:
        assert _lib.load().st_set_smoother(s._h, 6) == 1  # ST_ERR_ARG
        assert _lib.load().st_set_smoother(s._h, -1) == 1
        assert _lib.load().st_set_wave_rows(s._h, -1) == 1
        assert _lib.load().st_set_wave_rows(s._h, 65536) == 1


# K = 8: the binary32 candidates include the wide regions on level 8
@pytest.mark.parametrize("precision,K,J", [("fp64", 6, 4), ("mixed_precond", 6, 4), ("mixed", 8, 3)])
def test_autotune_keeps_solution_bitwise(precision, K, J):
    g, u0 = inputs.smooth_forcing(K, J, seed=3)
    g = torch.from_numpy(inputs.to_grid(K, 0, g)).pin_memory()
    u0 = torch.from_numpy(inputs.to_grid(K, 0, u0)).pin_memory()
    with Solver(K, J, precision=precision, use_graphs=True) as s:
        u1 = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
        it1, _ = s.solve_host(g, u0, u1)
        table = s.autotune()
        assert set(table) == set(range(2, K + 1))
        for row in table.values():
            for tiles_ms, wave_ms, regs_ms in row.values():
                assert tiles_ms > 0 and wave_ms > 0 and regs_ms > 0
        u2 = torch.zeros_like(u1)
        it2, _ = s.solve_host(g, u0, u2)
    assert it1 == it2
    assert torch.equal(u1, u2)
