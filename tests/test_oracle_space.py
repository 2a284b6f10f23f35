"""Pins of the oracle's spatial part (P1 matrices, prolongation, multigrid) against
closed forms and textbook identities; none of them re-types the oracle's formulas."""
import numpy as np
import pytest

from oracle import space


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_dof_counts(domain):
    # Sec. 5.1: N_x = (2^K - 1)^2 on the square; the L-shape drops the (2^(K-1))^2 nodes of the quadrant
    for K in (2, 3, 5):
        m = space.Mesh(K, domain)
        expect = (2 ** K - 1) ** 2 - (0 if domain == space.SQUARE else (2 ** (K - 1)) ** 2)
        assert m.N == expect


def test_mass_integrates_constants_and_quadratics():
    # 1^T M 1 over the interior hats = integral of the sum of interior hats; for a node
    # away from the boundary, (M 1)_p = int phi_p = h^2 (six triangles of area h^2/2, 1/3 each)
    for K in (3, 5):
        m = space.Mesh(K)
        M = space.mass_matrix(m)
        row_sum = np.asarray(M.sum(1)).ravel()
        inner = (m.node_i > 1) & (m.node_i < m.m - 1) & (m.node_j > 1) & (m.node_j < m.m - 1)
        np.testing.assert_allclose(row_sum[inner], m.h ** 2, rtol=1e-14)
    # v^T M v -> int sin^2(pi x) sin^2(pi y) = 1/4 at second order
    errs = []
    for K in (4, 5, 6):
        m = space.Mesh(K)
        x, y = m.coords()
        v = np.sin(np.pi * x) * np.sin(np.pi * y)
        errs.append(abs(v @ (space.mass_matrix(m) @ v) - 0.25))
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_stiffness_kernel_and_energy():
    m = space.Mesh(5)
    A = space.stiffness_matrix(m)
    x, y = m.coords()
    # linear functions are discrete-harmonic at nodes whose neighbours are all interior
    inner = (m.node_i > 1) & (m.node_i < m.m - 1) & (m.node_j > 1) & (m.node_j < m.m - 1)
    for v in (x, y, 2 * x - 3 * y + 1):
        assert np.abs((A @ v)[inner]).max() < 1e-12
    # energy of the interpolant of sin(pi x) sin(pi y) -> pi^2/2
    errs = []
    for K in (4, 5, 6):
        mm = space.Mesh(K)
        xx, yy = mm.coords()
        v = np.sin(np.pi * xx) * np.sin(np.pi * yy)
        errs.append(abs(v @ (space.stiffness_matrix(mm) @ v) - np.pi ** 2 / 2))
    assert errs[2] < errs[1] < errs[0] < 0.2


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_matrices_symmetric_positive(domain):
    m = space.Mesh(3, domain)
    for Mat in (space.mass_matrix(m), space.stiffness_matrix(m)):
        D = Mat.toarray()
        assert np.abs(D - D.T).max() == 0.0
        assert np.linalg.eigvalsh(D).min() > 0


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_prolongation_is_galerkin_exact(domain):
    # nested P1 spaces: P^T A_f P = A_c and P^T M_f P = M_c exactly (coarse form = restricted fine form)
    for K in (3, 4):
        c, f = space.Mesh(K - 1, domain), space.Mesh(K, domain)
        P = space.prolongation(c, f)
        Af, Ac = space.stiffness_matrix(f), space.stiffness_matrix(c)
        Mf, Mc = space.mass_matrix(f), space.mass_matrix(c)
        assert abs(P.T @ Af @ P - Ac).max() < 1e-13
        assert abs(P.T @ Mf @ P - Mc).max() < 1e-17
        # columns of P sum to 1 + 6 * 1/2 = 4 for a coarse hat away from the boundary
        colsum = np.asarray(P.sum(0)).ravel()
        assert colsum.max() == 4.0


def _dense_K(mg, N):
    return mg.apply(np.eye(N))


@pytest.mark.parametrize("a,s", [(1.0, 0.0), (0.3, 1.0), (0.3, 16.0)])
@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_multigrid_symmetric_spd_and_contracting(a, s, domain):
    K = 4
    mg = space.Multigrid(K, domain, a, s)
    m = mg.meshes[K]
    Kd = _dense_K(mg, m.N)
    assert np.abs(Kd - Kd.T).max() <= 1e-14 * np.abs(Kd).max()
    C = mg.C[K].toarray()
    # two V-cycles: error propagator E = I - K C; its C-energy norm is small
    E = np.eye(m.N) - Kd @ C
    Lc = np.linalg.cholesky(C)
    En = np.linalg.norm(Lc.T @ E @ np.linalg.inv(Lc.T), 2)
    assert En < 0.05
    assert np.linalg.eigvalsh(0.5 * (Kd + Kd.T)).min() > 0


def test_multigrid_reversed_post_order_is_what_makes_it_symmetric():
    # with the post-sweeps in the same colour order as the pre-sweeps the V-cycle is not
    # symmetric; this guards the colour-order reading (symmetric K is needed for S = S^T)
    mg = space.Multigrid(3, space.SQUARE, 1.0, 0.0)
    orig = mg._vcycle

    def vcycle_same_order(k, x, b):
        if k == mg.k0:
            return np.linalg.solve(mg.coarse_dense, b)
        for _ in range(mg.n_pre):
            for c in (0, 1, 2):
                x = mg._gs_colour(k, c, x, b)
        r = b - mg.C[k] @ x
        bc = mg.P[k].T @ r
        x = x + mg.P[k] @ vcycle_same_order(k - 1, np.zeros_like(bc), bc)
        for _ in range(mg.n_post):
            for c in (0, 1, 2):
                x = mg._gs_colour(k, c, x, b)
        return x

    mg._vcycle = vcycle_same_order
    Kd = mg.apply(np.eye(49))
    assert np.abs(Kd - Kd.T).max() > 1e-6
    mg._vcycle = orig
    Kd = mg.apply(np.eye(49))
    assert np.abs(Kd - Kd.T).max() < 1e-15


def test_multigrid_exact_on_coarsest_and_converges_to_inverse():
    mg = space.Multigrid(1, space.SQUARE, 1.0, 0.0)
    # K = 1: one node at (1/2, 1/2), A = [4] -> exact inverse 1/4
    assert mg.apply(np.array([1.0]))[0] == 0.25
    mg = space.Multigrid(4, space.SQUARE, 0.3, 4.0, n_cycles=40)
    m = mg.meshes[4]
    b = np.random.default_rng(3).standard_normal(m.N)
    x = mg.apply(b)
    xe = np.linalg.solve(mg.C[4].toarray(), b)
    assert np.abs(x - xe).max() < 1e-12 * np.abs(xe).max()
    mg2 = space.Multigrid(3, space.LSHAPE, 1.0, 0.0, n_cycles=40)
    b2 = np.random.default_rng(4).standard_normal(mg2.meshes[3].N)
    np.testing.assert_allclose(mg2.apply(b2), np.linalg.solve(mg2.C[3].toarray(), b2), rtol=1e-11, atol=1e-13)


def test_colour_classes_are_decoupled():
    # the 7-point pattern never couples two nodes of the same colour (i + j) mod 3
    for domain in (space.SQUARE, space.LSHAPE):
        mg = space.Multigrid(4, domain, 0.3, 2.0)
        C = mg.C[4].tocoo()
        col = mg.colour[4]
        off = C.row != C.col
        assert not np.any(col[C.row[off]] == col[C.col[off]])
