"""Pins of the oracle's reaction-diffusion operator (Sec. 4: a(eta, zeta) = <D grad eta, grad zeta>
+ c <eta, zeta>, D symmetric positive definite, c >= 0; A_x of Lemma 4.1).

The oracle assembles A_x element by element.  What pins it here:
* the interior stencil, derived by hand from the gradients of the P1 hat functions on the
  two triangle orientations of the mesh (centre 2(d11 + d22 - d12), x neighbours d12 - d11,
  y neighbours d12 - d22, (1,1) diagonal -d12, no (1,-1) coupling), plus c times the P1 mass
  stencil h^2/12 [6; 1 at the six neighbours];
* the symmetry of the mesh under x <-> y: A_x(D) with the grid transposed is A_x(D with d11
  and d22 swapped);
* the closed form of S for the exact K_x = A_x^-1 (L + L^T + Gamma_0 = e_N e_N^T), with the
  reaction-diffusion A_x in every place A_x appears;
* Lemma 4.1 equals Lemma 4.2 with the multigrid K_x, and the brute-force 3 x 3 S at K = J = 1;
* convergence of the whole solve to a manufactured solution of u_t - div(D grad u) + c u = g.
"""
import numpy as np
import pytest

from oracle import schur, space
from paper_2009_08875_gb300 import inputs

D_ANISO = np.array([[1.3, 0.4], [0.4, 0.7]])
C_REACT = 2.5


def test_interior_stencil_by_hand():
    K = 3
    mesh = space.Mesh(K)
    h = mesh.h
    A = space.operator_matrix(mesh, D_ANISO, C_REACT).toarray()
    (d11, d12), (_, d22) = D_ANISO
    m = h * h / 12.0
    n = 2 ** K - 1
    centre = 3 * n + 3                   # node (4, 4), all neighbours interior
    expect = {(0, 0): 2 * (d11 + d22 - d12) + C_REACT * 6 * m,
              (1, 0): d12 - d11 + C_REACT * m, (-1, 0): d12 - d11 + C_REACT * m,
              (0, 1): d12 - d22 + C_REACT * m, (0, -1): d12 - d22 + C_REACT * m,
              (1, 1): -d12 + C_REACT * m, (-1, -1): -d12 + C_REACT * m,
              (1, -1): 0.0, (-1, 1): 0.0}
    for (dx, dy), v in expect.items():
        assert abs(A[centre, centre + dy * n + dx] - v) <= 1e-14, (dx, dy)
    # nothing beyond the 7-point pattern
    assert np.count_nonzero(np.abs(A[centre]) > 1e-15) == 7


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_transpose_symmetry(domain):
    mesh = space.Mesh(3, domain)
    A = space.operator_matrix(mesh, D_ANISO, C_REACT).toarray()
    Dsw = np.array([[D_ANISO[1, 1], D_ANISO[0, 1]], [D_ANISO[0, 1], D_ANISO[0, 0]]])
    B = space.operator_matrix(mesh, Dsw, C_REACT).toarray()
    # dof of node (i, j) -> dof of node (j, i)
    perm = mesh.dof[mesh.node_i, mesh.node_j]
    assert np.all(perm >= 0)
    assert np.abs(A[np.ix_(perm, perm)] - B).max() <= 1e-14


def test_closed_form_with_exact_Kx():
    p = schur.Problem(3, 3, inverses="direct", D=D_ANISO, c=C_REACT)
    M, A = p.Mx.toarray(), p.Ax.toarray()
    eN = np.zeros((p.Nt, p.Nt))
    eN[-1, -1] = 1.0
    S_closed = np.kron(p.At, M @ np.linalg.solve(A, M)) + np.kron(p.Mt, A) + np.kron(eN, M)
    S = schur.dense(p.apply_S, (p.Nt, p.Nx))
    assert np.abs(S - S_closed).max() <= 1e-13 * np.abs(S_closed).max()


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_lemma_4_1_equals_lemma_4_2(domain):
    p = schur.Problem(3, 3, domain, D=D_ANISO, c=C_REACT)
    U = np.random.default_rng(3).standard_normal((p.Nt, p.Nx))
    s1, s2 = p.apply_S_route1(U), p.apply_S_route2(U)
    assert np.abs(s1 - s2).max() <= 1e-13 * np.abs(s1).max()


def test_brute_force_smallest_problem():
    # K = 1: one node at (1/2, 1/2), h = 1/2: M_x = [1/8] and A_x = [2(d11 + d22 - d12) + c/8];
    # the multigrid is exact; S = A_t M^2 / A + M_t A + e_3 e_3^T M with h_t = 1/2
    p = schur.Problem(1, 1, D=D_ANISO, c=C_REACT)
    a = 2 * (D_ANISO[0, 0] + D_ANISO[1, 1] - D_ANISO[0, 1]) + C_REACT / 8.0
    At = 2.0 * np.array([[1, -1, 0], [-1, 2, -1], [0, -1, 1]])
    Mt = np.array([[2, 1, 0], [1, 4, 1], [0, 1, 2]]) / 12.0
    e3 = np.zeros((3, 3))
    e3[2, 2] = 1.0
    S_hand = At / 64.0 / a + a * Mt + e3 / 8.0
    np.testing.assert_allclose(schur.dense(p.apply_S, (3, 1)), S_hand, rtol=1e-14, atol=1e-16)


def test_manufactured_solution_converges():
    # u = (1+t^2) sin(pi x) sin(pi y) solves u_t - div(D grad u) + c u = g for the g of
    # inputs.manufactured; the discrete L2(I;H^1_0) error falls at least linearly
    errs = []
    for L in (2, 3, 4, 5):
        p = schur.Problem(L, L, D=D_ANISO, c=C_REACT)
        g, u0, u = inputs.manufactured(L, L, D=D_ANISO, c=C_REACT)
        uh, _, info = schur.solve(p, g, u0, tol=1e-11)
        assert info["converged"]
        e = uh - u
        Alap = space.stiffness_matrix(p.mesh)
        errs.append(np.sqrt(np.sum(e * (p.Mt @ schur.rows(Alap, e)))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 0.9, (errs, rates)
    # a forcing with a wrong sign of the d12 term is not approximated
    p = schur.Problem(5, 5, D=D_ANISO, c=C_REACT)
    Dwrong = D_ANISO * np.array([[1, -1], [-1, 1]])
    g, u0, u = inputs.manufactured(5, 5, D=Dwrong, c=C_REACT)
    uh, _, _ = schur.solve(p, g, u0, tol=1e-11)
    e = uh - u
    assert np.sqrt(np.sum(e * (p.Mt @ schur.rows(space.stiffness_matrix(p.mesh), e)))) > 5 * errs[-1]
