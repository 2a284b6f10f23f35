"""Pins of the oracle's 3D problem (Sec. 5.2: the unit cube, P1 on a uniform tetrahedral mesh).

* Stencils by counting: every interior vertex of the Kuhn mesh lies in 24 tetrahedra of volume
  h^3/6; an axis edge and a body-diagonal edge lie in 6 of them, a face-diagonal edge in 4.  The
  P1 element mass matrix |T|/20 (1 + delta) then gives the mass stencil h^3 [24/60 = 2/5 at the
  centre; 6/120 = 1/20 at the six axis and the two body-diagonal neighbours; 4/120 = 1/30 at the
  six face-diagonal neighbours], and the stiffness matrix of this mesh is the 7-point
  Laplacian h [6; -1 at the axis neighbours] (known for Kuhn's subdivision; the face- and
  body-diagonal couplings cancel).
* Nestedness: Galerkin exactness P^T C_f P = C_c.
* The 4-colour V-cycle is symmetric and converges to C^-1.
* The closed form of S with K_x = A^-1, Lemma 4.1 = Lemma 4.2, the 3 x 3 S at K = J = 1.
* Convergence to the manufactured solution u = (1 + t^2) sin(pi x) sin(pi y) sin(pi z).
"""
import numpy as np
import pytest

from oracle import schur, space
from paper_2009_08875_gb300 import inputs

CUBE = space.CUBE


def _row(mesh, Mat, node):
    i0, j0, k0 = mesh.node_i[node], mesh.node_j[node], mesh.node_k[node]
    row = Mat.getrow(node).toarray().ravel()
    return {(int(mesh.node_i[q] - i0), int(mesh.node_j[q] - j0), int(mesh.node_k[q] - k0)): row[q]
            for q in np.nonzero(np.abs(row) > 1e-300)[0]}


def test_stencils_by_counting():
    mesh = space.Mesh3(3)
    h = mesh.h
    n = 2 ** 3 - 1
    centre = (3 * n + 3) * n + 3
    axis = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    face = [(1, 1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, -1, -1)]
    body = [(1, 1, 1), (-1, -1, -1)]
    M = _row(mesh, space.mass_matrix(mesh), centre)
    expect = {(0, 0, 0): 2 / 5}
    expect.update({o: 1 / 20 for o in axis + body})
    expect.update({o: 1 / 30 for o in face})
    assert set(M) == set(expect)
    for o, v in expect.items():
        assert abs(M[o] - v * h ** 3) <= 1e-15
    A = _row(mesh, space.stiffness_matrix(mesh), centre)
    assert set(A) == {(0, 0, 0)} | set(axis)
    assert abs(A[(0, 0, 0)] - 6 * h) <= 1e-14 and all(abs(A[o] + h) <= 1e-14 for o in axis)


def test_galerkin_exact_and_colouring_valid():
    fine, coarse = space.Mesh3(3), space.Mesh3(2)
    P = space.prolongation(coarse, fine)
    for f in (space.mass_matrix, space.stiffness_matrix):
        assert abs(P.T @ f(fine) @ P - f(coarse)).max() <= 1e-14
    # nodes of one colour are never coupled
    C = space.mass_matrix(fine).tocoo()
    col = fine.colour()
    off = C.row != C.col
    assert np.all(col[C.row[off]] != col[C.col[off]])


def test_vcycle_symmetric_and_convergent():
    mg = space.Multigrid(3, CUBE, 0.3, 4.0)
    K = mg.apply(np.eye(mg.C[3].shape[0]))
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > 0
    many = space.Multigrid(3, CUBE, 0.3, 4.0, n_cycles=40).apply(np.eye(mg.C[3].shape[0]))
    assert np.abs(many - np.linalg.inv(mg.C[3].toarray())).max() <= 1e-10 * np.abs(many).max()


def test_closed_form_with_exact_Kx():
    p = schur.Problem(2, 2, CUBE, inverses="direct")
    M, A = p.Mx.toarray(), p.Ax.toarray()
    eN = np.zeros((p.Nt, p.Nt))
    eN[-1, -1] = 1.0
    S_closed = np.kron(p.At, M @ np.linalg.solve(A, M)) + np.kron(p.Mt, A) + np.kron(eN, M)
    S = schur.dense(p.apply_S, (p.Nt, p.Nx))
    assert np.abs(S - S_closed).max() <= 1e-13 * np.abs(S_closed).max()


def test_lemma_4_1_equals_lemma_4_2():
    p = schur.Problem(3, 3, CUBE)
    U = np.random.default_rng(4).standard_normal((p.Nt, p.Nx))
    s1, s2 = p.apply_S_route1(U), p.apply_S_route2(U)
    assert np.abs(s1 - s2).max() <= 1e-13 * np.abs(s1).max()


def test_brute_force_smallest_problem():
    # K = 1: one node at the centre, h = 1/2: M = 2/5 h^3 = 1/20, A = 6 h = 3, multigrid exact
    p = schur.Problem(1, 1, CUBE)
    At = 2.0 * np.array([[1, -1, 0], [-1, 2, -1], [0, -1, 1]])
    Mt = np.array([[2, 1, 0], [1, 4, 1], [0, 1, 2]]) / 12.0
    e3 = np.zeros((3, 3))
    e3[2, 2] = 1.0
    S_hand = At * (1 / 20) ** 2 / 3.0 + 3.0 * Mt + e3 / 20.0
    np.testing.assert_allclose(schur.dense(p.apply_S, (3, 1)), S_hand, rtol=1e-14, atol=1e-16)


def test_manufactured_solution_converges():
    errs = []
    for L in (2, 3, 4):
        p = schur.Problem(L, L, CUBE)
        g, u0, u = inputs.manufactured(L, L, CUBE)
        uh, _, info = schur.solve(p, g, u0, tol=1e-11)
        assert info["converged"]
        e = uh - u
        errs.append(np.sqrt(np.sum(e * (p.Mt @ schur.rows(p.Ax, e)))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 0.9, (errs, rates)
