"""Pins of the oracle's Schur operator, preconditioner, right-hand side and PCG.

Each pin ties the oracle to something other than itself: the two matrix forms of
Lemmas 4.1 and 4.2 (independently assembled), the closed form that S takes when
K_x = A_x^-1, hand-computed entries at the smallest sizes, the printed condition
numbers of Table 5.1, a dense direct solve, and convergence to a manufactured
solution.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import schur, space
from paper_2009_08875_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(p, seed):
    return np.random.default_rng(seed).standard_normal((p.Nt, p.Nx))


@pytest.mark.parametrize("K,J,domain", [(3, 3, space.SQUARE), (3, 4, space.LSHAPE), (4, 2, space.SQUARE)])
def test_lemma_4_1_equals_lemma_4_2(K, J, domain):
    # route (i): B^T (O^-1 kron K_x) B + Gamma_0 kron M, built from the DG test-space matrices T, N, O
    # route (ii): the five Kronecker terms of Lemma 4.2; both with the multigrid K_x
    p = schur.Problem(K, J, domain)
    U = _rand(p, 7)
    s1, s2 = p.apply_S_route1(U), p.apply_S_route2(U)
    assert np.abs(s1 - s2).max() <= 1e-13 * np.abs(s1).max()


def test_closed_form_with_exact_Kx():
    # K_x = A^-1: since L + L^T + Gamma_0 = e_N e_N^T,
    # S = A_t kron M A^-1 M + M_t kron A + e_N e_N^T kron M (the discrete X-norm Gram matrix)
    p = schur.Problem(3, 3, inverses="direct")
    M, A = p.Mx.toarray(), p.Ax.toarray()
    eN = np.zeros((p.Nt, p.Nt))
    eN[-1, -1] = 1.0
    S_closed = np.kron(p.At, M @ np.linalg.solve(A, M)) + np.kron(p.Mt, A) + np.kron(eN, M)
    S = schur.dense(p.apply_S, (p.Nt, p.Nx))
    assert np.abs(S - S_closed).max() <= 1e-13 * np.abs(S_closed).max()


def test_brute_force_smallest_problem():
    # K = 1 (one node at (1/2,1/2)), J = 1 (N_t = 3): M_x = [1/8], A_x = [4], multigrid exact.
    # h_t = 1/2: A_t = 2 [[1,-1,0],[-1,2,-1],[0,-1,1]], M_t = 1/12 [[2,1,0],[1,4,1],[0,1,2]],
    # S = A_t (1/8)(1/4)(1/8) + 4 M_t + e_3 e_3^T / 8
    p = schur.Problem(1, 1)
    assert p.Nx == 1 and p.Nt == 3
    At = 2.0 * np.array([[1, -1, 0], [-1, 2, -1], [0, -1, 1]])
    Mt = np.array([[2, 1, 0], [1, 4, 1], [0, 1, 2]]) / 12.0
    e3 = np.zeros((3, 3))
    e3[2, 2] = 1.0
    S_hand = At / 256.0 + 4.0 * Mt + e3 / 8.0
    S = schur.dense(p.apply_S, (3, 1))
    np.testing.assert_allclose(S, S_hand, rtol=1e-14, atol=1e-16)
    # wavelets at J = 1: c_0 -> hats at the ends plus half the middle, d_0 -> sqrt(2)(phi_1 - phi_0 - phi_2)
    W = p.W.toarray()
    np.testing.assert_allclose(W, [[1, 0, -np.sqrt(2)], [0.5, 0.5, np.sqrt(2)], [0, 1, -np.sqrt(2)]], atol=1e-15)


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_S_and_Shat_spd(domain):
    p = schur.Problem(3, 2, domain)
    S = schur.dense(p.apply_S, (p.Nt, p.Nx))
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    np.linalg.cholesky(0.5 * (S + S.T))
    Sh = schur.dense(p.apply_Shat, (p.Nt, p.Nx))
    W = np.kron(p.W.toarray(), np.eye(p.Nx))
    assert np.abs(Sh - W.T @ S @ W).max() <= 1e-13 * np.abs(Sh).max()
    KX = schur.dense(p.apply_KX, (p.Nt, p.Nx))
    assert np.abs(KX - KX.T).max() <= 1e-14 * np.abs(KX).max()
    assert np.linalg.eigvalsh(0.5 * (KX + KX.T)).min() > 0


def _golden_table_5_1():
    rows = []
    with open(os.path.join(GOLDEN, "table_5_1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                nt, nx, k = line.split()
                rows.append((int(nt), int(nx), float(k)))
    return rows


@pytest.mark.parametrize("Nt,Nx,kappa", _golden_table_5_1())
def test_table_5_1_condition_numbers(Nt, Nx, kappa):
    # Sec. 5.1, Table 5.1: kappa_2(K_X S_hat) with direct inverses and alpha = 0.3.
    # Lanczos estimate from 120+ PCG steps; the paper's eigen-solver is not stated, accept 1%.
    J = int(np.log2(Nt - 1))
    K = int(np.log2(np.sqrt(Nx) + 1))
    p = schur.Problem(K, J, inverses="direct")
    b = _rand(p, 1)
    _, info = schur.pcg(p.apply_Shat, p.apply_KX, b, tol=1e-15, maxit=150)
    k_est, _ = schur.lanczos_kappa(info["alpha"], info["beta"])
    assert abs(k_est - kappa) <= 0.01 * kappa, (k_est, kappa)


def test_kappa_robust_in_space():
    # Sec. 5.1: with direct inverses the condition number is robust w.r.t. spatial refinement
    ks = []
    for K in (3, 4):
        p = schur.Problem(K, 7, inverses="direct")
        _, info = schur.pcg(p.apply_Shat, p.apply_KX, _rand(p, 1), tol=1e-15, maxit=150)
        ks.append(schur.lanczos_kappa(info["alpha"], info["beta"])[0])
    assert abs(ks[0] - ks[1]) < 0.005 * ks[0], ks


def test_lanczos_estimate_matches_dense_kappa():
    p = schur.Problem(3, 3)
    Sh = schur.dense(p.apply_Shat, (p.Nt, p.Nx))
    KX = schur.dense(p.apply_KX, (p.Nt, p.Nx))
    ev = sl.eigh(Sh, np.linalg.inv(KX), eigvals_only=True)
    _, info = schur.pcg(p.apply_Shat, p.apply_KX, _rand(p, 2), tol=1e-15, maxit=300)
    k_est, _ = schur.lanczos_kappa(info["alpha"], info["beta"])
    # Ritz values lie inside the spectrum, so the estimate is a slight underestimate
    kappa = ev[-1] / ev[0]
    assert kappa * (1 - 5e-3) <= k_est <= kappa * (1 + 1e-9)


def test_multigrid_preconditioned_kappa_stays_bounded():
    # K_X optimal (Thm. 3.1): kappa does not grow with the levels (an observed plateau)
    ks = []
    for K, J in [(2, 2), (3, 3), (4, 4), (4, 6)]:
        p = schur.Problem(K, J)
        _, info = schur.pcg(p.apply_Shat, p.apply_KX, _rand(p, 3), tol=1e-14, maxit=100)
        ks.append(schur.lanczos_kappa(info["alpha"], info["beta"])[0])
    assert max(ks) < 10.0, ks


def test_pcg_matches_dense_solve():
    # config-1 sizes: K = 3, J = 4, manufactured forcing; dense Cholesky of the materialised S_hat
    p = schur.Problem(3, 4)
    g, u0, _ = inputs.manufactured(3, 4)
    fhat = p.rhs_hat(g, u0)
    Sh = schur.dense(p.apply_Shat, (p.Nt, p.Nx))
    w_dense = sl.cho_solve(sl.cho_factor(0.5 * (Sh + Sh.T)), fhat.reshape(-1)).reshape(fhat.shape)
    w, info = schur.pcg(p.apply_Shat, p.apply_KX, fhat, tol=1e-13)
    assert info["converged"]
    assert np.abs(w - w_dense).max() <= 1e-11 * np.abs(w_dense).max()


def test_rhs_route_i_equals_reduced_form():
    # f = B^T K_Y (N kron M) g + u_0 equals (L^T kron MKM + M_t kron AKM) g + e_0 kron M u0
    p = schur.Problem(3, 3)
    g, u0, _ = inputs.manufactured(3, 3)
    f = p.rhs(g, u0)
    M, A = p.Mx, p.Ax
    Gm = schur.rows(M, g)
    f2 = p.L.T @ schur.rows(M, p.K_rows(Gm)) + p.Mt @ schur.rows(A, p.K_rows(Gm))
    f2[0] += M @ u0
    assert np.abs(f - f2).max() <= 1e-13 * np.abs(f).max()


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_manufactured_solution_converges(domain):
    # quasi-optimality (Thm. 2.2): the discrete L2(I;H^1_0) distance to the nodal interpolant of
    # u = (1+t^2) sin(k pi x) sin(k pi y) falls at least linearly as K = J grow together
    errs = []
    for L in (2, 3, 4, 5) if domain == space.SQUARE else (3, 4, 5):
        p = schur.Problem(L, L, domain)
        g, u0, u = inputs.manufactured(L, L, domain)
        uh, _, info = schur.solve(p, g, u0, tol=1e-11)
        e = uh - u
        errs.append(np.sqrt(np.sum(e * (p.Mt @ schur.rows(p.Ax, e)))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 0.9, (errs, rates)


def _golden_table_5_3():
    rows = []
    with open(os.path.join(GOLDEN, "table_5_3_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                rows.append((int(a), int(b)))
    return dict(rows)


@pytest.mark.parametrize("J", [3, 4])
def test_table_5_3_iterations_with_direct_inverses(J):
    # Sec. 5.2, Table 5.3 (N_x = 261121): PCG iterations to eps = 1e-6 in the K_X-norm, absolute,
    # for u = exp(-2 pi^2 t) sin(pi x) sin(pi y), g = 0.  With the direct inverses of Sec. 5.1 in
    # place of the multigrid (whose smoother the paper does not define) the oracle takes the
    # printed 8 and 11 iterations at N_t = 9 and 17 at K = 7, 8 and 9 (tests/golden/
    # table_5_3_oracle.txt holds K = 9); the window allows one more.  At K <= 6 the last iterate
    # misses 1e-6 by a small factor (9 at K = 6, N_t = 9).
    paper = _golden_table_5_3()[2 ** J + 1]
    p = schur.Problem(7, J, inverses="direct")
    g, u0, _ = inputs.decaying(7, J)
    _, _, info = schur.solve(p, g, u0, tol=1e-6, tol_mode="abs")
    assert paper <= info["iters"] <= paper + 1, (J, info["iters"], paper)


def test_table_5_3_direct_inverses_at_the_papers_space_level():
    # the stored K = 9 oracle counts (tests/golden/make_table_5_3_oracle.py): direct inverses within
    # one of Table 5.3 at every stored N_t, equal at N_t = 9 and 17
    paper = _golden_table_5_3()
    path = os.path.join(GOLDEN, "table_5_3_oracle.txt")
    if not os.path.exists(path):
        pytest.skip("table_5_3_oracle.txt not generated")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            Nt, direct = int(f[0]), int(f[4])
            assert paper[Nt] <= direct <= paper[Nt] + 1, (Nt, direct, paper[Nt])
            if Nt in (9, 17):
                assert direct == paper[Nt], (Nt, direct)


def test_inplace_layout_roundtrip():
    p = schur.Problem(2, 4)
    Wc = _rand(p, 5)
    assert np.array_equal(p.from_inplace(p.to_inplace(Wc)), Wc)
