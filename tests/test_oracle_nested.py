"""Pins of the oracle's nested iteration (Sec. 4.4, after Hackbusch Ch. 5).

* Injection of nodal data onto the coarser mesh equals sampling the function there.
* The prolongation of a coarse solution is exact: the fine synthesis of the prolongated wavelet
  coefficients is the space-time P1 interpolation of the coarse solution, written here from the
  midpoint rule (coarse values at coarse nodes, averages of the two end points at the midpoints
  of coarse time intervals and of horizontal, vertical and (1,1)-diagonal coarse edges).
* One level is plain PCG from zero with the absolute stopping rule.
* The returned solution meets the finest level's stopping rule, its error to the exact solution
  is the discretisation error, and the finest level needs only a few iterations (the point of
  nested iteration) where a cold start needs about thirty.
"""
import numpy as np
import pytest

from oracle import schur, space
from paper_2009_08875_gb300 import inputs


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_injection_equals_sampling(domain):
    K, J = 5, 4
    fine, coarse = schur.Problem(K, J, domain), schur.Problem(K - 1, J - 1, domain)
    g_f, u0_f, u_f = inputs.manufactured(K, J, domain)
    g_c, u0_c, u_c = inputs.manufactured(K - 1, J - 1, domain)
    assert np.array_equal(schur.inject_nodal(fine, coarse, g_f), g_c)
    assert np.array_equal(schur.inject_nodal(fine, coarse, u0_f), u0_c)
    assert np.array_equal(schur.inject_nodal(fine, coarse, u_f), u_c)


def _p1_interpolate(coarse, fine, Uc):
    """Space-time P1 interpolation of nodal values Uc (coarse mesh) at the fine nodes, by the
    midpoint rule."""
    # time: coarse node i is fine node 2i, fine node 2i+1 is the midpoint
    Ut = np.zeros((fine.Nt, coarse.Nx))
    Ut[0::2] = Uc
    Ut[1::2] = 0.5 * (Uc[:-1] + Uc[1:])
    # space: value of the coarse function at fine grid node (i, j)
    mc = coarse.mesh.m
    full = np.zeros((fine.Nt, mc + 1, mc + 1))            # coarse grid incl. boundary (zeros)
    full[:, coarse.mesh.node_j, coarse.mesh.node_i] = Ut
    out = np.zeros((fine.Nt, fine.Nx))
    for q, (i, j) in enumerate(zip(fine.mesh.node_i, fine.mesh.node_j)):
        a = (i // 2, j // 2)
        b = ((i + 1) // 2, (j + 1) // 2)   # = a at even-even nodes; the other end of the edge
        out[:, q] = 0.5 * (full[:, a[1], a[0]] + full[:, b[1], b[0]])
    return out


@pytest.mark.parametrize("domain", [space.SQUARE, space.LSHAPE])
def test_prolongation_is_p1_interpolation(domain):
    K, J = 4, 3
    fine, coarse = schur.Problem(K, J, domain), schur.Problem(K - 1, J - 1, domain)
    Wc = np.random.default_rng(2).standard_normal((coarse.Nt, coarse.Nx))
    Uf = fine.synth(schur.prolong_wavelet(coarse, fine, Wc))
    Uexpect = _p1_interpolate(coarse, fine, coarse.synth(Wc))
    assert np.abs(Uf - Uexpect).max() <= 1e-13 * np.abs(Uexpect).max()


def test_one_level_is_plain_pcg():
    K, J = 4, 4
    p = schur.Problem(K, J)
    g, u0, _ = inputs.manufactured(K, J)
    u1, w1, its = schur.nested_solve(K, J, 1, g, u0, 1e-4)
    w2, info = schur.pcg(p.apply_Shat, p.apply_KX, p.rhs_hat(g, u0), tol=1e-4, tol_mode="abs")
    assert its == [info["iters"]]
    assert np.array_equal(w1, w2)


@pytest.mark.parametrize("L", [4, 5, 6])
def test_nested_reaches_discretisation_accuracy_in_few_iterations(L):
    K = J = L
    eps = 1e-3
    p = schur.Problem(K, J)
    g, u0, u = inputs.manufactured(K, J)
    un, wn, its = schur.nested_solve(K, J, 3, g, u0, eps)
    # the finest level's stopping rule holds
    r = p.rhs_hat(g, u0) - p.apply_Shat(wn)
    assert np.sqrt(np.sum(r * p.apply_KX(r))) <= eps
    # error to the exact solution = the discretisation error (within 10 %)
    uex, _, info = schur.solve(p, g, u0, tol=1e-13)
    A = space.stiffness_matrix(p.mesh)

    def xerr(e):
        return np.sqrt(np.sum(e * (p.Mt @ schur.rows(A, e))))

    assert abs(xerr(un - u) - xerr(uex - u)) <= 0.1 * xerr(uex - u)
    # few iterations on the finest level, where the cold start needs many
    assert its[-1] <= 8 and info["iters"] >= 25
