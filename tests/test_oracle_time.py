"""Pins of the oracle's time matrices and three-point wavelet transform."""
import numpy as np
import pytest

from oracle import time as tm


@pytest.mark.parametrize("J", [1, 2, 4])
def test_time_matrices_closed_forms(J):
    t = tm.time_matrices(J)
    h = 1.0 / 2 ** J
    Nt = 2 ** J + 1
    one = np.ones(Nt)
    # int Phi_i: h/2 at the ends, h inside
    expect = np.full(Nt, h)
    expect[[0, -1]] = h / 2
    np.testing.assert_allclose(t["Mt"] @ one, expect, rtol=1e-14)
    # A_t kills constants; 1^T M_t 1 = |I| = 1
    assert np.abs(t["At"] @ one).max() < 1e-12
    assert abs(one @ t["Mt"] @ one - 1.0) < 1e-14
    # integration by parts: L + L^T = e_N e_N^T - e_0 e_0^T
    D = np.zeros((Nt, Nt))
    D[0, 0], D[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(t["L"] + t["L"].T, D, atol=1e-15)
    # L[i, j] = int Phi_j' Phi_i: with t (interpolated exactly), int t' Phi_i = int Phi_i
    tn = tm.nodes(J)
    np.testing.assert_allclose(t["L"] @ tn, expect, rtol=1e-13)
    # O = diag(h, h/3) for the Legendre basis 1, 2s-1
    np.testing.assert_allclose(np.diag(t["O"]), np.tile([h, h / 3], 2 ** J), rtol=1e-14)
    assert np.abs(t["O"] - np.diag(np.diag(t["O"]))).max() < 1e-16


@pytest.mark.parametrize("J", [1, 3, 5])
def test_lemma_4_2_time_identities(J):
    # the proof of Lemma 4.2: T^T O^-1 N = L^T, N^T O^-1 N = M_t, T^T O^-1 T = A_t
    t = tm.time_matrices(J)
    Oi = np.linalg.inv(t["O"])
    np.testing.assert_allclose(t["T"].T @ Oi @ t["N"], t["L"].T, atol=1e-13)
    np.testing.assert_allclose(t["N"].T @ Oi @ t["N"], t["Mt"], atol=1e-15)
    np.testing.assert_allclose(t["T"].T @ Oi @ t["T"], t["At"], atol=1e-10 * 2 ** J)


@pytest.mark.parametrize("J", [1, 2, 3, 6])
def test_wavelet_transform_structure(J):
    W = tm.wavelet_matrix(J).toarray()
    Nt = 2 ** J + 1
    t = tm.time_matrices(J)
    lev = tm.wavelet_levels(J)
    assert W.shape == (Nt, Nt)
    # invertible: solve round trip
    x = np.random.default_rng(J).standard_normal(Nt)
    np.testing.assert_allclose(np.linalg.solve(W, W @ x), x, rtol=1e-12, atol=1e-12)
    # c_0 = (1, 1) is the constant function
    np.testing.assert_allclose(W[:, :2].sum(1), 1.0, rtol=1e-15)
    # every wavelet (|lambda| >= 1) has a vanishing integral
    mom = np.ones(Nt) @ t["Mt"] @ W
    assert np.abs(mom[lev >= 1]).max() < 1e-14
    # uniformly local: a level-l wavelet is supported on 3 fine hats of level l
    for m in np.nonzero(lev >= 1)[0]:
        l = lev[m]
        nz = np.nonzero(W[:, m])[0]
        assert nz.max() - nz.min() <= 4 * 2 ** (J - l)
    # L2-normalised scaling: a wavelet's largest single-scale coefficient is 2^(|lambda|/2)
    for m in np.nonzero(lev >= 1)[0]:
        assert abs(np.abs(W[:, m]).max() - 2.0 ** (lev[m] / 2.0)) < 1e-13


def test_wavelet_inplace_permutation():
    for J in (1, 3, 5):
        perm = tm.inplace_permutation(J)
        lev = tm.wavelet_levels(J)
        assert sorted(perm.tolist()) == list(range(2 ** J + 1))
        # in-place row i carries level 0 at the two ends and J - ctz(i) elsewhere
        for m, row in enumerate(perm.tolist()):
            if row in (0, 2 ** J):
                assert lev[m] == 0
            else:
                ctz = (row & -row).bit_length() - 1
                assert lev[m] == J - ctz
        # the wavelet of in-place row i is centred on time node i
        W = tm.wavelet_matrix(J).toarray()
        for m, row in enumerate(perm):
            if lev[m] >= 1:
                assert np.argmax(W[:, m]) == row
