"""Temporal discretisation and the three-point wavelet transform of the oracle.

Test infrastructure only: see the package docstring.

* Sec. 5.1: I = (0, 1) split uniformly into 2^J intervals; X_t = H^1 ∩ P1 with
  the nodal (hat) basis Phi_t, N_t = 2^J + 1.
* Lemma 4.2: M_t = <Phi, Phi>, A_t = <Phi', Phi'>, L = <Phi', Phi> with
  L[i, j] = int Phi_j' Phi_i (the first argument of <.,.> is the column index,
  as for T and N in Lemma 4.1).
* Lemma 4.1: Y_t = DG-P1 with the piecewise shifted Legendre basis Xi (1 and
  2s - 1 on each interval, Sec. 4), O = <Xi, Xi>, T = <Phi', Xi>, N = <Phi, Xi>,
  Gamma_0 = Phi(0) Phi(0)^T.
  All of these are computed by 2-point Gauss quadrature per interval, which is
  exact for the polynomial degrees involved.
* Sec. 3.3, Eq. (3.1): W_J = M_{J-1} diag(W_{J-1}, Id), W_0 = Id, M_j = [P_j | Q_j],
  mapping wavelet coordinates (c_0, d_0, ..., d_{J-1}) to single-scale ones.
  P_j holds the level-j hats written in level-(j+1) hats (evaluated at the fine
  nodes).  The paper names the three-point wavelet of Sec. 5 but does not write
  it out.  Reading used: the level-(j+1) wavelet attached to odd fine node
  2k+1 is
      psi = 2^((j+1)/2) * (phi_{2k+1} - a_L phi_{2k} - a_R phi_{2k+2}),
  a = 1/2 next to an interior even node and a = 1 next to a boundary node, which
  is the choice that gives every wavelet a vanishing integral; d_j carries
  level |lambda| = j + 1 and c_0 level 0.  This reading reproduces the printed
  condition numbers of Table 5.1 to within 1% (checked by the tests).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_GX = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])   # Gauss points on [0,1]
_GW = np.array([0.5, 0.5])


def nodes(J: int) -> np.ndarray:
    return np.arange(2 ** J + 1) / 2.0 ** J


def _hat_local(s):
    """The two hats restricted to an interval, in local coordinate s in [0,1]: (left, right)."""
    return np.array([1.0 - s, s])


def _hat_local_dt(h):
    return np.array([-1.0 / h, 1.0 / h])


def time_matrices(J: int):
    """Return dict with M_t, A_t, L (N_t x N_t), T, N (2(N_t-1) x N_t), O, Gamma0."""
    n_int = 2 ** J
    Nt = n_int + 1
    h = 1.0 / n_int
    Mt = np.zeros((Nt, Nt))
    At = np.zeros((Nt, Nt))
    L = np.zeros((Nt, Nt))
    T = np.zeros((2 * n_int, Nt))
    N = np.zeros((2 * n_int, Nt))
    O = np.zeros((2 * n_int, 2 * n_int))
    for e in range(n_int):
        idx = [e, e + 1]
        dphi = _hat_local_dt(h)
        for q in range(2):
            s = _GX[q]
            w = _GW[q] * h
            phi = _hat_local(s)
            xi = np.array([1.0, 2.0 * s - 1.0])
            for a in range(2):
                for b in range(2):
                    Mt[idx[a], idx[b]] += w * phi[a] * phi[b]
                    At[idx[a], idx[b]] += w * dphi[a] * dphi[b]
                    # L[i, j] = int Phi_j' Phi_i
                    L[idx[a], idx[b]] += w * dphi[b] * phi[a]
                for m in range(2):
                    T[2 * e + m, idx[a]] += w * dphi[a] * xi[m]
                    N[2 * e + m, idx[a]] += w * phi[a] * xi[m]
            for m in range(2):
                for m2 in range(2):
                    O[2 * e + m, 2 * e + m2] += w * xi[m] * xi[m2]
    G0 = np.zeros((Nt, Nt))
    G0[0, 0] = 1.0        # Phi(0) = e_0
    return dict(Mt=Mt, At=At, L=L, T=T, N=N, O=O, Gamma0=G0, h=h)


def _P_matrix(j: int) -> sp.csr_matrix:
    """P_j: level-j hats in terms of level-(j+1) hats, P[f, c] = phi^j_c(t^{j+1}_f)."""
    nc = 2 ** j + 1
    nf = 2 ** (j + 1) + 1
    tf = np.arange(nf) / 2.0 ** (j + 1)
    tc = np.arange(nc) / 2.0 ** j
    hc = 1.0 / 2 ** j
    vals = np.maximum(0.0, 1.0 - np.abs(tf[:, None] - tc[None, :]) / hc)
    return sp.csr_matrix(vals)


def _Q_matrix(j: int) -> sp.csr_matrix:
    """Q_j: level-(j+1) three-point wavelets in terms of level-(j+1) hats."""
    nf = 2 ** (j + 1) + 1
    nw = 2 ** j
    scale = 2.0 ** ((j + 1) / 2.0)
    Q = np.zeros((nf, nw))
    for k in range(nw):
        left, mid, right = 2 * k, 2 * k + 1, 2 * k + 2
        a_left = 1.0 if left == 0 else 0.5
        a_right = 1.0 if right == nf - 1 else 0.5
        Q[mid, k] = scale
        Q[left, k] = -scale * a_left
        Q[right, k] = -scale * a_right
    return sp.csr_matrix(Q)


def wavelet_matrix(J: int) -> sp.csr_matrix:
    """W_t = W_J of Eq. (3.1), columns in the order (c_0, d_0, d_1, ..., d_{J-1})."""
    W = sp.identity(2, format="csr")
    for j in range(J):
        Mj = sp.hstack([_P_matrix(j), _Q_matrix(j)], format="csr")
        nd = 2 ** j
        W = (Mj @ sp.block_diag([W, sp.identity(nd)], format="csr")).tocsr()
    return W


def wavelet_levels(J: int) -> np.ndarray:
    """|lambda| of each wavelet coordinate, paper order: c_0 -> 0, d_j -> j + 1."""
    lev = [0, 0]
    for j in range(J):
        lev += [j + 1] * (2 ** j)
    return np.array(lev, dtype=np.int64)


def inplace_permutation(J: int) -> np.ndarray:
    """perm[m] = row of the in-place (lifting) layout that holds paper-order coordinate m.

    In the in-place layout c_0 sits at rows 0 and 2^J, and d_j[k] sits at the row of
    its fine node, (2k + 1) * 2^(J - j - 1).
    """
    perm = [0, 2 ** J]
    for j in range(J):
        stride = 2 ** (J - j - 1)
        perm += [(2 * k + 1) * stride for k in range(2 ** j)]
    return np.array(perm, dtype=np.int64)
