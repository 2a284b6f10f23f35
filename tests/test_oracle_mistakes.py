"""Planted mistakes: each test breaks one piece of the oracle the way an implementation plausibly
could (a transposed or negated term, a dropped term, a wrong shift or level), on CPU, and checks
that one of the pins that guard the oracle rejects it.  The unbroken oracle passes the same pins
in test_oracle_schur.py.
"""
import numpy as np

from oracle import schur, space

KAPPA_65_49 = 6.34  # Sec. 5.1, Table 5.1: N_t = 65, N_x = 49, direct inverses, alpha = 0.3


def _rand(p, seed):
    return np.random.default_rng(seed).standard_normal((p.Nt, p.Nx))


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _kappa(p):
    _, info = schur.pcg(p.apply_Shat, p.apply_KX, _rand(p, 1), tol=1e-15, maxit=150)
    return schur.lanczos_kappa(info["alpha"], info["beta"])[0]


def test_transposed_or_negated_L_breaks_lemma_4_1_equals_4_2():
    # Lemma 4.2's cross terms are L^T kron M K A and L kron A K M; route (i) does not use L.
    # Transposing L changes S by (L^T - L) kron (M K A - A K M), which vanishes for K = A^-1 and is
    # of the size of the multigrid's error otherwise: far above the pin's 1e-13, as is a sign error
    for mutate, floor in ((lambda L: L.T.copy(), 1e-6), (lambda L: -L, 1e-3)):
        p = schur.Problem(3, 3)
        U = _rand(p, 7)
        s1 = p.apply_S_route1(U)
        assert _rel(p.apply_S_route2(U), s1) <= 1e-13
        p.L = mutate(p.L)
        assert _rel(p.apply_S_route2(U), s1) > floor


def test_dropped_initial_trace_term_breaks_the_closed_form():
    # without Gamma_0 = e_0 e_0^T (kron M) the Gram-matrix closed form of S no longer holds
    p = schur.Problem(3, 3, inverses="direct")
    M, A = p.Mx.toarray(), p.Ax.toarray()
    eN = np.zeros((p.Nt, p.Nt))
    eN[-1, -1] = 1.0
    S_closed = np.kron(p.At, M @ np.linalg.solve(A, M)) + np.kron(p.Mt, A) + np.kron(eN, M)
    assert _rel(schur.dense(p.apply_S, (p.Nt, p.Nx)), S_closed) <= 1e-13
    p.Gamma0 = 0.0 * p.Gamma0
    assert _rel(schur.dense(p.apply_S, (p.Nt, p.Nx)), S_closed) > 1e-3


def test_wrong_shift_or_level_offset_in_K_X_misses_table_5_1():
    # K_l ~ (alpha A + 2^l M)^-1 with the detail d_j on level j + 1 reproduces Table 5.1; 4^l
    # instead of 2^l, or d_j on level j, does not
    p = schur.Problem(3, 6, inverses="direct")
    assert abs(_kappa(p) - KAPPA_65_49) <= 0.01 * KAPPA_65_49
    q = schur.Problem(3, 6, inverses="direct")
    q.Kl = {l: space.DirectInverse(3, space.SQUARE, 0.3, 4.0 ** l) for l in q.Kl}
    assert abs(_kappa(q) - KAPPA_65_49) > 0.05 * KAPPA_65_49
    r = schur.Problem(3, 6, inverses="direct")
    r.levels = np.maximum(r.levels - 1, 0)
    assert abs(_kappa(r) - KAPPA_65_49) > 0.05 * KAPPA_65_49


def test_unscaled_wavelets_miss_table_5_1():
    # the detail functions carry the factor 2^((j+1)/2) of Eq. 3.1 (L2 normalisation); dropping it
    # (W's columns of level l divided by 2^(l/2)) leaves K_X mis-scaled against S_hat
    p = schur.Problem(3, 6, inverses="direct")
    scale = 2.0 ** (-0.5 * p.levels.astype(float))
    p.W = p.W @ np.diag(scale)
    assert abs(_kappa(p) - KAPPA_65_49) > 0.05 * KAPPA_65_49


class _MirroredMesh(space.Mesh):
    """The same grid with every cell cut along the other diagonal, (I+1, J)-(I, J+1)."""

    def __init__(self, level):
        super().__init__(level)
        m = self.m
        I, J = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
        I, J = I.ravel(), J.ravel()
        a = np.stack([np.stack([I, J], 1), np.stack([I + 1, J], 1), np.stack([I, J + 1], 1)], 1)
        b = np.stack([np.stack([I + 1, J], 1), np.stack([I + 1, J + 1], 1), np.stack([I, J + 1], 1)], 1)
        self.tri = np.concatenate([a, b], 0)


def test_other_diagonal_breaks_the_three_colouring():
    # the colouring (i + j) mod 3 decouples the 7-point pattern of the (1,1)-diagonal mesh (the
    # pin in test_oracle_space.py); assembled on the mirrored mesh, mass and stiffness couple
    # (i, j) with (i + 1, j - 1), which has the same colour
    for make in (lambda k: space.Mesh(k), _MirroredMesh):
        m = make(4)
        col = m.colour()
        same = []
        for Mat in (space.mass_matrix(m), space.stiffness_matrix(m)):
            C = Mat.tocoo()
            off = (C.row != C.col) & (np.abs(C.data) > 0)
            same.append(bool(np.any(col[C.row[off]] == col[C.col[off]])))
        if isinstance(m, _MirroredMesh):
            assert same[0]        # the mass matrix couples the new diagonal
        else:
            assert not any(same)


def _bilinear_prolongation(coarse, fine):
    # Q1 interpolation: a cell-centre node takes the mean of the four cell corners instead of the
    # two end points of the cell's (1,1) diagonal
    P = np.zeros((fine.N, coarse.N))
    for f, (i, j) in enumerate(zip(fine.node_i, fine.node_j)):
        x, y = i / 2.0, j / 2.0
        I, J = int(np.floor(x)), int(np.floor(y))
        for di in (0, 1):
            for dj in (0, 1):
                w = (1 - abs(x - (I + di))) * (1 - abs(y - (J + dj)))
                ci, cj = I + di, J + dj
                if w > 0 and 0 <= ci <= coarse.m and 0 <= cj <= coarse.m and coarse.dof[cj, ci] >= 0:
                    P[f, coarse.dof[cj, ci]] += w
    return P


def test_bilinear_prolongation_breaks_galerkin_exactness():
    # nested P1 spaces make P^T A_f P = A_c exact (the pin in test_oracle_space.py); Q1 weights at
    # the cell centres do not, although their column sums are the same
    c, f = space.Mesh(3), space.Mesh(4)
    Af, Ac = space.stiffness_matrix(f).toarray(), space.stiffness_matrix(c).toarray()
    P = space.prolongation(c, f).toarray()
    assert np.abs(P.T @ Af @ P - Ac).max() < 1e-13
    Q = _bilinear_prolongation(c, f)
    assert np.allclose(Q.sum(0).max(), P.sum(0).max())
    assert np.abs(Q.T @ Af @ Q - Ac).max() > 1e-2


def test_time_matrix_slips_break_the_lemma_4_2_identities():
    # M_t, A_t and L are assembled independently of the DG test-space matrices T, N, O; the proof
    # identities N^T O^-1 N = M_t, T^T O^-1 T = A_t, T^T O^-1 N = L^T tie them together.  A corner
    # of M_t at h/6 instead of h/3, A_t without its corner, or L with the wrong end sign fails them.
    from oracle import time as tm
    J = 3
    t = tm.time_matrices(J)
    Oi = np.linalg.inv(t["O"])
    h = 2.0 ** -J
    Mt, At, L = t["Mt"].copy(), t["At"].copy(), t["L"].copy()
    assert np.abs(t["N"].T @ Oi @ t["N"] - Mt).max() < 1e-15
    Mt[0, 0] = h / 6
    assert np.abs(t["N"].T @ Oi @ t["N"] - Mt).max() > 1e-3
    At[-1, -1] = 2.0 / h
    assert np.abs(t["T"].T @ Oi @ t["T"] - At).max() > 1.0
    L[0, 0] = +0.5
    assert np.abs(t["T"].T @ Oi @ t["N"] - L.T).max() > 0.5


def test_three_colours_do_not_decouple_the_cube():
    # the Kuhn mesh couples a node with index-sum offsets +-1, +-2 and +-3 (the body diagonal), so
    # (i + j + k) mod 4 separates every coupled pair and (i + j + k) mod 3 does not
    m = space.Mesh3(3)
    C = space.mass_matrix(m).tocoo()
    off = C.row != C.col
    s = m.node_i + m.node_j + m.node_k
    assert np.all(m.colour()[C.row[off]] != m.colour()[C.col[off]])
    assert np.any((s % 3)[C.row[off]] == (s % 3)[C.col[off]])


def test_shifted_injection_or_detail_placement_fail_the_nested_pins():
    # injection takes coarse time node i from fine node 2i and grid node (i, j) from (2i, 2j): the
    # odd fine nodes instead give values that are not the coarse mesh's samples; the coarse
    # solution enters the fine level as its first 2^(J-1) + 1 wavelet rows, and placing it in the
    # last rows instead is not the space-time P1 interpolation
    from paper_2009_08875_gb300 import inputs
    K, J = 5, 4
    fine, coarse = schur.Problem(K, J), schur.Problem(K - 1, J - 1)
    g_f = inputs.manufactured(K, J)[0]
    g_c = inputs.manufactured(K - 1, J - 1)[0]
    assert np.array_equal(schur.inject_nodal(fine, coarse, g_f), g_c)
    fi = fine.mesh.dof[2 * coarse.mesh.node_j, 2 * coarse.mesh.node_i]
    assert np.abs(g_f[1::2][:, fi] - g_c[:-1]).max() > 1e-2       # odd time nodes
    fi_odd = fine.mesh.dof[2 * coarse.mesh.node_j - 1, 2 * coarse.mesh.node_i - 1]
    assert np.abs(g_f[::2][:, fi_odd] - g_c).max() > 1e-2          # odd grid nodes
    # detail placement: the coarse rows go first; moving them to the end changes the function
    Wc = np.random.default_rng(2).standard_normal((coarse.Nt, coarse.Nx))
    right = fine.synth(schur.prolong_wavelet(coarse, fine, Wc))
    wrong = np.zeros((fine.Nt, fine.Nx))
    wrong[-coarse.Nt:] = schur.prolong_wavelet(coarse, fine, Wc)[:coarse.Nt]
    assert np.abs(fine.synth(wrong) - right).max() > 1e-2 * np.abs(right).max()
