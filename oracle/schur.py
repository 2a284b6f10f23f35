"""Schur-complement operator, preconditioner, right-hand side and PCG of the oracle.

Test infrastructure only: see the package docstring.

State layout: a space-time coefficient vector is an array U of shape (N_t, N_x);
row i belongs to time basis function i (single-scale) or to wavelet coordinate i
(paper order c_0, d_0, ..., d_{J-1}, Sec. 3.3), and column p to spatial node p.
For a Kronecker product, (B_t kron B_x) vec(U) is B_t U B_x^T (Eq. 5.1 read
row-wise), i.e. B_x applied to every row followed by B_t across rows.

* Lemma 4.1 (route i):  S = B^T K_Y B + Gamma_0 kron M_x, B = T kron M_x + N kron A_x,
  K_Y = O^-1 kron K_x (Sec. 3.1).
* Lemma 4.2 (route ii): S = A_t kron MKM + M_t kron AKA + L^T kron MKA + L kron AKM
  + Gamma_0 kron M (five Kronecker terms, each applied as written).
* Sec. 3.4: S_hat = W^T S W, f_hat = W^T f, W = W_t kron Id, u = W w.
* Thm. 3.1 with the alpha of Sec. 5.1: K_X = blockdiag[K_|l| A_x K_|l|], with
  K_j ~ (alpha A_x + 2^j M_x)^-1.
* Lemma 4.1: f = B^T K_Y g + u_0.  The paper leaves the quadrature of g and u_0
  open; reading used: g is interpolated in P1 (x) P1 at the space-time nodes
  and u_0 in P1, so g_vec = (N kron M_x) g_nodal and u_0-vector =
  e_0 kron M_x u0_nodal.
* Sec. 3.4, Eq. (3.3): PCG on S_hat w = f_hat with K_X, from w_0 = 0, monitoring
  r^T K_X r.  Stopping: absolute (sqrt(r^T K_X r) <= eps, as in Sec. 5.2) or
  relative to the initial value (this project's default for its workloads).
* Sec. 4.4 (complexity with nested iteration, after Hackbusch Ch. 5): solve on a
  hierarchy of meshes refined in space and time together, each solve started from
  the previous level's solution and stopped at an algebraic error proportional to
  the discretisation error.  The paper gives no details; readings used here:
  levels (K - m, J - m) for m = levels-1 .. 0; the data g, u_0 of a coarse level are
  the fine nodal values at the coarse nodes; the previous solution enters the next
  level exactly (the coarse wavelet basis is the first 2^(J-1) + 1 functions of the
  fine one, Eq. 3.1 with zero new details, and the coarse P1 space in x is a subspace
  of the fine one); level m stops when sqrt(r^T K_X r) <= eps 2^(rate m) (Eq. 3.3,
  absolute), eps being the finest level's tolerance and 2^rate the expected ratio of
  discretisation errors between consecutive levels.
"""
from __future__ import annotations

import numpy as np

from . import space, time as tmod


def rows(Bx, U):
    """Apply the spatial matrix Bx to every row of U."""
    return np.asarray((Bx @ U.T).T)


class Problem:
    """The discrete problem of Sec. 5 on mesh level K, time level J: the heat equation, or with
    D (2 x 2 symmetric positive definite) and c >= 0 the reaction-diffusion equation of Sec. 4,
    whose A_x = <D grad, grad> + c M_x enters S, f and every K (Lemma 4.1, Thm. 3.1)."""

    def __init__(self, K: int, J: int, domain: int = space.SQUARE, alpha: float = 0.3,
                 n_cycles: int = 2, n_pre: int = 3, n_post: int = 3, inverses: str = "mg",
                 D=None, c: float = 0.0):
        if J < 1:
            raise ValueError("time level must be >= 1")
        self.K, self.J, self.domain, self.alpha = K, J, domain, alpha
        self.D = None if D is None else np.asarray(D, dtype=np.float64).reshape(2, 2)
        self.c = float(c)
        self.mesh = space.make_mesh(K, domain)
        self.Mx = space.mass_matrix(self.mesh)
        self.Ax = space.operator_matrix(self.mesh, self.D, self.c)
        tm = tmod.time_matrices(J)
        self.Mt, self.At, self.L = tm["Mt"], tm["At"], tm["L"]
        self.T, self.Nm, self.O, self.Gamma0 = tm["T"], tm["N"], tm["O"], tm["Gamma0"]
        self.Nt = 2 ** J + 1
        self.Nx = self.mesh.N
        self.W = tmod.wavelet_matrix(J)
        self.levels = tmod.wavelet_levels(J)
        self.perm = tmod.inplace_permutation(J)

        def make(a, s):
            if inverses == "mg":
                return space.Multigrid(K, domain, a, s, n_cycles, n_pre, n_post, self.D, self.c)
            if inverses == "direct":
                return space.DirectInverse(K, domain, a, s, self.D, self.c)
            raise ValueError(inverses)

        # K_x ~ A_x^-1 inside K_Y (Sec. 3.1); K_l ~ (alpha A_x + 2^l M_x)^-1 inside K_X
        self.Kx = make(1.0, 0.0)
        self.Kl = {l: make(alpha, 2.0 ** l) for l in range(J + 1)}

    # -- spatial preconditioner on rows -------------------------------------------------
    def K_rows(self, U):
        return self.Kx.apply(np.asarray(U).T).T

    # -- Lemma 4.1, route (i) -------------------------------------------------------------
    def apply_B(self, U):
        return self.T @ rows(self.Mx, U) + self.Nm @ rows(self.Ax, U)

    def apply_BT(self, V):
        return self.T.T @ rows(self.Mx, V) + self.Nm.T @ rows(self.Ax, V)

    def apply_KY(self, V):
        return np.linalg.solve(self.O, self.K_rows(V))

    def apply_S_route1(self, U):
        return self.apply_BT(self.apply_KY(self.apply_B(U))) + self.Gamma0 @ rows(self.Mx, U)

    # -- Lemma 4.2, route (ii) ------------------------------------------------------------
    def apply_S_route2(self, U):
        M, A = self.Mx, self.Ax
        out = self.At @ rows(M, self.K_rows(rows(M, U)))
        out = out + self.Mt @ rows(A, self.K_rows(rows(A, U)))
        out = out + self.L.T @ rows(M, self.K_rows(rows(A, U)))
        out = out + self.L @ rows(A, self.K_rows(rows(M, U)))
        out = out + self.Gamma0 @ rows(M, U)
        return out

    apply_S = apply_S_route2

    # -- wavelet coordinates (Sec. 3.3-3.4) -----------------------------------------------
    def synth(self, Wc):
        """u = W w (paper-order wavelet rows -> single-scale rows)."""
        return self.W @ Wc

    def analysis(self, U):
        """W^T u."""
        return self.W.T @ U

    def apply_Shat(self, Wc):
        return self.analysis(self.apply_S(self.synth(Wc)))

    def apply_KX(self, R):
        """K_X r = blockdiag[K_l A_x K_l] r, block l = |lambda| of each wavelet row (Thm. 3.1)."""
        Z = np.zeros_like(R)
        for l in range(self.J + 1):
            sel = self.levels == l
            if not sel.any():
                continue
            Kl = self.Kl[l]
            Y = Kl.apply(R[sel].T)
            Z[sel] = Kl.apply(self.Ax @ Y).T
        return Z

    # -- right-hand side (Lemma 4.1) ------------------------------------------------------
    def rhs(self, g_nodal, u0_nodal):
        """f = B^T K_Y g + u_0 with g_vec = (N kron M_x) g_nodal, u_0 = e_0 kron M_x u0."""
        gvec = self.Nm @ rows(self.Mx, g_nodal)
        f = self.apply_BT(self.apply_KY(gvec))
        f[0] += self.Mx @ u0_nodal
        return f

    def rhs_hat(self, g_nodal, u0_nodal):
        return self.analysis(self.rhs(g_nodal, u0_nodal))

    # -- layout helpers -------------------------------------------------------------------
    def to_inplace(self, Wc):
        """Paper-order wavelet rows -> in-place (lifting) row order."""
        out = np.empty_like(Wc)
        out[self.perm] = Wc
        return out

    def from_inplace(self, Wi):
        return Wi[self.perm]


def pcg(apply_A, apply_P, b, tol=1e-10, tol_mode="rel", maxit=500, x0=None):
    """Preconditioned CG (Hestenes-Stiefel), monitoring rho = r^T P r (Eq. 3.3).

    Stops when sqrt(rho_k) <= tol (tol_mode 'abs', the paper's rule with eps = tol)
    or sqrt(rho_k / rho_0) <= tol (tol_mode 'rel').  Returns (x, info) where info
    has the iteration count, the rho history and the CG coefficients alpha, beta.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    z = apply_P(r)
    rho = float(np.vdot(r, z))
    rho0 = rho
    hist = [rho]
    alphas, betas = [], []
    p = z.copy()
    it = 0
    converged = (np.sqrt(rho) <= tol) if tol_mode == "abs" else (rho == 0.0)
    while not converged and it < maxit:
        q = apply_A(p)
        pq = float(np.vdot(p, q))
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        z = apply_P(r)
        rho_new = float(np.vdot(r, z))
        beta = rho_new / rho
        alphas.append(alpha)
        betas.append(beta)
        hist.append(rho_new)
        it += 1
        rho = rho_new
        if tol_mode == "abs":
            converged = np.sqrt(rho) <= tol
        else:
            converged = np.sqrt(rho / rho0) <= tol
        if not converged:
            p = z + beta * p
    return x, dict(iters=it, rho=hist, alpha=alphas, beta=betas, converged=bool(converged))


def lanczos_kappa(alphas, betas):
    """Condition estimate of P A from the CG coefficients (the Lanczos tridiagonal)."""
    k = len(alphas)
    Tm = np.zeros((k, k))
    for j in range(k):
        Tm[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            Tm[j, j + 1] = Tm[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(Tm)
    return ev[-1] / ev[0], ev


def dense(apply, shape):
    """Materialise a linear operator on arrays of `shape` column by column (tiny sizes only)."""
    n = int(np.prod(shape))
    out = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        out[:, j] = apply(e.reshape(shape)).reshape(-1)
        e[j] = 0.0
    return out


def solve(prob: Problem, g_nodal, u0_nodal, tol=1e-10, tol_mode="rel", maxit=500):
    """Full solve: f_hat, PCG on S_hat w = f_hat with K_X, u = W w.  Wavelet rows in paper order."""
    fhat = prob.rhs_hat(g_nodal, u0_nodal)
    w, info = pcg(prob.apply_Shat, prob.apply_KX, fhat, tol=tol, tol_mode=tol_mode, maxit=maxit)
    return prob.synth(w), w, info


# -- nested iteration (Sec. 4.4) ------------------------------------------------------------
def inject_nodal(fine: Problem, coarse: Problem, V):
    """Nodal values on the coarse space-time mesh of a function given by its fine nodal values V
    (N_t x N_x, or N_x): time node i of the coarse mesh is fine node 2i, space grid node (i, j)
    is fine grid node (2i, 2j)."""
    assert fine.K == coarse.K + 1 and fine.J == coarse.J + 1 and fine.domain == coarse.domain
    if fine.domain == space.CUBE:
        fi = fine.mesh.dof[2 * coarse.mesh.node_k, 2 * coarse.mesh.node_j, 2 * coarse.mesh.node_i]
    else:
        fi = fine.mesh.dof[2 * coarse.mesh.node_j, 2 * coarse.mesh.node_i]
    V = np.asarray(V, dtype=np.float64)
    return V[::2][:, fi] if V.ndim == 2 else V[fi]


def prolong_wavelet(coarse: Problem, fine: Problem, Wc):
    """The coarse solution (wavelet coordinates, paper order) as a fine-level vector: the first
    2^(J-1) + 1 fine wavelets are the coarse ones, the new details get 0; in x the coarse P1
    function is written in the fine basis (prolongation P)."""
    P = space.prolongation(coarse.mesh, fine.mesh)
    Wf = np.zeros((fine.Nt, fine.Nx))
    Wf[:coarse.Nt] = rows(P, Wc)
    return Wf


def nested_solve(K, J, levels, g_nodal, u0_nodal, eps, rate=1.0, domain=space.SQUARE, D=None, c=0.0,
                 maxit=500):
    """Nested iteration over the meshes (K - m, J - m), m = levels-1 .. 0, with level tolerances
    eps 2^(rate m) (absolute, Eq. 3.3).  Returns (u, w, iterations per level, coarsest first)."""
    if levels < 1 or K - levels + 1 < space.coarsest_level(domain) or J - levels + 1 < 1:
        raise ValueError("too many nested levels for this mesh")
    probs = [Problem(K - m, J - m, domain, D=D, c=c) for m in range(levels - 1, -1, -1)]
    data = [None] * levels
    data[-1] = (np.asarray(g_nodal, dtype=np.float64), np.asarray(u0_nodal, dtype=np.float64))
    for l in range(levels - 2, -1, -1):
        gf, uf = data[l + 1]
        data[l] = (inject_nodal(probs[l + 1], probs[l], gf), inject_nodal(probs[l + 1], probs[l], uf))
    w, its = None, []
    for l, p in enumerate(probs):
        m = levels - 1 - l
        fhat = p.rhs_hat(*data[l])
        x0 = None if w is None else prolong_wavelet(probs[l - 1], p, w)
        w, info = pcg(p.apply_Shat, p.apply_KX, fhat, tol=eps * 2.0 ** (rate * m), tol_mode="abs",
                      maxit=maxit, x0=x0)
        its.append(info["iters"])
    return probs[-1].synth(w), w, its
