"""Spatial discretisation and multigrid of the oracle (FP64, numpy / scipy.sparse).

Test infrastructure only: see the package docstring.

What is computed, and where the paper fixes it
----------------------------------------------
* Sec. 4 and Sec. 5.1: X_x = H^1_0 ∩ P1 on a uniform triangulation of the unit
  square (or of the L-shape (0,1)^2 minus [1/2,1)^2, a domain the paper does not
  use; it serves the mixed-precision workload).  Mesh level k has mesh width
  h = 2^-k and (2^k - 1)^2 interior nodes on the square (Sec. 5.1).
  Reading: the paper's "4^K triangles" is taken as 2^K x 2^K squares, each cut
  along its lower-left to upper-right diagonal, which is what the stated
  N_x = (2^K - 1)^2 requires.
* Lemma 4.1: M_x = <phi, phi>_{L2}, A_x = <D grad phi, grad phi>_{L2} + c M_x
  for the reaction-diffusion form of Sec. 4 (a constant symmetric positive
  definite 2 x 2 matrix D and a constant c >= 0; D = Id, c = 0 is the heat
  equation of Sec. 5).  Both are assembled here element by element from the P1
  element matrices; no stencil is written down.
* Sec. 5.2, the 3D problem: Omega = (0,1)^3 "triangulated uniformly into 8^K
  tetrahedra", N_x = (2^K - 1)^3.  Reading: 2^K x 2^K x 2^K cubes, each cut into the
  six tetrahedra of Kuhn's subdivision along its (0,0,0)-(1,1,1) diagonal (vertices
  0, e_a, e_a + e_b, (1,1,1) for the six orderings (a, b, c) of the axes); this mesh
  is nested under uniform refinement, so the P1 spaces are nested as in 2D.  Its edges
  run along the axes, the face diagonals (1,1,0), (1,0,1), (0,1,1) and the body
  diagonal (1,1,1), so the Gauss-Seidel colours are (i + j + k) mod 4 (offsets with
  coordinate sums +-1, +-2, +-3), pre-sweeps in colour order 0..3, post-sweeps 3..0.
* Sec. 3.1 / Thm. 3.1 / Sec. 5.1: K_x ~ A_x^-1 and K_j ~ (alpha A_x + 2^j M_x)^-1
  are "2 V-cycles with 3 Gauss-Seidel smoothing steps per grid".  The paper does
  not define the smoother ordering or the coarse grid.  Reading used here:
  - nested P1 spaces; the prolongation P_k is the natural embedding, i.e.
    P_k[f, c] = (coarse basis function c evaluated at fine node f); restriction
    is P_k^T; the coarse operator is the same bilinear form rediscretised on the
    coarse mesh (for nested P1 this is exactly P^T C P);
  - Gauss-Seidel in three colours, colour(i, j) = (i + j) mod 3 of the node's
    grid indices; 3 pre-sweeps visit colours 0, 1, 2 and 3 post-sweeps visit
    colours 2, 1, 0 (so the V-cycle, and K, are symmetric as S requires);
  - the coarsest level (1 on the square, 2 on the L-shape) is solved exactly;
  - every application starts from x = 0 and runs 2 cycles, so K is a fixed
    linear symmetric positive definite operator.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp

SQUARE = 0
LSHAPE = 1
CUBE = 2


class Mesh:
    """Uniform triangulation of level `level` of the unit square or the L-shape.

    Grid node (i, j) sits at (x, y) = (i h, j h), 0 <= i, j <= 2^level.  Active
    (degree-of-freedom) nodes are the nodes interior to the domain, numbered
    lexicographically with i (x) fastest.
    """

    def __init__(self, level: int, domain: int = SQUARE):
        if level < 1:
            raise ValueError("mesh level must be >= 1")
        self.level = level
        self.domain = domain
        self.m = 2 ** level                  # intervals per side
        self.h = 1.0 / self.m
        m = self.m
        half = m // 2
        ii, jj = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="xy")
        interior = (ii >= 1) & (ii <= m - 1) & (jj >= 1) & (jj <= m - 1)
        if domain == LSHAPE:
            # nodes with x >= 1/2 and y >= 1/2 are outside or on the boundary
            interior &= ~((ii >= half) & (jj >= half))
        self.active = interior               # shape (m+1, m+1), indexed [j, i]
        self.dof = -np.ones((m + 1, m + 1), dtype=np.int64)
        self.dof[interior] = np.arange(int(interior.sum()))
        self.N = int(interior.sum())
        self.node_i = ii[interior]
        self.node_j = jj[interior]

        # triangles: every cell (I, J) of the domain, cut along its (I,J)-(I+1,J+1) diagonal
        I, J = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
        I = I.ravel()
        J = J.ravel()
        if domain == LSHAPE:
            keep = ~((I >= half) & (J >= half))
            I, J = I[keep], J[keep]
        lower = np.stack([np.stack([I, J], 1), np.stack([I + 1, J], 1), np.stack([I + 1, J + 1], 1)], 1)
        upper = np.stack([np.stack([I, J], 1), np.stack([I + 1, J + 1], 1), np.stack([I, J + 1], 1)], 1)
        self.tri = np.concatenate([lower, upper], 0)   # (T, 3, 2) grid indices

    def coords(self):
        return self.node_i * self.h, self.node_j * self.h

    def colour(self):
        """Gauss-Seidel colour (i + j) mod 3 of every active node."""
        return (self.node_i + self.node_j) % 3

    ncolours = 3


class Mesh3:
    """Uniform Kuhn tetrahedral mesh of level `level` of the unit cube.

    Grid node (i, j, k) sits at (i h, j h, k h); active nodes are the interior ones,
    numbered lexicographically with i (x) fastest, then j, then k.
    """

    ncolours = 4

    def __init__(self, level: int):
        if level < 1:
            raise ValueError("mesh level must be >= 1")
        self.level = level
        self.domain = CUBE
        self.m = 2 ** level
        self.h = 1.0 / self.m
        m = self.m
        kk, jj, ii = np.meshgrid(np.arange(m + 1), np.arange(m + 1), np.arange(m + 1), indexing="ij")
        interior = (ii >= 1) & (ii <= m - 1) & (jj >= 1) & (jj <= m - 1) & (kk >= 1) & (kk <= m - 1)
        self.dof = -np.ones((m + 1, m + 1, m + 1), dtype=np.int64)     # indexed [k, j, i]
        self.dof[interior] = np.arange(int(interior.sum()))
        self.N = int(interior.sum())
        self.node_i, self.node_j, self.node_k = ii[interior], jj[interior], kk[interior]
        # six Kuhn tetrahedra per cell: 0 -> e_a -> e_a + e_b -> (1,1,1)
        C = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)[:, ::-1]
        E = np.eye(3, dtype=np.int64)
        tets = []
        for a, b, c in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
            v1 = E[a]
            v2 = E[a] + E[b]
            tets.append(np.stack([C, C + v1, C + v2, C + 1], 1))
        self.tet = np.concatenate(tets, 0)                              # (T, 4, 3) grid (i, j, k)

    def coords(self):
        return self.node_i * self.h, self.node_j * self.h, self.node_k * self.h

    def colour(self):
        """Gauss-Seidel colour (i + j + k) mod 4 of every active node."""
        return (self.node_i + self.node_j + self.node_k) % 4


def make_mesh(level: int, domain: int = SQUARE):
    return Mesh3(level) if domain == CUBE else Mesh(level, domain)


def _assemble(mesh, kind: str, D=None) -> sp.csr_matrix:
    """Assemble the P1 mass ('M') or stiffness ('A', <D grad, grad>) matrix over the active nodes."""
    if isinstance(mesh, Mesh3):
        return _assemble3(mesh, kind, D)
    P = mesh.tri.astype(np.float64) * mesh.h          # (T, 3, 2) vertex coordinates
    e1 = P[:, 1] - P[:, 0]
    e2 = P[:, 2] - P[:, 0]
    det = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    area = 0.5 * np.abs(det)
    if kind == "M":
        # P1 element mass matrix: |T|/12 * (1 + delta_ab)
        Ke = (area / 12.0)[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None]
    elif kind == "A":
        # gradients of the barycentric coordinates: grad lambda_a = rot(opposite edge) / (2|T|)
        grads = np.empty((P.shape[0], 3, 2))
        for a in range(3):
            b, c = (a + 1) % 3, (a + 2) % 3
            edge = P[:, c] - P[:, b]
            grads[:, a, 0] = edge[:, 1] / det
            grads[:, a, 1] = -edge[:, 0] / det
        Dm = np.eye(2) if D is None else np.asarray(D, dtype=np.float64).reshape(2, 2)
        Ke = area[:, None, None] * np.einsum("tad,de,tbe->tab", grads, Dm, grads)
    else:
        raise ValueError(kind)
    gid = mesh.dof[mesh.tri[:, :, 1], mesh.tri[:, :, 0]]   # (T, 3), -1 for Dirichlet nodes
    rows = np.repeat(gid, 3, axis=1).ravel()
    cols = np.tile(gid, (1, 3)).ravel()
    vals = Ke.reshape(-1)
    keep = (rows >= 0) & (cols >= 0)
    Mat = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(mesh.N, mesh.N)).tocsr()
    Mat.sum_duplicates()
    Mat.eliminate_zeros()
    return Mat


def _assemble3(mesh: Mesh3, kind: str, D=None) -> sp.csr_matrix:
    """P1 mass / stiffness on the tetrahedra of a Mesh3."""
    P = mesh.tet.astype(np.float64) * mesh.h                  # (T, 4, 3)
    E = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 2)   # columns = edges
    vol = np.abs(np.linalg.det(E)) / 6.0
    if kind == "M":
        # P1 element mass matrix: |T|/20 * (1 + delta_ab)
        Ke = (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
    elif kind == "A":
        # barycentric lambda_1..3 = E^-1 (x - P_0): their gradients are the rows of E^-1
        Einv = np.linalg.inv(E)
        grads = np.concatenate([-Einv.sum(1, keepdims=True), Einv], 1)          # (T, 4, 3)
        Dm = np.eye(3) if D is None else np.asarray(D, dtype=np.float64).reshape(3, 3)
        Ke = vol[:, None, None] * np.einsum("tad,de,tbe->tab", grads, Dm, grads)
    else:
        raise ValueError(kind)
    gid = mesh.dof[mesh.tet[:, :, 2], mesh.tet[:, :, 1], mesh.tet[:, :, 0]]     # (T, 4)
    rows = np.repeat(gid, 4, axis=1).ravel()
    cols = np.tile(gid, (1, 4)).ravel()
    vals = Ke.reshape(-1)
    keep = (rows >= 0) & (cols >= 0)
    Mat = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(mesh.N, mesh.N)).tocsr()
    Mat.sum_duplicates()
    Mat.eliminate_zeros()
    return Mat


def mass_matrix(mesh: Mesh) -> sp.csr_matrix:
    """M_x = <phi_q, phi_p>_{L2(Omega)} (Lemma 4.1)."""
    return _assemble(mesh, "M")


def stiffness_matrix(mesh: Mesh, D=None) -> sp.csr_matrix:
    """<D grad phi_q, grad phi_p>_{L2(Omega)} (D = Id when None)."""
    return _assemble(mesh, "A", D)


def operator_matrix(mesh: Mesh, D=None, c: float = 0.0) -> sp.csr_matrix:
    """A_x of Lemma 4.1 for the reaction-diffusion form of Sec. 4:
    <D grad phi_q, grad phi_p> + c <phi_q, phi_p>."""
    A = stiffness_matrix(mesh, D)
    if c != 0.0:
        A = (A + float(c) * mass_matrix(mesh)).tocsr()
    return A


def _prolongation3(coarse: Mesh3, fine: Mesh3) -> sp.csr_matrix:
    """P[f, c] for the Kuhn mesh: the fine node's containing coarse tetrahedron is found by
    sorting its fractional coordinates in the coarse cell (descending, x_(1) >= x_(2) >= x_(3));
    its barycentric coordinates are 1 - x_(1), x_(1) - x_(2), x_(2) - x_(3), x_(3) at the
    vertices 0, e_(1), e_(1) + e_(2), (1,1,1) of the cell."""
    X = np.stack([fine.node_i, fine.node_j, fine.node_k], 1).astype(np.float64) / 2.0
    cell = np.minimum(np.floor(X).astype(np.int64), coarse.m - 1)
    xi = X - cell
    order = np.argsort(-xi, axis=1, kind="stable")
    srt = np.take_along_axis(xi, order, 1)
    lam = np.stack([1 - srt[:, 0], srt[:, 0] - srt[:, 1], srt[:, 1] - srt[:, 2], srt[:, 2]], 1)
    verts = np.zeros((X.shape[0], 4, 3), dtype=np.int64)
    for v in range(1, 4):
        verts[:, v] = verts[:, v - 1]
        np.put_along_axis(verts[:, v], order[:, v - 1:v], 1, axis=1)
    verts += cell[:, None, :]
    cid = coarse.dof[verts[:, :, 2], verts[:, :, 1], verts[:, :, 0]]
    rows = np.repeat(np.arange(fine.N), 4)
    cols = cid.ravel()
    vals = lam.ravel()
    keep = (cols >= 0) & (vals != 0.0)
    P = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(fine.N, coarse.N)).tocsr()
    P.sum_duplicates()
    return P


def prolongation(coarse: Mesh, fine: Mesh) -> sp.csr_matrix:
    """P[f, c] = value of coarse P1 basis function c at fine node f (nested spaces)."""
    assert fine.level == coarse.level + 1 and fine.domain == coarse.domain
    if isinstance(fine, Mesh3):
        return _prolongation3(coarse, fine)
    xf = fine.node_i.astype(np.float64) / 2.0      # fine node in coarse grid units
    yf = fine.node_j.astype(np.float64) / 2.0
    I = np.minimum(np.floor(xf).astype(np.int64), coarse.m - 1)
    J = np.minimum(np.floor(yf).astype(np.int64), coarse.m - 1)
    xi = xf - I
    eta = yf - J
    lower = xi >= eta
    # barycentric coordinates in the containing coarse triangle
    # lower: (I,J),(I+1,J),(I+1,J+1) -> (1-xi, xi-eta, eta)
    # upper: (I,J),(I+1,J+1),(I,J+1) -> (1-eta, xi, eta-xi)
    vi = np.where(lower[:, None], np.stack([I, I + 1, I + 1], 1), np.stack([I, I + 1, I], 1))
    vj = np.where(lower[:, None], np.stack([J, J, J + 1], 1), np.stack([J, J + 1, J + 1], 1))
    lam = np.where(lower[:, None], np.stack([1 - xi, xi - eta, eta], 1), np.stack([1 - eta, xi, eta - xi], 1))
    cid = coarse.dof[vj, vi]
    rows = np.repeat(np.arange(fine.N), 3)
    cols = cid.ravel()
    vals = lam.ravel()
    keep = (cols >= 0) & (vals != 0.0)
    P = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(fine.N, coarse.N)).tocsr()
    P.sum_duplicates()
    return P


def coarsest_level(domain: int) -> int:
    return 2 if domain == LSHAPE else 1


class Multigrid:
    """Symmetric multigrid for C = a*A_x + s*M_x on the hierarchy coarsest..level,
    A_x = <D grad, grad> + c M_x rediscretised on every level.

    `apply(B)` returns X with each column X[:, m] = K B[:, m], where K is
    `n_cycles` V-cycles started from zero (Sec. 5.1: 2 V-cycles, 3 Gauss-Seidel
    steps per grid).  B may be (N,) or (N, m).
    """

    def __init__(self, level: int, domain: int, a: float, s: float,
                 n_cycles: int = 2, n_pre: int = 3, n_post: int = 3, D=None, c: float = 0.0):
        self.level = level
        self.domain = domain
        self.a, self.s = float(a), float(s)
        self.n_cycles, self.n_pre, self.n_post = n_cycles, n_pre, n_post
        self.k0 = coarsest_level(domain)
        if level < self.k0:
            raise ValueError("mesh level below the coarsest multigrid level")
        self.meshes = {k: make_mesh(k, domain) for k in range(self.k0, level + 1)}
        self.ncolours = self.meshes[level].ncolours
        self.C = {}
        self.diag = {}
        self.colour = {}
        self.P = {}
        for k, mesh in self.meshes.items():
            C = (self.a * operator_matrix(mesh, D, c) + self.s * mass_matrix(mesh)).tocsr()
            self.C[k] = C
            self.diag[k] = C.diagonal()
            self.colour[k] = mesh.colour()
            if k > self.k0:
                self.P[k] = prolongation(self.meshes[k - 1], mesh)
        self.coarse_dense = self.C[self.k0].toarray()

    def _gs_colour(self, k, c, x, b):
        # one Gauss-Seidel step restricted to colour c; nodes of one colour are not
        # coupled, so this equals sequential Gauss-Seidel over that colour
        sel = self.colour[k] == c
        r = b - self.C[k] @ x
        x = x.copy()
        x[sel] += r[sel] / (self.diag[k][sel] if x.ndim == 1 else self.diag[k][sel][:, None])
        return x

    def _vcycle(self, k, x, b):
        if k == self.k0:
            return scipy.linalg.solve(self.coarse_dense, b, assume_a="pos")
        for _ in range(self.n_pre):
            for c in range(self.ncolours):
                x = self._gs_colour(k, c, x, b)
        r = b - self.C[k] @ x
        bc = self.P[k].T @ r
        xc = self._vcycle(k - 1, np.zeros_like(bc), bc)
        x = x + self.P[k] @ xc
        for _ in range(self.n_post):
            for c in reversed(range(self.ncolours)):
                x = self._gs_colour(k, c, x, b)
        return x

    def apply(self, B):
        B = np.asarray(B, dtype=np.float64)
        X = np.zeros_like(B)
        for _ in range(self.n_cycles):
            X = self._vcycle(self.level, X, B)
        return X


class DirectInverse:
    """K = C^-1 exactly (sparse LU), for C = a*A_x + s*M_x (the 'direct inverses' of Sec. 5.1)."""

    def __init__(self, level: int, domain: int, a: float, s: float, D=None, c: float = 0.0):
        import scipy.sparse.linalg as spla
        mesh = make_mesh(level, domain)
        C = (a * operator_matrix(mesh, D, c) + s * mass_matrix(mesh)).tocsc()
        self._lu = spla.splu(C)

    def apply(self, B):
        return self._lu.solve(np.asarray(B, dtype=np.float64))
