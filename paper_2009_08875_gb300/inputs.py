"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only lays out problem data: it samples closed-form functions at the
space-time grid nodes and draws seeded random arrays.  It holds none of the
solver's arithmetic (no finite-element matrices, multigrid or wavelets).

Layout (the library's): a space-time array has shape (N_t, N_x); row i is time
node t_i = i / 2^J, column p is the p-th interior node of the spatial grid in
lexicographic order with x fastest.  Grid node (i, j) sits at (i h, j h),
h = 2^-K.  On the unit square the interior nodes are 1 <= i, j <= 2^K - 1; on the
L-shape (0,1)^2 minus [1/2,1)^2 the nodes with x >= 1/2 and y >= 1/2 are left out;
on the unit cube the interior nodes (i, j, k) are numbered with x fastest, then y.
"""
from __future__ import annotations

import numpy as np

SQUARE = 0
LSHAPE = 1
CUBE = 2


def dims(K: int, J: int, domain: int = SQUARE):
    n = 2 ** K - 1
    Nx = {SQUARE: n * n, LSHAPE: n * n - (2 ** (K - 1)) ** 2, CUBE: n ** 3}[domain]
    return 2 ** J + 1, Nx


def node_coords(K: int, domain: int = SQUARE):
    """(x, y) (or (x, y, z) on the cube) of the interior nodes in lexicographic order, x fastest."""
    m = 2 ** K
    if domain == CUBE:
        k, j, i = np.meshgrid(np.arange(1, m), np.arange(1, m), np.arange(1, m), indexing="ij")
        return i.ravel() / m, j.ravel() / m, k.ravel() / m
    i, j = np.meshgrid(np.arange(1, m), np.arange(1, m), indexing="xy")
    keep = np.ones_like(i, dtype=bool)
    if domain == LSHAPE:
        keep = ~((i >= m // 2) & (j >= m // 2))
    return i[keep] / m, j[keep] / m


def time_nodes(J: int):
    return np.arange(2 ** J + 1) / 2.0 ** J


def manufactured(K: int, J: int, domain: int = SQUARE, D=None, c: float = 0.0):
    """u = (1 + t^2) sin(k pi x) sin(k pi y), k = 1 on the square, 2 on the L-shape.

    Returns (g_nodal, u0_nodal, u_nodal) with g = u_t - div(D grad u) + c u sampled at the
    nodes (D = Id, c = 0: the heat equation).
    """
    t = time_nodes(J)
    if domain == CUBE:
        # u = (1 + t^2) sin(pi x) sin(pi y) sin(pi z), D = Id
        if D is not None:
            raise ValueError("the cube supports D = Id only")
        x, y, z = node_coords(K, CUBE)
        phi = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        tt = (1.0 + t[:, None] ** 2)
        g = (2.0 * t[:, None] + (3.0 * np.pi ** 2 + c) * tt) * phi[None, :]
        return g, phi.copy(), tt * phi[None, :]
    x, y = node_coords(K, domain)
    k = 1.0 if domain == SQUARE else 2.0
    d11, d12, d22 = (1.0, 0.0, 1.0) if D is None else (D[0][0], D[0][1], D[1][1])
    phi = np.sin(k * np.pi * x) * np.sin(k * np.pi * y)
    cross = np.cos(k * np.pi * x) * np.cos(k * np.pi * y)
    tt = (1.0 + t[:, None] ** 2)
    u = tt * phi[None, :]
    g = (2.0 * t[:, None] + ((d11 + d22) * (k * np.pi) ** 2 + c) * tt) * phi[None, :] \
        - 2.0 * d12 * (k * np.pi) ** 2 * tt * cross[None, :]
    return g, phi.copy(), u


def decaying(K: int, J: int, domain: int = SQUARE):
    """The workloads of the paper's scaling runs (g = 0): u = exp(-2 pi^2 t) sin(pi x) sin(pi y)
    on the square, u = exp(-3 pi^2 t) sin(pi x) sin(pi y) sin(pi z) on the cube."""
    t = time_nodes(J)
    if domain == CUBE:
        x, y, z = node_coords(K, CUBE)
        phi = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        rate = 3.0
    else:
        x, y = node_coords(K, SQUARE)
        phi = np.sin(np.pi * x) * np.sin(np.pi * y)
        rate = 2.0
    u = np.exp(-rate * np.pi ** 2 * t)[:, None] * phi[None, :]
    return np.zeros_like(u), phi.copy(), u


def smooth_forcing(K: int, J: int, seed: int, domain: int = SQUARE, modes: int = 8):
    """g = sum_m c_m cos(k_m pi t) sin(a_m pi x) sin(b_m pi y), c ~ N(0,1); u0 = 0."""
    rng = np.random.default_rng(seed)
    xyz = node_coords(K, domain)
    x, y = xyz[0], xyz[1]
    zf = np.sin(np.pi * xyz[2]) if domain == CUBE else 1.0
    t = time_nodes(J)
    c = rng.standard_normal(modes)
    a = rng.integers(1, 5, modes)
    b = rng.integers(1, 5, modes)
    kk = rng.integers(0, 4, modes)
    g = np.zeros((t.size, x.size))
    for m in range(modes):
        g += c[m] * np.cos(kk[m] * np.pi * t)[:, None] * (np.sin(a[m] * np.pi * x) * np.sin(b[m] * np.pi * y)
                                                          * zf)[None, :]
    return g, np.zeros(x.size)


def random_state(Nt: int, Nx: int, seed: int):
    """Standard-normal (N_t, N_x) array, seeded."""
    return np.random.default_rng(seed).standard_normal((Nt, Nx))


def grid_mask(K: int, domain: int = SQUARE):
    """Boolean mask over the (2^K - 1)^2 storage grid of the library: True at nodes of the domain."""
    n = 2 ** K - 1
    if domain == CUBE:
        return np.ones(n ** 3, dtype=bool)
    ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    keep = np.ones((n, n), dtype=bool)
    if domain == LSHAPE:
        q = (n - 1) // 2
        keep = ~((ix >= q) & (iy >= q))
    return keep.ravel()


def to_grid(K: int, domain: int, a):
    """Place domain-node values (last axis in domain-node order) on the storage grid, zeros outside."""
    a = np.asarray(a)
    m = grid_mask(K, domain)
    out = np.zeros(a.shape[:-1] + (m.size,), dtype=a.dtype)
    out[..., m] = a
    return out


def from_grid(K: int, domain: int, a):
    """Values at the domain nodes of a storage-grid array."""
    return np.asarray(a)[..., grid_mask(K, domain)]
