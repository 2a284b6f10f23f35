"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only lays out problem data: it samples closed-form functions at the
space-time grid nodes and draws seeded random arrays.  It holds none of the
solver's arithmetic (no finite-element matrices, multigrid or wavelets).

Layout (the library's): a space-time array has shape (N_t, N_x); row i is time
node t_i = i / 2^J, column p is the p-th interior node of the spatial grid in
lexicographic order with x fastest.  Grid node (i, j) sits at (i h, j h),
h = 2^-K.  On the unit square the interior nodes are 1 <= i, j <= 2^K - 1; on the
L-shape (0,1)^2 minus [1/2,1)^2 the nodes with x >= 1/2 and y >= 1/2 are left out.
"""
from __future__ import annotations

import numpy as np

SQUARE = 0
LSHAPE = 1


def dims(K: int, J: int, domain: int = SQUARE):
    n = 2 ** K - 1
    Nx = n * n if domain == SQUARE else n * n - (2 ** (K - 1)) ** 2
    return 2 ** J + 1, Nx


def node_coords(K: int, domain: int = SQUARE):
    """(x, y) of the interior nodes in lexicographic order, x fastest."""
    m = 2 ** K
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
    x, y = node_coords(K, domain)
    t = time_nodes(J)
    k = 1.0 if domain == SQUARE else 2.0
    d11, d12, d22 = (1.0, 0.0, 1.0) if D is None else (D[0][0], D[0][1], D[1][1])
    phi = np.sin(k * np.pi * x) * np.sin(k * np.pi * y)
    cross = np.cos(k * np.pi * x) * np.cos(k * np.pi * y)
    tt = (1.0 + t[:, None] ** 2)
    u = tt * phi[None, :]
    g = (2.0 * t[:, None] + ((d11 + d22) * (k * np.pi) ** 2 + c) * tt) * phi[None, :] \
        - 2.0 * d12 * (k * np.pi) ** 2 * tt * cross[None, :]
    return g, phi.copy(), u


def decaying(K: int, J: int):
    """The 2D workload of the paper's scaling runs: u = exp(-2 pi^2 t) sin(pi x) sin(pi y), g = 0."""
    x, y = node_coords(K, SQUARE)
    t = time_nodes(J)
    phi = np.sin(np.pi * x) * np.sin(np.pi * y)
    u = np.exp(-2.0 * np.pi ** 2 * t)[:, None] * phi[None, :]
    return np.zeros_like(u), phi.copy(), u


def smooth_forcing(K: int, J: int, seed: int, domain: int = SQUARE, modes: int = 8):
    """g = sum_m c_m cos(k_m pi t) sin(a_m pi x) sin(b_m pi y), c ~ N(0,1); u0 = 0."""
    rng = np.random.default_rng(seed)
    x, y = node_coords(K, domain)
    t = time_nodes(J)
    c = rng.standard_normal(modes)
    a = rng.integers(1, 5, modes)
    b = rng.integers(1, 5, modes)
    kk = rng.integers(0, 4, modes)
    g = np.zeros((t.size, x.size))
    for m in range(modes):
        g += c[m] * np.cos(kk[m] * np.pi * t)[:, None] * (np.sin(a[m] * np.pi * x) * np.sin(b[m] * np.pi * y))[None, :]
    return g, np.zeros(x.size)


def random_state(Nt: int, Nx: int, seed: int):
    """Standard-normal (N_t, N_x) array, seeded."""
    return np.random.default_rng(seed).standard_normal((Nt, Nx))


def grid_mask(K: int, domain: int = SQUARE):
    """Boolean mask over the (2^K - 1)^2 storage grid of the library: True at nodes of the domain."""
    n = 2 ** K - 1
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
