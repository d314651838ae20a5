"""Lattice index tables (L^3 x T, periodic).

Site index s = x + L (y + L (z + L t)); direction mu = 0 is t, mu = 1, 2, 3
are x, y, z.  Parity p(s) = (x + y + z + t) mod 2, even sites p = 0.  Within
each parity the sites are numbered in lexicographic order; for even L this is
s // 2.  These tables must agree bit for bit with the GPU library's.
"""
import numpy as np


def coords(L: int, T: int) -> np.ndarray:
    """[V, 4] integer coordinates (t, x, y, z) of each lexicographic site."""
    V = L ** 3 * T
    s = np.arange(V)
    x = s % L
    y = (s // L) % L
    z = (s // L ** 2) % L
    t = s // L ** 3
    return np.stack([t, x, y, z], axis=1)


def site_index(c: np.ndarray, L: int, T: int) -> np.ndarray:
    """Inverse of coords, with periodic wrap of every coordinate."""
    t = c[..., 0] % T
    x = c[..., 1] % L
    y = c[..., 2] % L
    z = c[..., 3] % L
    return x + L * (y + L * (z + L * t))


def neighbours(L: int, T: int):
    """(fwd, bwd): [4, V] site index of s + mu_hat and s - mu_hat."""
    c = coords(L, T)
    fwd = np.empty((4, c.shape[0]), dtype=np.int64)
    bwd = np.empty_like(fwd)
    for mu in range(4):
        e = np.zeros(4, dtype=np.int64)
        e[mu] = 1
        fwd[mu] = site_index(c + e, L, T)
        bwd[mu] = site_index(c - e, L, T)
    return fwd, bwd


def parity(L: int, T: int) -> np.ndarray:
    return coords(L, T).sum(axis=1) % 2


def eo_tables(L: int, T: int):
    """(even_sites, odd_sites, eo_index): lexicographic site lists of each
    parity, in increasing order, and the compressed index of every site within
    its own parity."""
    p = parity(L, T)
    even = np.nonzero(p == 0)[0]
    odd = np.nonzero(p == 1)[0]
    eo = np.empty(p.shape[0], dtype=np.int64)
    eo[even] = np.arange(even.shape[0])
    eo[odd] = np.arange(odd.shape[0])
    return even, odd, eo


def spatial_neighbours(L: int):
    """(fwd, bwd): [3, L^3] neighbour tables inside one timeslice, j = 1..3
    (x, y, z) stored at index j - 1."""
    Vs = L ** 3
    m = np.arange(Vs)
    c = np.stack([m % L, (m // L) % L, m // L ** 2], axis=1)
    fwd = np.empty((3, Vs), dtype=np.int64)
    bwd = np.empty_like(fwd)
    for j in range(3):
        e = np.zeros(3, dtype=np.int64)
        e[j] = 1
        cf = (c + e) % L
        cb = (c - e) % L
        fwd[j] = cf[:, 0] + L * (cf[:, 1] + L * cf[:, 2])
        bwd[j] = cb[:, 0] + L * (cb[:, 1] + L * cb[:, 2])
    return fwd, bwd
