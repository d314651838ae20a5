"""Spatial covariant Laplacian of Eq. 1 and its low modes (oracle).

  (lap(t) v)(m) = -6 v(m) + sum_{j=1..3} [ U_j(m, t) v(m + j) + U_j(m - j, t)^dag v(m - j) ]

acting on colour vectors of one timeslice (it is spin-diagonal, so every
colour eigenvector carries four degenerate Dirac eigenvectors v (x) e_alpha,
Sec. 1).  "Low-lying modes" (Sec. 2) is read as the N eigenpairs of -lap(t)
with the smallest eigenvalues (the spectrum of lap(t) lies in [-12, 0]);
eigenvalues are returned as those of -lap(t), ascending.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import lattice as lat


def timeslice_links(U, L, t):
    """Spatial links U_j(m, t), j = 1..3, as [3, L^3, 3, 3]."""
    Vs = L ** 3
    return np.ascontiguousarray(np.transpose(U[t * Vs:(t + 1) * Vs, 1:4], (1, 0, 2, 3)))


def lap_apply(Ut, L, v):
    """lap(t) v for links Ut [3, Vs, 3, 3] and v [..., Vs, 3]."""
    fwd, bwd = lat.spatial_neighbours(L)
    out = -6.0 * v
    for j in range(3):
        out = out + np.einsum("mab,...mb->...ma", Ut[j], v[..., fwd[j], :])
        out = out + np.einsum("mba,...mb->...ma", np.conj(Ut[j][bwd[j]]), v[..., bwd[j], :])
    return out


def lap_dense(Ut, L):
    """lap(t) as a dense (3 Vs x 3 Vs) matrix, index 3 m + c."""
    n = 3 * L ** 3
    eye = np.eye(n, dtype=np.complex128).reshape(n, L ** 3, 3)
    cols = lap_apply(Ut, L, eye)                  # [n, Vs, 3]: images of unit vectors
    return cols.reshape(n, n).T


def lap_modes(Ut, L, n_modes, dense_limit=3072, tol=1e-14, seed=0):
    """Lowest n_modes eigenpairs of -lap(t).  Returns (lam [n], V [n, Vs, 3])
    with lam ascending.  Dense eigh (LAPACK) up to dense_limit rows, else
    ARPACK Lanczos on the largest-algebraic end of lap(t)."""
    Vs = L ** 3
    n = 3 * Vs
    if n <= dense_limit:
        w, Z = np.linalg.eigh(-lap_dense(Ut, L))
        return w[:n_modes], Z[:, :n_modes].T.reshape(n_modes, Vs, 3)

    def mv(x):
        return lap_apply(Ut, L, x.reshape(Vs, 3)).reshape(n)

    op = spla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    rng = np.random.Generator(np.random.PCG64(seed))
    v0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w, Z = spla.eigsh(op, k=n_modes, which="LA", tol=tol, v0=v0, ncv=max(2 * n_modes + 1, 40))
    order = np.argsort(-w)
    return -w[order], Z[:, order].T.reshape(n_modes, Vs, 3)
