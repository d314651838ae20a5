"""Dirac solves x = D^-1 b (oracle).

The paper's solver type is not stated (Sec. 2 only says the propagators are
computed with openQ*D).  Reading used: even-odd Schur system
Dhat x_e = bhat, solved by the conjugate-gradient method on the normal
equations Dhat^dag Dhat x_e = Dhat^dag bhat (CGNE) in complex128, stopped on
the TRUE full-lattice residual ||b - D x||_2 / ||b||_2 <= tol.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .dirac import EvenOdd, dirac_sparse


def _vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def true_residual(eo: EvenOdd, x, b):
    """||b - D x|| / ||b|| on the full lattice."""
    return np.linalg.norm((b - eo.apply_full(x)).ravel()) / np.linalg.norm(b.ravel())


def cgne(eo: EvenOdd, b, tol=1e-12, maxiter=20000, check_every=10):
    """Solve D x = b for one full-lattice source b [V, 4, 3].
    Returns (x, iterations, true_residual)."""
    bhat = eo.prepare(b)
    x = np.zeros_like(bhat)
    r = eo.schur_dag(bhat)           # normal-equation residual, x0 = 0
    p = r.copy()
    rr = _vdot(r, r).real
    it = 0
    res = np.inf
    while it < maxiter:
        q = eo.schur(p)
        alpha = rr / _vdot(q, q).real
        x = x + alpha * p
        r = r - alpha * eo.schur_dag(q)
        rr_new = _vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if it % check_every == 0 or rr == 0.0:
            res = true_residual(eo, eo.reconstruct(x, b), b)
            if res <= tol:
                break
    xf = eo.reconstruct(x, b)
    return xf, it, true_residual(eo, xf, b)


def lu_solver_dag(eo: EvenOdd):
    """Sparse LU of D^dag (the conjugate transpose of the matrix itself, not
    the gamma_5 identity): maps g [n, V, 4, 3] to D^-dag g."""
    D = dirac_sparse(eo.U, eo.Tclov, eo.L, eo.T, eo.bc_t).conj().T.tocsc()
    lu = spla.splu(D)
    V = eo.V

    def solve(g):
        x = lu.solve(np.ascontiguousarray(g.reshape(-1, 12 * V).T))
        return x.T.reshape(g.shape)

    return solve


def lu_solver(eo: EvenOdd):
    """Sparse LU factorisation of the full D (library routine; the dense-LU
    cross-check).  Returns a function mapping sources [n, V, 4, 3] to
    solutions."""
    D = dirac_sparse(eo.U, eo.Tclov, eo.L, eo.T, eo.bc_t).tocsc()
    lu = spla.splu(D)
    V = eo.V

    def solve(b):
        bb = b.reshape(-1, 12 * V).T
        x = lu.solve(np.ascontiguousarray(bb))
        return x.T.reshape(b.shape)

    return solve
