"""Conventional low-mode averaging with Dirac low modes (oracle, complex128):
the control the paper names in Sec. 1 and after Eq. 2.  TEST INFRASTRUCTURE
ONLY.

With Box built from eigenmodes of the Dirac operator instead of the spatial
Laplacian, Box and the propagator commute and the mixed term of Eq. 2 vanishes.
Reading used (the paper states the fact, not the construction):

  * The modes are those of the hermitian even-odd operator Qhat = g5 Dhat on the
    even sites (Dhat = T_ee - D_eo T_oo^-1 D_oe is the Schur complement, and the
    even-even block of D^-1 is Dhat^-1), with the n smallest |lambda|;
    P = sum_i u_i u_i^dag.
  * Dhat^-1 = Qhat^-1 g5, so a projector that commutes with the propagator at its
    sink commutes at its source after conjugation with g5: the mixed block is
        P Dhat^-1 (1 - g5 P g5) = Qhat^-1 P (1 - P) g5 = 0,
    while the Laplacian Box (spin-diagonal, so g5 Box g5 = Box) leaves
    Box Dhat^-1 (1 - Box) nonzero: the C_mixed of Eq. 2 that the paper measures.
"""
import numpy as np

from . import dirac as dr
from . import gamma as g


def schur_matrix(eo: dr.EvenOdd):
    """Dhat as a dense matrix on the even sites (index 12 i + 3 alpha + c, i the
    compressed even index), from the sparse D: D_ee - D_eo D_oo^-1 D_oe."""
    D = dr.dirac_sparse(eo.U, eo.Tclov, eo.L, eo.T, eo.bc_t).toarray()
    ie = (12 * eo.even[:, None] + np.arange(12)[None]).ravel()
    io = (12 * eo.odd[:, None] + np.arange(12)[None]).ravel()
    Dee, Deo, Doe, Doo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)]
    return Dee - Deo @ np.linalg.solve(Doo, Doe)


def gamma5_matrix(n_sites):
    return np.kron(np.eye(n_sites), np.kron(g.GAMMA5, np.eye(3)))


def dirac_low_modes(eo: dr.EvenOdd, n):
    """The n eigenpairs of Qhat = g5 Dhat with the smallest |lambda| (dense eigh):
    (lambda [n], u [n, V/2, 4, 3]), sorted by |lambda|."""
    Dh = schur_matrix(eo)
    G5 = gamma5_matrix(Dh.shape[0] // 12)
    Q = G5 @ Dh
    w, U = np.linalg.eigh(0.5 * (Q + np.conj(Q.T)))
    order = np.argsort(np.abs(w), kind="stable")[:n]
    return w[order], np.transpose(U[:, order]).reshape(n, -1, 4, 3)


def project(u, v, conj_g5=False):
    """P v (or g5 P g5 v) for even-site fields v [..., V/2, 4, 3], P = sum u u^dag."""
    if conj_g5:
        v = dr.apply_gamma5(v)
    c = np.einsum("nisc,...isc->...n", np.conj(u), v)
    out = np.einsum("nisc,...n->...isc", u, c)
    return dr.apply_gamma5(out) if conj_g5 else out
