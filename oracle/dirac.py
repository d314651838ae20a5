"""O(a)-improved Wilson-clover Dirac operator (oracle, complex128).

The paper only names the operator: O(a)-improved (Sheikholeslami-Wohlert)
Wilson quarks with periodic boundary conditions (abstract; Sec. 2, Table 1).
Reading used (m0-normalised, r = 1):

  (D psi)(x) = T(x) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ],
  T(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x),
  Fhat_{mu nu} = (1/8) (Q_{mu nu} - Q_{nu mu}),

Q_{mu nu}(x) the sum of the four plaquette leaves at x in the (mu, nu) plane,
all with the same orientation, and m0 = 1/(2 kappa) - 4.  With bc_t = 1 the
time hops across t = T-1 -> 0 pick up a factor -1 (antiperiodic quarks).

Even-odd blocks: D = [[T_ee, D_eo], [D_oe, T_oo]] with D_eo the hopping term
from odd to even sites; Schur complement Dhat = T_ee - D_eo T_oo^-1 D_oe.
"""
import numpy as np
import scipy.sparse as sp

from . import gamma as g
from . import lattice as lat


def _dag(u):
    return np.conj(np.swapaxes(u, -1, -2))


def plaquette_leaves(U, L, T, mu, nu):
    """Q_{mu nu}(x): sum of the four plaquettes based at x in the (mu, nu)
    plane, each traversed mu-then-nu (counter-clockwise)."""
    fwd, bwd = lat.neighbours(L, T)
    Um, Un = U[:, mu], U[:, nu]
    xp_mu, xp_nu = fwd[mu], fwd[nu]
    xm_mu, xm_nu = bwd[mu], bwd[nu]
    xp_mu_m_nu = bwd[nu][xp_mu]      # x + mu - nu
    xm_mu_p_nu = fwd[nu][xm_mu]      # x - mu + nu
    xm_mu_m_nu = bwd[nu][xm_mu]      # x - mu - nu
    q = Um @ Un[xp_mu] @ _dag(Um[xp_nu]) @ _dag(Un)
    q = q + Un @ _dag(Um[xm_mu_p_nu]) @ _dag(Un[xm_mu]) @ Um[xm_mu]
    q = q + _dag(Um[xm_mu]) @ _dag(Un[xm_mu_m_nu]) @ Um[xm_mu_m_nu] @ Un[xm_nu]
    q = q + _dag(Un[xm_nu]) @ Um[xm_nu] @ Un[xp_mu_m_nu] @ _dag(Um)
    return q


def field_strength(U, L, T):
    """Fhat[mu, nu] = (Q_{mu nu} - Q_{nu mu}) / 8, shape [4, 4, V, 3, 3]."""
    V = U.shape[0]
    F = np.zeros((4, 4, V, 3, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                F[mu, nu] = (plaquette_leaves(U, L, T, mu, nu) - plaquette_leaves(U, L, T, nu, mu)) / 8.0
    return F


def clover_field(U, L, T, m0, csw):
    """T(x) as a [V, 12, 12] matrix on (spin, colour) with index 3*alpha + c."""
    V = U.shape[0]
    F = field_strength(U, L, T)
    Tm = np.zeros((V, 12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                Tm += np.einsum("ab,xij->xaibj", g.sigma(mu, nu), F[mu, nu]).reshape(V, 12, 12)
    Tm *= csw * 0.25j
    Tm += (4.0 + m0) * np.eye(12)
    return Tm


def apply_site_matrix(M, psi):
    """(M psi)(x) = M(x) psi(x) for M [V, 12, 12], psi [..., V, 4, 3]."""
    shp = psi.shape
    out = np.einsum("xij,...xj->...xi", M, psi.reshape(shp[:-2] + (12,)))
    return out.reshape(shp)


def _time_phases(L, T, bc_t):
    """(phase_fwd, phase_bwd) [V]: -1 on time hops crossing the boundary when
    bc_t = 1 (antiperiodic), else +1."""
    t = lat.coords(L, T)[:, 0]
    pf = np.ones(t.shape[0])
    pb = np.ones(t.shape[0])
    if bc_t:
        pf[t == T - 1] = -1.0
        pb[t == 0] = -1.0
    return pf, pb


def hop(U, psi, L, T, bc_t=0):
    """Hopping term: -1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]."""
    fwd, bwd = lat.neighbours(L, T)
    pf, pb = _time_phases(L, T, bc_t)
    out = np.zeros_like(psi)
    for mu in range(4):
        ph_f = pf if mu == 0 else 1.0
        ph_b = pb if mu == 0 else 1.0
        uf = np.einsum("xab,...xsb->...xsa", U[:, mu], psi[..., fwd[mu], :, :])
        uf = uf * (ph_f[:, None, None] if mu == 0 else 1.0)
        ub = np.einsum("xba,...xsb->...xsa", np.conj(U[bwd[mu], mu]), psi[..., bwd[mu], :, :])
        ub = ub * (ph_b[:, None, None] if mu == 0 else 1.0)
        out -= 0.5 * (np.einsum("st,...xta->...xsa", g.ID4 - g.GAMMA[mu], uf)
                      + np.einsum("st,...xta->...xsa", g.ID4 + g.GAMMA[mu], ub))
    return out


def apply_dw(U, Tclov, psi, L, T, bc_t=0):
    """Full-lattice D psi."""
    return apply_site_matrix(Tclov, psi) + hop(U, psi, L, T, bc_t)


def apply_gamma5(psi):
    return np.einsum("st,...xta->...xsa", g.GAMMA5, psi)


def apply_spin(M, psi):
    """Apply a 4x4 spin matrix at every site."""
    return np.einsum("st,...xta->...xsa", M, psi)


class EvenOdd:
    """Even-odd blocks of D on an L^3 x T lattice (half-lattice vectors are
    [..., V/2, 4, 3] in the compressed order of ``lattice.eo_tables``)."""

    def __init__(self, U, L, T, m0, csw, bc_t=0):
        self.U, self.L, self.T, self.bc_t = U, L, T, bc_t
        self.V = U.shape[0]
        self.even, self.odd, _ = lat.eo_tables(L, T)
        self.Tclov = clover_field(U, L, T, m0, csw)
        self.T_ee = self.Tclov[self.even]
        self.T_oo_inv = np.linalg.inv(self.Tclov[self.odd])

    def _embed(self, v, sites):
        full = np.zeros(v.shape[:-3] + (self.V, 4, 3), dtype=np.complex128)
        full[..., sites, :, :] = v
        return full

    def D_eo(self, v_o):
        """Hopping from odd to even sites."""
        return hop(self.U, self._embed(v_o, self.odd), self.L, self.T, self.bc_t)[..., self.even, :, :]

    def D_oe(self, v_e):
        """Hopping from even to odd sites."""
        return hop(self.U, self._embed(v_e, self.even), self.L, self.T, self.bc_t)[..., self.odd, :, :]

    def schur(self, v_e):
        """Dhat v_e = T_ee v_e - D_eo T_oo^-1 D_oe v_e."""
        return apply_site_matrix(self.T_ee, v_e) - self.D_eo(apply_site_matrix(self.T_oo_inv, self.D_oe(v_e)))

    def schur_dag(self, v_e):
        """Dhat^dag = gamma_5 Dhat gamma_5 (gamma_5-hermiticity; T commutes
        with gamma_5)."""
        return apply_gamma5(self.schur(apply_gamma5(v_e)))

    def prepare(self, b):
        """bhat = b_e - D_eo T_oo^-1 b_o for a full-lattice source b."""
        b_e, b_o = b[..., self.even, :, :], b[..., self.odd, :, :]
        return b_e - self.D_eo(apply_site_matrix(self.T_oo_inv, b_o))

    def reconstruct(self, x_e, b):
        """Full solution from x_e: x_o = T_oo^-1 (b_o - D_oe x_e)."""
        x_o = apply_site_matrix(self.T_oo_inv, b[..., self.odd, :, :] - self.D_oe(x_e))
        return self._embed(x_e, self.even) + self._embed(x_o, self.odd)

    def apply_full(self, psi):
        return apply_dw(self.U, self.Tclov, psi, self.L, self.T, self.bc_t)


def dirac_sparse(U, Tclov, L, T, bc_t=0):
    """D as a sparse (12V x 12V) matrix, row/column index 12*s + 3*alpha + c;
    the same definition as ``apply_dw`` written out block by block."""
    V = U.shape[0]
    fwd, bwd = lat.neighbours(L, T)
    pf, pb = _time_phases(L, T, bc_t)
    rows, cols, vals = [], [], []
    base = 12 * np.arange(V)
    ii, jj = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")

    def add(blocks, src):
        rows.append((base[:, None, None] + ii[None]).ravel())
        cols.append((12 * src[:, None, None] + jj[None]).ravel())
        vals.append(blocks.ravel())

    add(Tclov, np.arange(V))
    for mu in range(4):
        ph_f = pf if mu == 0 else np.ones(V)
        ph_b = pb if mu == 0 else np.ones(V)
        bf = -0.5 * np.einsum("st,xab->xsatb", g.ID4 - g.GAMMA[mu], U[:, mu]).reshape(V, 12, 12)
        bb = -0.5 * np.einsum("st,xab->xsatb", g.ID4 + g.GAMMA[mu], _dag(U[bwd[mu], mu])).reshape(V, 12, 12)
        add(bf * ph_f[:, None, None], fwd[mu])
        add(bb * ph_b[:, None, None], bwd[mu])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(12 * V, 12 * V))
