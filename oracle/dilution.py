"""Colour x even-odd diluted stochastic wall sources with the spin-explicit
one-end insertion (oracle, complex128).  TEST INFRASTRUCTURE ONLY.

Sec. 3 measures with "six independent colour and even-odd diluted wall
sources" per noise vector (and the caption of Fig. 1 counts 24 wall sources:
six dilution pieces times four source spins).  The estimator is that of Eq. 3
with the noise outer product eta eta^dag replaced by the sum over the dilution
pieces, sum_d eta_d eta_d^dag, whose noise average is the identity.

Readings (the paper names the dilution but gives no formulae):
  * A wall noise is one Z2 x Z2 number per site and colour of the source
    timeslice t' (eta [N_r, L^3, 3]); it carries no spin index.
  * Dilution piece d = 2 c + p keeps colour c and the sites of t' whose
    four-dimensional parity (x + y + z + t') mod 2 is p.
  * Spin is treated exactly ("spin-explicit"): every piece is solved for the
    four source spins, eta_d (x) e_beta, so the source Gamma enters through its
    spin matrix instead of extra solves:
        phi_{d,beta}    = D^-1 (eta_d (x) e_beta)
        phibar_{d,beta} = D^-1 ((1 - Box(t')) eta_d (x) e_beta)
    and, by cyclicity of the trace in Eq. 3 with B = G' g5 acting on the source
    spin,
        C_P(t) = 1/N_r sum_{r,d} sum_{beta,beta'} B[beta,beta'] sum_{x in t}
                 phibar_{d,beta'}(x)^dag g5 G [P_t phi_{d,beta}](x)
    with P_t = 1 - Box(t) (rest) or Box(t) (mixed): 48 solves per noise vector.
  * C_dist is unchanged (distillation solves); C = C_rest + 2 C_mixed + C_dist.

Two independent statements of the same estimator live here: the solve-based
contraction above (the algorithm) and `diluted_trace`, the trace of Eq. 3 with
the dense propagator block and the dilution outer product written out as a
matrix (the definition).
"""
import numpy as np

from . import dlma
from . import gamma as g


def dilution_pieces(eta_wall, L, tp):
    """eta_wall [N_r, Vs, 3] -> eta_d [N_r, 6, Vs, 3], piece d = 2 c + p."""
    Nr, Vs = eta_wall.shape[0], eta_wall.shape[1]
    m = np.arange(Vs)
    x, y, z = m % L, (m // L) % L, m // (L * L)
    par = (x + y + z + tp) % 2
    out = np.zeros((Nr, 6, Vs, 3), dtype=np.complex128)
    for c in range(3):
        for p in range(2):
            sel = par == p
            out[:, 2 * c + p, sel, c] = eta_wall[:, sel, c]
    return out


def wall_sources(eta_d, Vtp, L, T, tp):
    """Spin-explicit sources of the dilution pieces eta_d [N_r, 6, Vs, 3]:
    returns (b_phi, b_phibar), each [N_r, 6, 4 (beta), V, 4, 3], with
    b_phi = eta_d (x) e_beta and b_phibar = ((1 - Box(t')) eta_d) (x) e_beta."""
    Nr, Vs = eta_d.shape[0], eta_d.shape[2]
    # (1 - Box) acts on colour only: apply it to eta_d placed in one spin component
    e1 = np.zeros((Nr, 6, Vs, 4, 3), dtype=np.complex128)
    e1[:, :, :, 0, :] = eta_d
    pe = (e1 - dlma.box(Vtp, e1))[:, :, :, 0, :]
    V = L ** 3 * T
    sl = slice(tp * Vs, (tp + 1) * Vs)
    b = np.zeros((Nr, 6, 4, V, 4, 3), dtype=np.complex128)
    bb = np.zeros_like(b)
    for beta in range(4):
        b[:, :, beta, sl, beta, :] = eta_d
        bb[:, :, beta, sl, beta, :] = pe
    return b, bb


def diluted_noise_parts(V_all, phi, phibar, L, T):
    """C_rest and C_mixed [4, T] from phi, phibar [N_r, 6, 4, V, 4, 3] (the
    solve-based contraction of the module docstring)."""
    Nr = phi.shape[0]
    rest = np.zeros((4, T), dtype=np.complex128)
    mixed = np.zeros((4, T), dtype=np.complex128)
    for t in range(T):
        Vt = V_all[t]
        ph = dlma.timeslice(phi, L, t)        # [Nr, 6, 4, Vs, 4, 3]
        pb = dlma.timeslice(phibar, L, t)
        bph = dlma.box(Vt, ph)
        for ch, G in enumerate(g.CHANNELS):
            A = g.GAMMA5 @ G
            B = G @ g.GAMMA5
            Ab = np.einsum("st,rdbmtc->rdbmsc", A, bph)
            Aall = np.einsum("st,rdbmtc->rdbmsc", A, ph)
            # W[r, d, beta', beta] = <phibar_{beta'}, A P phi_beta>_t
            Wm = np.einsum("rdqmsc,rdbmsc->rdqb", np.conj(pb), Ab)
            Wf = np.einsum("rdqmsc,rdbmsc->rdqb", np.conj(pb), Aall)
            mixed[ch, t] = np.einsum("bq,rdqb->", B, Wm) / Nr
            rest[ch, t] = np.einsum("bq,rdqb->", B, Wf - Wm) / Nr
    return rest, mixed


def diluted_correlators(solve, V_all, eta_wall, L, T, tp):
    """The whole estimator with diluted wall sources on one configuration.

    solve(b [n, V, 4, 3]) -> D^-1 b; V_all [T, N_c, Vs, 3]; eta_wall [N_r, Vs, 3].
    Returns dict with C_dist, C_rest, C_mixed, C (each complex [4, T] over the
    channels PS, V1, V2, V3) and the solutions."""
    Nr = eta_wall.shape[0]
    V = L ** 3 * T
    bd = dlma.distillation_sources(V_all[tp], L, T, tp)
    phid = solve(bd)
    tau = dlma.perambulator(V_all, phid, L, T)
    cd = dlma.c_dist(tau)
    eta_d = dilution_pieces(eta_wall, L, tp)
    b, bb = wall_sources(eta_d, V_all[tp], L, T, tp)
    phi = solve(b.reshape(Nr * 24, V, 4, 3)).reshape(Nr, 6, 4, V, 4, 3)
    phibar = solve(bb.reshape(Nr * 24, V, 4, 3)).reshape(Nr, 6, 4, V, 4, 3)
    rest, mixed = diluted_noise_parts(V_all, phi, phibar, L, T)
    return {"C_dist": cd, "C_rest": rest, "C_mixed": mixed, "C": rest + 2 * mixed + cd,
            "phi": phi, "phibar": phibar, "phi_dist": phid}


def plain_diluted(phi, L, T):
    """The plain (no distillation) estimator with spin-explicit diluted
    sources: Eq. 3's trace with no Box, eta eta^dag -> sum_d eta_d eta_d^dag,
        C(t) = 1/N_r sum_{r,d} sum_{beta,beta'} B[beta,beta'] sum_{x in t}
               phi_{d,beta'}(x)^dag g5 G phi_{d,beta}(x),   B = G g5,
    from phi [N_r, n_pieces, 4 (beta), V, 4, 3], phi_{d,beta} = D^-1 (eta_d (x) e_beta)
    (any number of pieces per noise vector).  Returns complex [4, T]."""
    Nr = phi.shape[0]
    out = np.zeros((4, T), dtype=np.complex128)
    for t in range(T):
        ph = dlma.timeslice(phi, L, t)
        for ch, G in enumerate(g.CHANNELS):
            A = g.GAMMA5 @ G
            B = G @ g.GAMMA5
            Aph = np.einsum("st,rdbmtc->rdbmsc", A, ph)
            W = np.einsum("rdqmsc,rdbmsc->rdqb", np.conj(ph), Aph)     # [r, d, beta', beta]
            out[ch, t] = np.einsum("bq,rdqb->", B, W) / Nr
    return out


def plain_diluted_correlators(solve, eta_wall, L, T, tp):
    """The plain estimator with the six colour x even-odd diluted wall sources
    of every noise vector eta_wall [N_r, Vs, 3]: 24 solves per noise vector."""
    Nr = eta_wall.shape[0]
    V = L ** 3 * T
    eta_d = dilution_pieces(eta_wall, L, tp)
    sl = slice(tp * L ** 3, (tp + 1) * L ** 3)
    b = np.zeros((Nr, 6, 4, V, 4, 3), dtype=np.complex128)
    for beta in range(4):
        b[:, :, beta, sl, beta, :] = eta_d
    phi = solve(b.reshape(Nr * 24, V, 4, 3)).reshape(Nr, 6, 4, V, 4, 3)
    return plain_diluted(phi, L, T), phi


def source_outer(pieces):
    """P = sum_d (eta_d (x) 1_spin)(eta_d (x) 1_spin)^dag on the source timeslice,
    as an [12 Vs, 12 Vs] matrix with index 12 m + 3 alpha + c.
    pieces [n_pieces, Vs, 3] (the pieces of one noise vector)."""
    Vs = pieces.shape[1]
    Pc = np.einsum("dmc,dne->mcne", pieces, np.conj(pieces))          # colour-site block
    P = np.einsum("mcne,ab->macnbe", Pc, np.eye(4))
    return P.reshape(12 * Vs, 12 * Vs)


def diluted_trace(S, V_all, pieces_all, L, T, tp):
    """The definition: C^{X,Y}(t) = 1/N_r sum_r tr[g5 G X S(t,t') P_r G g5 Y S(t,t')^dag]
    (Eq. 3 with eta eta^dag -> P_r = sum_d eta_d eta_d^dag), from the exact
    propagator columns S [Vs, 4, 3, V, 4, 3] of timeslice t' (as in
    `dlma.exact_parts`) and the dilution pieces of every noise vector
    pieces_all [N_r, n_pieces, Vs, 3].  Returns (rest, mixed) [4, T] with
    rest = (X, Y) = (1 - Box, 1 - Box) and mixed = (Box, 1 - Box)."""
    Vs = L ** 3
    n = 12 * Vs
    Nr = pieces_all.shape[0]

    def box_full(Vt):
        Pc = np.einsum("kmc,knd->mcnd", Vt, np.conj(Vt))
        return np.einsum("mcnd,ab->macnbd", Pc, np.eye(4)).reshape(n, n)

    def spin_full(M):
        return np.kron(np.eye(Vs), np.kron(M, np.eye(3)))

    Yr = np.eye(n) - box_full(V_all[tp])
    Pm = sum(source_outer(pieces_all[r]) for r in range(Nr)) / Nr
    Smat = S.reshape(n, L ** 3 * T, 4, 3)
    rest = np.zeros((4, T), dtype=np.complex128)
    mixed = np.zeros((4, T), dtype=np.complex128)
    for t in range(T):
        St = Smat[:, t * Vs:(t + 1) * Vs].reshape(n, n).T     # rows: sink; columns: source
        Xb = box_full(V_all[t])
        Xr = np.eye(n) - Xb
        for ch, G in enumerate(g.CHANNELS):
            G1 = spin_full(g.GAMMA5 @ G)
            G2 = spin_full(G @ g.GAMMA5)
            R = St @ Pm @ G2 @ Yr @ np.conj(St.T)
            rest[ch, t] = np.trace(G1 @ Xr @ R)
            mixed[ch, t] = np.trace(G1 @ Xb @ R)
    return rest, mixed
