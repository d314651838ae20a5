"""Distillation low-mode averaging: sources, projector, perambulator and the
C_rest / C_mixed / C_dist contractions (oracle, complex128).

Eq. 1:  Box(t) = V(t) V(t)^dag, V(t)'s columns the Laplacian eigenvectors,
        acting on the colour index and diagonal in spin.
Eq. 2:  C = C_rest + 2 C_mixed + C_dist from inserting 1 = (1 - Box) + Box at
        sink and source (the two mixed terms merged by time reversal).
Eq. 3:  C_dist(t)  = tr[g5 G  tau(t) G' g5 tau(t)^dag],  tau(t) = V(t)^dag D^-1(t,t') V(t')
        C_rest(t)  = (1/N_r) sum_r tr[g5 G (1-Box(t)) D^-1 eta eta^dag G' g5 (1-Box(t')) D^-1^dag]
        C_mixed(t) = (1/N_r) sum_r tr[g5 G Box(t)     D^-1 eta eta^dag G' g5 (1-Box(t')) D^-1^dag]
Eq. 4:  phi_r = D^-1 eta_r,  phibar_r = D^-1 (1 - Box(t')) eta_r.

Readings (the paper is silent or ambiguous on these):
  * D^-1^dag(t', t) is the adjoint of the t <- t' propagator block.
  * By cyclicity tr[A eta eta^dag B] = (B^dag eta)^dag (A eta), so
        C_part(t) = (1/N_r) sum_r sum_{x in t} chi_r(x)^dag g5 G [P_t phi_r](x)
    with P_t = 1 - Box(t) (rest) or Box(t) (mixed) and the left vector
    chi_r = D^-1 (1 - Box(t')) g5 G'^dag eta_r: for G' = g5 this is phibar_r,
    for G' = g_k it is psibar_{r,k} = D^-1 g5 g_k (1 - Box(t')) eta_r, one more
    solve per noise and k (the noise is not spin-diluted).  So each noise
    vector costs 5 solves: phi, phibar, psibar_1..3.
  * Sink and source Gamma are the same channel: G = G' = g5 (pseudoscalar) or
    g_k (vector, k = 1..3, averaged by the caller).
  * No fermion-loop minus sign (Eq. 3 literally); C(t) is kept complex.
  * Distillation source index j = 4 k + alpha (mode-major): source
    v_k(t') (x) e_alpha on timeslice t'.
"""
import numpy as np

from . import gamma as g


def timeslice(psi, L, t):
    """Restriction of [..., V, 4, 3] to timeslice t: [..., Vs, 4, 3]."""
    Vs = L ** 3
    return psi[..., t * Vs:(t + 1) * Vs, :, :]


def coeffs(Vt, psi_t):
    """c[..., k, alpha] = sum_{m, c} conj(v_k(m, c)) psi(m, alpha, c)  (V^dag psi)."""
    return np.einsum("kmc,...mac->...ka", np.conj(Vt), psi_t)


def box(Vt, psi_t):
    """Box(t) psi = V (V^dag psi), spin by spin."""
    return np.einsum("kmc,...ka->...mac", Vt, coeffs(Vt, psi_t))


def distillation_sources(Vtp, L, T, tp):
    """[4 N_c, V, 4, 3]: source 4k + alpha is v_k(t') (x) e_alpha on timeslice t'."""
    Nc, Vs = Vtp.shape[0], Vtp.shape[1]
    b = np.zeros((Nc, 4, L ** 3 * T, 4, 3), dtype=np.complex128)
    for a in range(4):
        b[:, a, tp * Vs:(tp + 1) * Vs, a, :] = Vtp
    return b.reshape(4 * Nc, L ** 3 * T, 4, 3)


def noise_sources(eta, Vtp, L, T, tp):
    """For each noise eta_r [Vs, 4, 3] on t': the five sources
    [eta, (1-Box')eta, g5 g_1 (1-Box')eta, g5 g_2 (1-Box')eta, g5 g_3 (1-Box')eta].
    Returns [N_r, 5, V, 4, 3]."""
    Nr, Vs = eta.shape[0], eta.shape[1]
    pe = eta - box(Vtp, eta)
    b = np.zeros((Nr, 5, L ** 3 * T, 4, 3), dtype=np.complex128)
    sl = slice(tp * Vs, (tp + 1) * Vs)
    b[:, 0, sl] = eta
    b[:, 1, sl] = pe
    for k in range(1, 4):
        b[:, 1 + k, sl] = np.einsum("st,rmtc->rmsc", g.GAMMA5 @ g.GAMMA[k], pe)
    return b


def perambulator(V_all, phi_dist, L, T):
    """tau[t, k, alpha, l, beta] = sum_{m in t, c} conj(v_k(m,c;t)) phi^{(l,beta)}(m, t, alpha, c)
    for solutions phi_dist [4 N_c, V, 4, 3] of the distillation sources."""
    Nc = V_all.shape[1]
    tau = np.empty((T, Nc, 4, Nc, 4), dtype=np.complex128)
    for t in range(T):
        c = coeffs(V_all[t], timeslice(phi_dist, L, t))      # [4Nc (l,beta), k, alpha]
        tau[t] = np.transpose(c.reshape(Nc, 4, Nc, 4), (2, 3, 0, 1))
    return tau


def c_dist(tau):
    """C_dist^G(t) = tr[(1 x g5 G) tau (1 x G g5) tau^dag] for the four channels.
    Returns complex [4, T]."""
    out = np.empty((4, tau.shape[0]), dtype=np.complex128)
    for ch, G in enumerate(g.CHANNELS):
        A = g.GAMMA5 @ G
        B = G @ g.GAMMA5
        out[ch] = np.einsum("ab,tkblc,cd,tkald->t", A, tau, B, np.conj(tau))
    return out


def noise_parts(V_all, phi, phibar, psibar, L, T):
    """C_rest and C_mixed [4, T] from the noise solutions.
    phi, phibar [N_r, V, 4, 3]; psibar [N_r, 3, V, 4, 3]."""
    Nr = phi.shape[0]
    rest = np.zeros((4, T), dtype=np.complex128)
    mixed = np.zeros((4, T), dtype=np.complex128)
    for t in range(T):
        Vt = V_all[t]
        ph = timeslice(phi, L, t)
        bph = box(Vt, ph)
        for ch, G in enumerate(g.CHANNELS):
            chi = timeslice(phibar if ch == 0 else psibar[:, ch - 1], L, t)
            A = g.GAMMA5 @ G
            Ab = np.einsum("st,rmtc->rmsc", A, bph)
            Ar = np.einsum("st,rmtc->rmsc", A, ph) - Ab
            mixed[ch, t] = np.vdot(chi.ravel(), Ab.ravel()) / Nr
            rest[ch, t] = np.vdot(chi.ravel(), Ar.ravel()) / Nr
    return rest, mixed


def mixed_src(V_all, phi_dist, L, T):
    """The source-side mixed term of Eq. 2 (Box at the source, 1 - Box at the
    sink), exact, from the distillation solutions phi_dist [4 N_c, V, 4, 3]
    (row 4k + beta solves v_k(t') (x) e_beta).  With Box(t') = sum_{k,beta}
    w_{k beta} w_{k beta}^dag, w = v_k(t') (x) e_beta, and S w = phi:
        tr[g5 G (1 - Box(t)) S G g5 Box(t') S^dag]
          = sum_{k, b, b'} (G g5)_{b' b} <phi^(k,b), g5 G (1 - Box(t)) phi^(k,b')>_t.
    Returns complex [4, T] over the channels (PS, V1, V2, V3)."""
    Nc = phi_dist.shape[0] // 4
    out = np.zeros((4, T), dtype=np.complex128)
    for t in range(T):
        ph = timeslice(phi_dist, L, t)
        pr = (ph - box(V_all[t], ph)).reshape(Nc, 4, L ** 3, 4, 3)
        ph = ph.reshape(Nc, 4, L ** 3, 4, 3)
        for ch, G in enumerate(g.CHANNELS):
            A = g.GAMMA5 @ G
            B = G @ g.GAMMA5
            Apr = np.einsum("st,kbmtc->kbmsc", A, pr)
            # W[k, b, b'] = <phi^(k,b), A (1 - Box) phi^(k,b')>_t
            W = np.einsum("kbmsc,kqmsc->kbq", np.conj(ph), Apr)
            out[ch, t] = np.einsum("qb,kbq->", B, W)
    return out


def plain_sources(eta, L, T, tp):
    """Sources of the plain (no distillation) one-end estimator with undiluted
    noise eta [N_r, Vs, 4, 3] on t': [N_r, 4, V, 4, 3] = eta, g5 g_k eta (k = 1..3)."""
    Nr, Vs = eta.shape[0], eta.shape[1]
    b = np.zeros((Nr, 4, L ** 3 * T, 4, 3), dtype=np.complex128)
    sl = slice(tp * Vs, (tp + 1) * Vs)
    b[:, 0, sl] = eta
    for k in range(1, 4):
        b[:, k, sl] = np.einsum("st,rmtc->rmsc", g.GAMMA5 @ g.GAMMA[k], eta)
    return b


def plain_estimator(phi, chi, L, T):
    """The plain stochastic estimator of the correlator of Eq. 2's left-hand
    side (no Box anywhere): by cyclicity tr[g5 G S eta eta^dag G g5 S^dag] =
    <S g5 G eta, g5 G S eta>, so with phi_r = D^-1 eta_r and
    chi_{r,k} = D^-1 g5 g_k eta_r (chi = phi for G = g5)
        C(t) = 1/N_r sum_r sum_{x in t} chi_r^dag g5 G phi_r.
    phi [N_r, V, 4, 3], chi [N_r, 3, V, 4, 3].  Returns complex [4, T]."""
    Nr = phi.shape[0]
    out = np.zeros((4, T), dtype=np.complex128)
    for t in range(T):
        ph = timeslice(phi, L, t)
        for ch, G in enumerate(g.CHANNELS):
            left = ph if ch == 0 else timeslice(chi[:, ch - 1], L, t)
            Aph = np.einsum("st,rmtc->rmsc", g.GAMMA5 @ G, ph)
            out[ch, t] = np.vdot(left.ravel(), Aph.ravel()) / Nr
    return out


def dlma_correlators(solve, V_all, eta, L, T, tp):
    """The whole estimator of Eqs. 2-4 on one configuration.

    solve(b [n, V, 4, 3]) -> D^-1 b; V_all [T, N_c, Vs, 3]; eta [N_r, Vs, 4, 3].
    Returns dict with C_dist, C_rest, C_mixed, C (= C_rest + 2 C_mixed + C_dist),
    each complex [4, T] over channels (PS, V1, V2, V3), plus tau and the
    solutions."""
    Nc = V_all.shape[1]
    Nr = eta.shape[0]
    bd = distillation_sources(V_all[tp], L, T, tp)
    bn = noise_sources(eta, V_all[tp], L, T, tp)
    phid = solve(bd)
    phin = solve(bn.reshape(Nr * 5, L ** 3 * T, 4, 3)).reshape(Nr, 5, L ** 3 * T, 4, 3)
    tau = perambulator(V_all, phid, L, T)
    cd = c_dist(tau)
    rest, mixed = noise_parts(V_all, phin[:, 0], phin[:, 1], phin[:, 2:5], L, T)
    return {"C_dist": cd, "C_rest": rest, "C_mixed": mixed, "C": rest + 2 * mixed + cd,
            "tau": tau, "phi_dist": phid, "phi_noise": phin, "Nc": Nc}


def ps_loss(solve, V_all, eta, w, L, T, tp):
    """L = sum_t w(t) Re C_PS(t) with C_PS = C_rest + 2 C_mixed + C_dist (Eq. 2,
    Gamma = gamma_5).  Returns (L, correlator dict)."""
    r = dlma_correlators(solve, V_all, eta, L, T, tp)
    return float(np.sum(w * r["C"][0].real)), r


def ps_loss_grads(solve, solve_dag, V_all, eta, w, L, T, tp):
    """Adjoint-method gradients of ps_loss with respect to m0 and eta, written
    as dL/dRe + i dL/dIm.  With Gamma = gamma_5, C_dist = sum |V^dag phi|^2 and
    C_rest + 2 C_mixed = 1/N_r sum_r <phibar_r, (1 + Box) phi_r>, so
      G(phi_dist) = 2 w Box phi,  G(phi_r) = w/N_r (1 + Box) phibar_r,
      G(phibar_r) = w/N_r (1 + Box) phi_r;
    y = D^-dag G; dL/dm0 = -sum Re <y, phi> (dD/dm0 = 1);
    dL/deta_r = y_{phi_r} + (1 - Box(t')) y_{phibar_r} on t'."""
    loss, r = ps_loss(solve, V_all, eta, w, L, T, tp)
    Nr = eta.shape[0]
    Vs = L ** 3
    phid = r["phi_dist"]
    phi, phibar = r["phi_noise"][:, 0], r["phi_noise"][:, 1]

    def per_t(f, field):
        out = np.zeros_like(field)
        for t in range(T):
            sl = slice(t * Vs, (t + 1) * Vs)
            out[..., sl, :, :] = f(t, field[..., sl, :, :])
        return out

    Gd = per_t(lambda t, x: 2 * w[t] * box(V_all[t], x), phid)
    G_phi = per_t(lambda t, x: w[t] / Nr * (x + box(V_all[t], x)), phibar)
    G_phibar = per_t(lambda t, x: w[t] / Nr * (x + box(V_all[t], x)), phi)
    yd = solve_dag(Gd)
    y_phi = solve_dag(G_phi)
    y_phibar = solve_dag(G_phibar)
    dm0 = -(np.vdot(yd.ravel(), phid.ravel()).real + np.vdot(y_phi.ravel(), phi.ravel()).real
            + np.vdot(y_phibar.ravel(), phibar.ravel()).real)
    a = timeslice(y_phi, L, tp)
    b = timeslice(y_phibar, L, tp)
    deta = a + b - box(V_all[tp], b)
    return loss, dm0, deta


def exact_parts(S, V_all, L, T, tp):
    """Exact (noise-free) correlator pieces from the propagator columns of
    timeslice t'.  S [Vs, 4, 3, V, 4, 3]: S[y, beta, b] = D^-1 (delta_y e_beta e_b).

    C^{X,Y}(t) = tr[g5 G X S(t,t') G g5 Y S(t,t')^dag] for X (sink) and Y
    (source) each 1 - Box or Box.  Returns dict of complex [4, T]:
    'rest' (1-Box, 1-Box), 'mixed_snk' (Box, 1-Box) -- the term the paper's
    C_mixed estimates --, 'mixed_src' (1-Box, Box), 'dist' (Box, Box) and
    'full' (1, 1)."""
    Vs = L ** 3
    n = 12 * Vs
    Vp = V_all[tp]

    # Box on (site, spin, colour) with index 12 m + 3 alpha + c
    def box_full(Vt):
        Pc = np.einsum("kmc,knd->mcnd", Vt, np.conj(Vt))          # [m, c, n, d]
        P = np.einsum("mcnd,ab->macnbd", Pc, np.eye(4))
        return P.reshape(n, n)

    def spin_full(M):
        return np.kron(np.eye(Vs), np.kron(M, np.eye(3)))

    Ysrc = {"box": box_full(Vp)}
    Ysrc["rest"] = np.eye(n) - Ysrc["box"]
    out = {k: np.zeros((4, T), dtype=np.complex128) for k in ("rest", "mixed_snk", "mixed_src", "dist", "full")}
    Smat_all = S.reshape(n, L ** 3 * T, 4, 3)
    for t in range(T):
        St = Smat_all[:, t * Vs:(t + 1) * Vs].reshape(n, n).T   # rows: sink (m, alpha, a); cols: source
        Xb = box_full(V_all[t])
        Xr = np.eye(n) - Xb
        for ch, G in enumerate(g.CHANNELS):
            G1 = spin_full(g.GAMMA5 @ G)
            G2 = spin_full(G @ g.GAMMA5)

            def C(X, Y):
                return np.trace(G1 @ X @ St @ G2 @ Y @ np.conj(St.T))

            out["rest"][ch, t] = C(Xr, Ysrc["rest"])
            out["mixed_snk"][ch, t] = C(Xb, Ysrc["rest"])
            out["mixed_src"][ch, t] = C(Xr, Ysrc["box"])
            out["dist"][ch, t] = C(Xb, Ysrc["box"])
            out["full"][ch, t] = C(np.eye(n), np.eye(n))
    return out


def point_sources(L, T, tp):
    """[Vs, 4, 3, V, 4, 3] unit sources delta_y e_beta e_b for every y on t'."""
    Vs = L ** 3
    b = np.zeros((Vs, 4, 3, L ** 3 * T, 4, 3), dtype=np.complex128)
    for m in range(Vs):
        for a in range(4):
            for c in range(3):
                b[m, a, c, tp * Vs + m, a, c] = 1.0
    return b
