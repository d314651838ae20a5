"""The cost model of the paper's last section (Eqs. 6-9) and a GPU sweep over
the number of Laplacian modes per timeslice.

Eq. 6 balances the time spent on distillation against more stochastic sources:
    t_{N/4, l} + t_{N, D} + 2 t_{R1, D} = t_{R0, D},
the time of the Laplacian modes, of the N distillation solves (N = 4 N_c Dirac
sources for N_c colour modes) and of two solves per stochastic source with
distillation (phi and phibar) buys R0 stochastic sources of one solve each
without it.  With a common time t_D per solve and t_{R, D} = R t_D:
    R0 = 2 R1 + N + t_{N/4, l} / t_D,
whose t_{N/4, l} -> 0 limit is the bound R0 > 2 R1 + N of Eq. 7.  Since the
variance of the correlator scales as 1/R (Eq. 8), distillation pays off only if
the stochastic remainder 1 - C_dist/C is at most R1/R0 <= 1/(N/R1 + 2) (Eq. 9).

`sweep` measures t_{N/4, l} (the batched eigensolve), the time per solve and
C_dist/C on the GPU for several N_c, through the library's public calls.

    python -m paper_2201_09729_gb300.costmodel --workload precision_16c32 --Nc 8 16 32 64
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def r0_equivalent(t_lap: float, n_dist: int, t_solve: float, r1: int, solves_per_noise: int = 2) -> float:
    """R0 of Eq. 6: the number of plain stochastic sources (one solve each) that
    cost as much as the modes (t_lap), n_dist distillation solves and r1
    stochastic sources with distillation (solves_per_noise solves each), every
    solve taking t_solve."""
    if not t_solve > 0:
        raise ValueError("t_solve must be positive")
    return (t_lap + n_dist * t_solve + solves_per_noise * r1 * t_solve) / t_solve


def rest_fraction_bound(n_dist: int, r1: int) -> float:
    """Eq. 9's right-hand side: 1 / (N / R1 + 2), the largest stochastic remainder
    1 - C_dist/C for which distillation can pay off even with free modes."""
    return 1.0 / (n_dist / r1 + 2.0)


def pays_off(c_dist_over_c: float, r1: int, r0: float) -> bool:
    """Eq. 9: 1 - C_dist/C <= R1 / R0."""
    return 1.0 - c_dist_over_c <= r1 / r0


def sweep(ctx, t_src: int, nc_list, eta, tol: float, inner: int, t_ratio: int | None = None):
    """For each N_c: time the eigensolve of all timeslices (split into its
    Laplacian applications and its orthogonalisation, the two columns of
    Table 2) and one source timeslice's correlators (4 N_c + 5 n_noise solves),
    and evaluate Eqs. 6-9 for the pseudoscalar channel at sink time t_ratio
    (default: T / 4 after t_src).  Every row also carries C_dist / C at every
    sink time for the pseudoscalar and for the vector channel (the average of
    gamma_1..3: the quantity Figs. 3 and 5 plot against the number of modes).
    eta: noise [n_noise, L^3, 4, 3] (numpy or a CUDA tensor)."""
    T = ctx.T
    tr = (t_src + T // 4) % T if t_ratio is None else t_ratio
    nn = int(eta.shape[0])
    rows = []
    for nc in nc_list:
        ctx.dlma_laplacian_eigs(-1, int(nc), 1e-10, want_vecs=False)
        tm = ctx.dlma_last_timing()
        t_lap = float(tm[0]) / 1e3
        r = ctx.dlma_correlators(t_src, int(nc), eta, tol, inner)
        t_corr = float(ctx.dlma_last_timing()[0]) / 1e3
        n_dist = 4 * int(nc)
        n_solves = n_dist + 5 * nn
        t_solve = t_corr / n_solves                # the paper's equal cost per source
        ratio = float(r["C_dist"][0][tr].real / r["C"][0][tr].real)
        cv_dist = r["C_dist"][1:4].real.mean(axis=0)
        cv = r["C"][1:4].real.mean(axis=0)
        r0 = r0_equivalent(t_lap, n_dist, t_solve, nn)
        rows.append({"Nc": int(nc), "N": n_dist, "R1": nn, "t_lap_s": t_lap, "t_solve_s": t_solve,
                     "t_lap_matvec_s": float(tm[3]) / 1e3, "t_lap_ortho_s": float(tm[4]) / 1e3,
                     "C_dist_over_C_PS": ratio, "t": tr, "R0": r0, "R1_over_R0": nn / r0,
                     "bound_eq9": rest_fraction_bound(n_dist, nn), "pays_off": pays_off(ratio, nn, r0),
                     "C_dist_over_C_PS_t": [float(x) for x in r["C_dist"][0].real / r["C"][0].real],
                     "C_dist_over_C_V_t": [float(x) for x in cv_dist / cv],
                     "converged": all(i["converged"] for i in r["info"])})
    return rows


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import synth
    from paper_2201_09729_gb300 import FP32, Context, build

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="precision_16c32")
    ap.add_argument("--Nc", type=int, nargs="+", default=[8, 16, 32, 64])
    a = ap.parse_args()
    build.build()
    wl = synth.WORKLOADS[a.workload]
    U, eta = synth.workload_inputs(wl)
    ctx = Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    rows = sweep(ctx, wl.t_src[0], a.Nc, eta[0], wl.tol, FP32)
    for row in rows:
        print(json.dumps(row))
    ctx.close()


if __name__ == "__main__":
    main()
