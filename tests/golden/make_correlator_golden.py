"""Writes tests/golden/oracle_correlators_precision_16c32_N2_R1.json by running
the FP64 oracle only (no GPU code): every correlator part of Eqs. 2-3 on a
declared subset of the 16^3 x 32 precision workload (kappa 0.1225, c_sw 1.0,
eps 0.2, source timeslice t' = 0), small enough for the oracle:

  * N_c = 2 Laplacian modes per timeslice (ARPACK on each of the 32 timeslices),
  * one Z2 x Z2 noise vector (the first of the workload's noise seed),
  * 4 N_c + 5 = 13 CGNE solves to true residual 1e-12, run in parallel
    processes (one thread each).

Stored: C_dist, C_rest, C_mixed, C_mixed_src and C = C_rest + 2 C_mixed + C_dist
for the channels (PS, V1, V2, V3), each complex [4][T], plus the Laplacian
eigenvalues and the gap above the cut on every timeslice.  The GPU test runs
the same subset through dlma_correlators with FP32 and FP16S inner solves and
reports each part's error against these values.

    python tests/golden/make_correlator_golden.py      (about 30 min on 8 cores)
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N_C, N_R, TOL = 2, 1, 1e-12
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_correlators_precision_16c32_N2_R1.json")


def _solve_one(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    import synth
    from oracle import dirac, solve
    j, b = args
    wl = synth.WORKLOADS["precision_16c32"]
    U, _ = synth.workload_inputs(wl, n_noise=1)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    x, it, res = solve.cgne(eo, b, tol=TOL, check_every=25)
    return j, x, it, res


def _modes(t):
    import synth
    from oracle import laplacian as lap
    wl = synth.WORKLOADS["precision_16c32"]
    U, _ = synth.workload_inputs(wl, n_noise=1)
    w, V = lap.lap_modes(lap.timeslice_links(U, wl.L, t), wl.L, N_C + 1)
    return t, w, V[:N_C]


def main():
    import numpy as np

    import synth
    from oracle import dlma

    wl = synth.WORKLOADS["precision_16c32"]
    _, eta = synth.workload_inputs(wl, n_noise=N_R)
    L, T, tp = wl.L, wl.T, wl.t_src[0]
    t0 = time.time()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"           # one thread per worker process
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        modes = sorted(pool.map(_modes, range(T)))
        lam = np.array([m[1][:N_C] for m in modes])
        gap = np.array([m[1][N_C] - m[1][N_C - 1] for m in modes])
        V_all = np.stack([m[2] for m in modes])
        bd = dlma.distillation_sources(V_all[tp], L, T, tp)
        bn = dlma.noise_sources(eta[0], V_all[tp], L, T, tp).reshape(5 * N_R, wl.volume, 4, 3)
        b = np.concatenate([bd, bn])
        sols = sorted(pool.map(_solve_one, list(enumerate(b))), key=lambda r: r[0])
    x = np.stack([s[1] for s in sols])
    iters = [int(s[2]) for s in sols]
    resid = [float(s[3]) for s in sols]
    phid = x[:4 * N_C]
    phin = x[4 * N_C:].reshape(N_R, 5, wl.volume, 4, 3)
    tau = dlma.perambulator(V_all, phid, L, T)
    parts = {"C_dist": dlma.c_dist(tau)}
    parts["C_rest"], parts["C_mixed"] = dlma.noise_parts(V_all, phin[:, 0], phin[:, 1], phin[:, 2:5], L, T)
    parts["C_mixed_src"] = dlma.mixed_src(V_all, phid, L, T)
    parts["C"] = parts["C_rest"] + 2 * parts["C_mixed"] + parts["C_dist"]
    out = {
        "workload": wl.name, "subset": f"N_c = {N_C}, {N_R} Z2xZ2 noise vector (noise seed "
                                       f"{synth.NOISE_SEED_BASE + wl.cfg}, first vector), t' = {tp}",
        "n_modes": N_C, "n_noise": N_R, "t_src": tp, "solve_tol": TOL,
        "solve_iterations": iters, "solve_true_residuals": resid,
        "laplacian_eigenvalues": lam.tolist(), "gap_above_cut": gap.tolist(),
        "channels": ["PS", "V1", "V2", "V3"],
        "parts": {k: {"re": v.real.tolist(), "im": v.imag.tolist()} for k, v in parts.items()},
        "seconds": time.time() - t0,
        "written_by": "tests/golden/make_correlator_golden.py (oracle only)",
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: out[k] for k in ("subset", "solve_iterations", "seconds")}))


if __name__ == "__main__":
    main()
