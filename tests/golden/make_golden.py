"""Writes tests/golden/oracle_cgne_precision_16c32.json by running the FP64
oracle only (no GPU code): the number of CGNE iterations the oracle needs to
reach the true residual 1e-10 on the 16^3 x 32 precision workload (kappa
0.1225, c_sw 1.0, eps 0.2) for a Z2 x Z2 noise source on t' = 0, and the
seconds per iteration on this machine.  The benchmark's CPU baseline scales a
short timed slice of oracle iterations by this count.

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import dirac, solve  # noqa: E402


def main():
    wl = synth.WORKLOADS["precision_16c32"]
    U, eta = synth.workload_inputs(wl, n_noise=1)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    b = np.zeros((wl.volume, 4, 3), dtype=np.complex128)
    b[: wl.vol_s] = eta[0, 0]
    t0 = time.time()
    x, iters, res = solve.cgne(eo, b, tol=wl.tol, check_every=25)
    dt = time.time() - t0
    out = {
        "workload": wl.name,
        "source": f"Z2xZ2 noise on t'=0 (noise seed {synth.NOISE_SEED_BASE + wl.cfg}, first vector)",
        "tol": wl.tol,
        "iterations": int(iters),
        "true_residual": float(res),
        "seconds": dt,
        "seconds_per_iteration": dt / iters,
        "threads": os.cpu_count(),
        "written_by": "tests/golden/make_golden.py (oracle only)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cgne_precision_16c32.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
