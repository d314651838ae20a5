"""Run the batched Laplacian eigensolver (all timeslices) on a synthetic gauge
field for profiling, e.g.

    ncu --metrics gpu__time_duration.sum --clock-control none --csv \\
        python -m paper_2201_09729_gb300.profile_eigs --L 16 --T 32 --N 32

Prints the CUDA-event time, the FP32 / FP64 iteration counts and the split
of the time into Laplacian applications (matvec) and orthogonalisation
(Gram matrices, small eigenproblems, rotations, residuals) of each run --
the two columns of the paper's Table 2.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--T", type=int, default=32)
    ap.add_argument("--N", type=int, default=32)
    ap.add_argument("--eps", type=float, default=0.2)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()

    import synth
    from paper_2201_09729_gb300 import Context, build

    build.build()
    U = synth.gauge_field(a.L, a.T, a.eps, 20220126)
    ctx = Context(a.L, a.T, 0, 0)
    ctx.dlma_set_gauge(U)
    for r in range(a.reps):
        lam, _ = ctx.dlma_laplacian_eigs(-1, a.N, a.tol, want_vecs=False)
        ms, it32, it64, mv, ortho, host = ctx.dlma_last_timing()[:6]
        print(f"rep {r}: {ms:.1f} ms (matvec {mv:.1f}, orthogonalisation {ortho:.1f}, host {host:.1f}), "
              f"iterations fp32 {int(it32)} fp64 {int(it64)}, lam[0] {lam[0, 0]:.6f} lam[N-1] {lam[0, -1]:.6f}")
    ctx.close()


if __name__ == "__main__":
    main()
