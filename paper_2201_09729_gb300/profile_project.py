"""Time the V(t)^dag psi projection (Eq. 1, Eq. 3) of the correlator pipeline
for profiling: nrhs seeded solutions on an L^3 x T lattice with N modes per
timeslice, on the tensor cores (default) and, with --fp64, on the FP64 CUDA
cores, e.g.

    ncu --metrics gpu__time_duration.sum --clock-control none --csv \\
        python -m paper_2201_09729_gb300.profile_project --nrhs 168

Prints the CUDA-event time of each call.
"""
import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--T", type=int, default=32)
    ap.add_argument("--N", type=int, default=32)
    ap.add_argument("--nrhs", type=int, default=168)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--fp64", action="store_true")
    a = ap.parse_args()
    if a.fp64:
        os.environ["DLMA_PROJECT_FP64"] = "1"
    import torch

    import synth
    from paper_2201_09729_gb300 import Context, build

    build.build()
    U = synth.gauge_field(a.L, a.T, 0.2, 20220126)
    ctx = Context(a.L, a.T, 0, 0)
    ctx.dlma_set_gauge(U)
    _, V = ctx.dlma_laplacian_eigs(-1, a.N, 1e-10, device_out=True)
    g = torch.Generator(device="cuda").manual_seed(3)
    psi = torch.randn((a.nrhs, a.L ** 3 * a.T, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
    for r in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.dlma_project(-1, V, psi)
        torch.cuda.synchronize()
        print(f"rep {r}: {1e3 * (time.perf_counter() - t0):.2f} ms "
              f"({'FP64 CUDA cores' if a.fp64 else 'tensor cores'}, {a.nrhs} solutions, N = {a.N})")
    ctx.close()


if __name__ == "__main__":
    main()
