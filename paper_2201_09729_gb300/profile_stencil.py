"""Run the even-odd Schur stencil (two hop launches per application) on a
synthetic gauge field for profiling, e.g.

    ncu --set full --clock-control none -k regex:k_hop -s 2 -c 2 \\
        python -m paper_2201_09729_gb300.profile_stencil --prec fp32 --nrhs 32

Prints the CUDA-event time of each application and the algorithmic bytes.
With --sweep, every FP32 variant the autotuner chooses from (one or two
right-hand sides per thread, 12- or 18-real links; each with its best block
shape) is timed in a fresh context and reported; with --chunks, every chunk
size of the block order (DLMA_FORCE_CHUNK).
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
    ap.add_argument("--nrhs", type=int, default=32)
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "fp16s"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--chunks", action="store_true", help="time each chunk size of the block order")
    a = ap.parse_args()
    import torch

    import synth
    from bench import schur_bytes
    from paper_2201_09729_gb300 import FP16S, FP32, FP64, Context, build

    build.build()
    prec = {"fp64": FP64, "fp32": FP32, "fp16s": FP16S}[a.prec]
    U = synth.gauge_field(a.L, a.T, 0.2, 20220126)
    ctx = Context(a.L, a.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(1 / (2 * 0.1225) - 4, 1.0)
    Vh = a.L ** 3 * a.T // 2
    g = torch.Generator(device="cuda").manual_seed(1)
    v = torch.randn((a.nrhs, Vh, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
    by = schur_bytes(Vh, a.nrhs, a.prec)
    if a.chunks:
        ctx.close()
        for ch in (16, 32, 64, 128):
            os.environ["DLMA_FORCE_CHUNK"] = str(ch)
            c = Context(a.L, a.T, 0, 0)
            c.dlma_set_gauge(U)
            c.dlma_set_params(1 / (2 * 0.1225) - 4, 1.0)
            ms = []
            for r in range(a.reps + 1):
                c.dlma_apply_schur(v, 0, prec)
                ms.append(c.dlma_last_timing()[0])
            best = min(ms[1:])
            print(f"chunk {ch}: best {best:.3f} ms  {by / best / 1e6:.1f} GB/s algorithmic")
            c.close()
        return
    if a.sweep:
        ctx.close()
        for nr, links in ((1, 12), (1, 18), (2, 12), (2, 18)):
            os.environ["DLMA_FORCE_NR"], os.environ["DLMA_FORCE_LINKS"] = str(nr), str(links)
            c = Context(a.L, a.T, 0, 0)
            c.dlma_set_gauge(U)
            c.dlma_set_params(1 / (2 * 0.1225) - 4, 1.0)
            ms = []
            for r in range(a.reps + 1):
                c.dlma_apply_schur(v, 0, prec)
                ms.append(c.dlma_last_timing()[0])
            best = min(ms[1:])
            print(f"nr {nr} links {links}: best {best:.3f} ms  {by / best / 1e6:.1f} GB/s algorithmic")
            c.close()
        return
    for r in range(a.reps):
        ctx.dlma_apply_schur(v, 0, prec)
        ms = ctx.dlma_last_timing()[0]
        print(f"rep {r}: {ms:.3f} ms  {by / ms / 1e6:.1f} GB/s algorithmic ({by / 1e6:.1f} MB)")
    ctx.close()


if __name__ == "__main__":
    main()
