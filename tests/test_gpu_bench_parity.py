"""Element-by-element parity of the projections and contractions at the size
and in the launch configuration the benchmark runs: the 16^3 x 32 workload,
N = 32 Laplacian modes per timeslice (computed by the library), 4N + 5 N_r =
168 right-hand sides (N_r = 8).  The "solutions" are seeded Gaussian fields
drawn on the device (no solve is needed for this parity), so every site tile,
every grid-y block of the projection and the source-side Box term over 32
modes run exactly as in the benchmark.  The oracle computes sampled
timeslices (the contractions are local in t): coefficients V(t)^dag psi to
1e-12, and C_dist, C_rest, C_mixed, C_mixed_src, C to 1e-12 of max |C| per
channel."""
import numpy as np
import pytest

import synth
from oracle import dlma

pytestmark = pytest.mark.gpu

T_SAMPLE = (0, 9, 31)


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def test_projection_and_contraction_at_bench_size(dl):
    import torch

    wl = synth.WORKLOADS["precision_16c32"]
    U, _ = synth.workload_inputs(wl)
    N, nn, L, T, Vs = wl.n_modes, wl.n_noise, wl.L, wl.T, wl.vol_s
    J = 4 * N + 5 * nn
    assert J == 168
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    _, Vd = ctx.dlma_laplacian_eigs(-1, N, 1e-10, device_out=True)        # [T, N, Vs, 3] on the device
    gen = torch.Generator(device="cuda").manual_seed(20221126)
    phi = torch.complex(torch.randn((J, wl.volume, 4, 3), dtype=torch.float64, device="cuda", generator=gen),
                        torch.randn((J, wl.volume, 4, 3), dtype=torch.float64, device="cuda", generator=gen))
    got = ctx.dlma_contract(0, Vd, phi, nn)
    coeff = ctx.dlma_project(-1, Vd, phi).cpu().numpy()                    # [J, T, 4, N]
    # sampled timeslices as a lattice of their own (contractions and projections are local in t)
    Ts = len(T_SAMPLE)
    V_s = np.ascontiguousarray(Vd[list(T_SAMPLE)].cpu().numpy())          # [Ts, N, Vs, 3]
    ph = np.concatenate([phi[:, t * Vs:(t + 1) * Vs].cpu().numpy() for t in T_SAMPLE], axis=1)
    del phi
    torch.cuda.empty_cache()
    for i, t in enumerate(T_SAMPLE):
        w = dlma.coeffs(V_s[i], ph[:, i * Vs:(i + 1) * Vs])               # [J, k, alpha]
        assert np.abs(coeff[:, t] - np.transpose(w, (0, 2, 1))).max() <= 1e-12 * np.abs(w).max()
    tau = dlma.perambulator(V_s, ph[:4 * N], L, Ts)
    noise = ph[4 * N:].reshape(nn, 5, Ts * Vs, 4, 3)
    rest, mixed = dlma.noise_parts(V_s, noise[:, 0], noise[:, 1], noise[:, 2:5], L, Ts)
    want = {"C_dist": dlma.c_dist(tau), "C_rest": rest, "C_mixed": mixed,
            "C_mixed_src": dlma.mixed_src(V_s, ph[:4 * N], L, Ts)}
    want["C"] = want["C_rest"] + 2 * want["C_mixed"] + want["C_dist"]
    for key, w in want.items():
        g = got[key][:, list(T_SAMPLE)]
        scale = np.abs(w).max(axis=1, keepdims=True)
        assert np.all(np.abs(g - w) <= 1e-12 * scale), (key, (np.abs(g - w) / scale).max())
