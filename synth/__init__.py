"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module draws random numbers and lays them out in the canonical host
layout; it contains none of the method's arithmetic (no Dirac operator, no
Laplacian, no projector, no contraction).  Both the oracle and the GPU
library consume exactly the arrays produced here.

Canonical layout (complex128, C order):
  * site index  s = x + L*(y + L*(z + L*t))   (t slowest: every timeslice is a
    contiguous block of L^3 sites);
  * links       U[s, mu, a, b]  with mu = 0 time, mu = 1, 2, 3 the x, y, z
    directions, (a, b) the SU(3) row / column;
  * spinors     psi[s, alpha, c] with alpha the Dirac index (4), c colour (3).

Workloads (the paper's ensembles are 64 x 32^3 CLS fields with O(a)-improved
Wilson quarks, Table 1; these synthetic near-unit SU(3) fields of the same or
smaller shape stand in for them):
  GAUGE_SEED_BASE + cfg    link generator,
  NOISE_SEED_BASE + cfg    Z2 x Z2 noise,
  WEIGHT_SEED_BASE + cfg   w(t) weights of the differentiable loss.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GAUGE_SEED_BASE = 20220124
NOISE_SEED_BASE = GAUGE_SEED_BASE + 1000
WEIGHT_SEED_BASE = GAUGE_SEED_BASE + 2000


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: lattice L^3 x T, gauge roughness eps, kappa,
    c_sw, N_c Laplacian modes per timeslice, N_r noise vectors per source
    timeslice, the source timeslices and the target true residual."""

    name: str
    L: int
    T: int
    eps: float
    kappa: float
    csw: float
    n_modes: int
    n_noise: int
    t_src: tuple
    tol: float
    cfg: int

    @property
    def m0(self) -> float:
        # bare mass of the m0-normalised Wilson operator, m0 = 1/(2 kappa) - 4
        return 1.0 / (2.0 * self.kappa) - 4.0

    @property
    def volume(self) -> int:
        return self.L ** 3 * self.T

    @property
    def vol_s(self) -> int:
        return self.L ** 3


# The five workloads of the hot-path scope: plain FP64 (4^3x8), precision
# form (16^3x32), batched form (24^3x48), differentiation form (16^3x32) and
# the full pipeline at the paper's lattice shape (32^3x64).
WORKLOADS = {
    "plain_4c8": Workload("plain_4c8", 4, 8, 0.2, 0.120, 1.0, 8, 2, (0,), 1e-12, 1),
    "precision_16c32": Workload("precision_16c32", 16, 32, 0.2, 0.1225, 1.0, 32, 8, (0,), 1e-10, 2),
    "batched_24c48": Workload("batched_24c48", 24, 48, 0.25, 0.1225, 1.2, 64, 16, (0, 12, 24, 36), 1e-10, 3),
    "grad_16c32": Workload("grad_16c32", 16, 32, 0.2, 0.1225, 1.0, 32, 4, (0,), 1e-10, 4),
    "full_32c64": Workload("full_32c64", 32, 64, 0.3, 0.1230, 1.5, 96, 32, (0,), 1e-10, 5),
}


def _gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a (a = 1..8) as an [8, 3, 3] array."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Project [..., 3, 3] matrices back onto SU(3): Gram-Schmidt on rows 1
    and 2, row 3 = conj(row1 x row2)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def gauge_field(L: int, T: int, eps: float, seed: int) -> np.ndarray:
    """Random near-unit SU(3) links U_mu(x) = exp(i eps sum_a w_a lambda_a / 2),
    w_a ~ N(0, 1) drawn in site-lexicographic order (t, z, y, x slowest first),
    then mu, then a; reunitarised.  Returns complex128 [V, 4, 3, 3]."""
    V = L ** 3 * T
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((V, 4, 8))
    H = np.einsum("sma,aij->smij", w, _gell_mann()) * 0.5
    h, W = np.linalg.eigh(H)
    U = np.einsum("smij,smj,smkj->smik", W, np.exp(1j * eps * h), np.conj(W))
    return np.ascontiguousarray(_reunitarise(U))


def unit_gauge(L: int, T: int) -> np.ndarray:
    """The free field U_mu(x) = 1."""
    V = L ** 3 * T
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def random_su3(n: int, seed: int) -> np.ndarray:
    """n Haar-ish random SU(3) matrices (QR of complex Gaussians, phases fixed,
    determinant divided out); used for random gauge transformations G(x)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return _reunitarise(q)


def z2z2_noise(n: int, vol_s: int, seed: int) -> np.ndarray:
    """n Z2 x Z2 noise vectors on one timeslice, every spin-colour-site
    component drawn from {(+-1 +- i)/sqrt 2} with two independent bits.
    Returns complex128 [n, vol_s, 4, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bits = rng.integers(0, 2, size=(n, vol_s, 4, 3, 2))
    sgn = 1.0 - 2.0 * bits.astype(np.float64)
    return (sgn[..., 0] + 1j * sgn[..., 1]) / np.sqrt(2.0)


def wall_noise(n: int, vol_s: int, seed: int) -> np.ndarray:
    """n Z2 x Z2 wall-noise vectors on one timeslice: one number per site and
    colour (no spin index) from {(+-1 +- i)/sqrt 2}, two independent bits each.
    Returns complex128 [n, vol_s, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bits = rng.integers(0, 2, size=(n, vol_s, 3, 2))
    sgn = 1.0 - 2.0 * bits.astype(np.float64)
    return (sgn[..., 0] + 1j * sgn[..., 1]) / np.sqrt(2.0)


def gaussian_spinors(n: int, V: int, seed: int) -> np.ndarray:
    """n complex Gaussian spinor fields [n, V, 4, 3] (test vectors)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, V, 4, 3)) + 1j * rng.standard_normal((n, V, 4, 3))


def loss_weights(T: int, seed: int) -> np.ndarray:
    """w(t) ~ N(0, 1), t = 0..T-1, for the scalar loss sum_t w(t) Re C_PS(t)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(T)


def workload_inputs(wl: Workload, n_noise: int | None = None):
    """Gauge field and noise for a named workload.  Returns (U, eta) with
    eta [len(t_src), n_noise, vol_s, 4, 3]."""
    U = gauge_field(wl.L, wl.T, wl.eps, GAUGE_SEED_BASE + wl.cfg)
    nn = wl.n_noise if n_noise is None else n_noise
    eta = z2z2_noise(nn * len(wl.t_src), wl.vol_s, NOISE_SEED_BASE + wl.cfg)
    eta = eta.reshape(len(wl.t_src), nn, wl.vol_s, 4, 3)
    return U, eta
