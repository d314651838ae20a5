"""Dirac matrices in the chiral basis.

The paper never fixes a basis (Sec. 1 only names gamma_mu, gamma_nu and
gamma_5).  Reading used here: chiral basis with 2x2 blocks
    gamma_0 = -[[0, 1], [1, 0]],  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
    gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).
mu = 0 is time, mu = 1, 2, 3 the spatial directions j of Eq. 1.
Correlators built with Gamma and the distillation projector are
basis-independent; the noise vectors are basis-dependent but seed-fixed.
"""
import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def gammas() -> np.ndarray:
    """gamma_mu, mu = 0..3, as a [4, 4, 4] array."""
    g0 = np.block([[_Z2, -_I2], [-_I2, _Z2]])
    gk = [np.block([[_Z2, -1j * PAULI[k]], [1j * PAULI[k], _Z2]]) for k in range(3)]
    return np.array([g0] + gk)


GAMMA = gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# Channels of the connected correlators: Gamma = gamma_5 (pseudoscalar) and
# Gamma = gamma_k, k = 1, 2, 3 (vector; averaged over k).
CHANNELS = (GAMMA5, GAMMA[1], GAMMA[2], GAMMA[3])
CHANNEL_NAMES = ("PS", "V1", "V2", "V3")
