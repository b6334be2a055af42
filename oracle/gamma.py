"""Euclidean gamma matrices in the chiral basis (test infrastructure, oracle only).

The paper takes the Wilson operator's notation from its reference [Bloch:2006cd]
(Section 1) and prints no gamma matrices. Reading used here:
  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3)
  gamma_4 = [[0, 1], [1, 0]]
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1)
All are Hermitian and satisfy {gamma_mu, gamma_nu} = 2 delta_mu_nu.
"""
import numpy as np

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)

_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = tuple(
    [_block(_Z2, -1j * s, 1j * s, _Z2) for s in SIGMA] + [_block(_Z2, _I2, _I2, _Z2)]
)
"""GAMMA[nu] for nu = 0, 1, 2, 3 = x, y, z, t (the paper's directions 1..4)."""

GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
