"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws random numbers and lays them out in the canonical formats of the
library boundary. It holds none of the method's arithmetic (no Dirac operator, no sign
function, no Krylov step); both sides receive the same arrays from here.

Canonical layouts (complex128, C order):
  links   U[4][Lt][Lz][Ly][Lx][3][3]   direction index 0..3 = x, y, z, t; U[nu][site][a][b]
  spinor  psi[Lt][Lz][Ly][Lx][4][3]   spin then colour, colour fastest
  site    ((t*Lz + z)*Ly + y)*Lx + x

Workload recipe (stands in for the quenched beta=5.1 configurations of the paper's
numerical section, which are not available): links U = exp(i*eps*H) with H a random
traceless Hermitian 3x3 matrix per link, eps = 0.5, seed = field id; sources with
i.i.d. Gaussian real and imaginary parts (seed 1000 + request id) or b = (1,...,1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "gauge_links",
    "gaussian_source",
    "ones_source",
    "random_su3_field",
    "unit_links",
]


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _exp_i_eps_h(g: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for H = (G+G^H)/2 - tr/3, batched over leading axes, via eigh."""
    h = 0.5 * (g + np.conj(np.swapaxes(g, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1)
    h = h - (tr / 3.0)[..., None, None] * np.eye(3)
    w, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ab,...b,...cb->...ac", q, ph, np.conj(q))


def gauge_links(dims, seed: int, eps: float = 0.5) -> np.ndarray:
    """SU(3) links U = exp(i*eps*H), drawn in the order [nu][t][z][y][x][3][3][re,im]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((4, lt, lz, ly, lx, 3, 3, 2))
    g = raw[..., 0] + 1j * raw[..., 1]
    return np.ascontiguousarray(_exp_i_eps_h(g, eps))


def unit_links(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    lx, ly, lz, lt = (int(d) for d in dims)
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def random_su3_field(dims, seed: int) -> np.ndarray:
    """One random SU(3) matrix per site, G[Lt][Lz][Ly][Lx][3][3] (gauge transformations)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((lt, lz, ly, lx, 3, 3, 2))
    g = raw[..., 0] + 1j * raw[..., 1]
    return np.ascontiguousarray(_exp_i_eps_h(g, 2.0))


def gaussian_source(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Gaussian source(s): real and imaginary parts i.i.d. N(0,1).

    Returns psi[Lt][Lz][Ly][Lx][4][3] (nrhs None) or [nrhs][Lt][Lz][Ly][Lx][4][3].
    """
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    shape = (1 if nrhs is None else int(nrhs), lt, lz, ly, lx, 4, 3, 2)
    raw = rng.standard_normal(shape)
    b = raw[..., 0] + 1j * raw[..., 1]
    return np.ascontiguousarray(b[0] if nrhs is None else b)


def ones_source(dims) -> np.ndarray:
    """The paper-shaped source b = (1, ..., 1)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return np.ones((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
