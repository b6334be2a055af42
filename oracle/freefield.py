"""Closed-form sign(H_W(mu)) psi for unit links, any lattice size (oracle only).

Derivation (from the operator reading in ``wilson``): a plane wave e^{ip.x} u with
p_nu = 2 pi n_nu / L_nu (spatial) and p_t = pi (2 n_t + 1)/L_t (antiperiodic time; 2 pi n_t/L_t
for periodic) gives, with ptilde_nu = p_nu - i mu delta_{nu,t},
   D_W(p) = a(p) + i sum_nu gamma_nu s_nu(p),   a = 1 - 2 kappa sum_nu cos ptilde_nu,
   s_nu = 2 kappa sin ptilde_nu,
so H_W(p) = gamma5 D_W(p) squares to (a^2 + sum s_nu^2) times the identity and
sign(H_W(p)) = H_W(p) / sqrt(a^2 + sum s_nu^2) with the principal root (eigenvalues
+-sqrt(.), sign taken on the real part as in the paper's definition of sign z).
The same momentum-space matrices give D_W psi and the free spectrum.
"""
from __future__ import annotations

import numpy as np

from .gamma import GAMMA, GAMMA5
from .wilson import kappa


def _momenta(dims, t_bc):
    lx, ly, lz, lt = dims
    pt = 2 * np.pi * np.fft.fftfreq(lt) * 1.0
    if t_bc == -1:
        pt = pt + np.pi / lt
    pz = 2 * np.pi * np.fft.fftfreq(lz)
    py = 2 * np.pi * np.fft.fftfreq(ly)
    px = 2 * np.pi * np.fft.fftfreq(lx)
    return np.meshgrid(pt, pz, py, px, indexing="ij")  # arrays [Lt][Lz][Ly][Lx]


def symbol(dims, m_w, mu, t_bc=-1):
    """Per-momentum a(p), s_nu(p) (nu = x,y,z,t) on the FFT grid [Lt][Lz][Ly][Lx]."""
    dims = tuple(int(d) for d in dims)
    k = kappa(m_w)
    pt, pz, py, px = _momenta(dims, t_bc)
    ptil = [px, py, pz, pt - 1j * mu]
    a = 1.0 - 2.0 * k * sum(np.cos(p) for p in ptil)
    s = [2.0 * k * np.sin(p) for p in ptil]
    return a, s


def _dw_matrices(dims, m_w, mu, t_bc):
    a, s = symbol(dims, m_w, mu, t_bc)
    eye = np.eye(4, dtype=np.complex128)
    dp = a[..., None, None] * eye
    for nu in range(4):
        dp = dp + 1j * s[nu][..., None, None] * GAMMA[nu]
    return dp, a, s


def _apply_momentum(psi, mats, t_bc):
    """Apply a per-momentum 4x4 spin matrix (identity in colour) to psi[...][Lt][Lz][Ly][Lx][4][3]."""
    lt = psi.shape[-6]
    t = np.arange(lt).reshape(lt, 1, 1, 1, 1, 1)
    twist = np.exp(1j * np.pi * t / lt) if t_bc == -1 else np.ones_like(t, dtype=np.complex128)
    phi = psi / twist
    axes = (-6, -5, -4, -3)
    ft = np.fft.fftn(phi, axes=axes)
    ft = np.einsum("...st,...tc->...sc", mats, ft)
    return np.fft.ifftn(ft, axes=axes) * twist


def apply_dw_free(psi, dims, m_w, mu, t_bc=-1):
    dp, _, _ = _dw_matrices(dims, m_w, mu, t_bc)
    return _apply_momentum(psi, dp, t_bc)


def sign_hw_free(psi, dims, m_w, mu, t_bc=-1):
    """x* = sign(H_W(mu)) psi for unit links (exact up to FFT rounding)."""
    dp, a, s = _dw_matrices(dims, m_w, mu, t_bc)
    hp = np.einsum("st,...tu->...su", GAMMA5, dp)
    e2 = a * a + sum(x * x for x in s)
    root = np.sqrt(e2.astype(np.complex128))  # principal branch
    return _apply_momentum(psi, hp / root[..., None, None], t_bc)


def dw_free_spectrum(dims, m_w, mu, t_bc=-1):
    """Eigenvalues of the free D_W: a(p) +- i sqrt(sum s_nu^2), each 6-fold (2 spin x 3 colour)."""
    _, a, s = _dw_matrices(dims, m_w, mu, t_bc)
    r = np.sqrt(sum(x * x for x in s).astype(np.complex128))
    ev = np.concatenate([(a + 1j * r).ravel(), (a - 1j * r).ravel()])
    return np.repeat(ev, 6)


def hw_free_gap(dims, m_w, mu, t_bc=-1):
    """min |Re lambda| over eigenvalues +-sqrt(a^2 + sum s^2) of the free H_W."""
    _, a, s = _dw_matrices(dims, m_w, mu, t_bc)
    root = np.sqrt((a * a + sum(x * x for x in s)).astype(np.complex128))
    return float(np.min(np.abs(root.real)))
