"""Pins for the oracle's Wilson operator (no GPU).

The paper defers D_W to its reference; these tests pin the reading by properties it must
have: Clifford algebra, gamma5-hermiticity gamma5 D_W(mu) gamma5 = D_W(-mu)^H (so that
H_W(mu)^H = H_W(-mu)), Hermiticity of H_W at mu = 0, gauge covariance, translation
covariance, the free-field spectrum in closed form, and agreement of three independent
constructions (dense, sparse, matrix-free) plus a site-by-site evaluation.
"""
import numpy as np
import pytest

import synth
from oracle import deflation, freefield, wilson
from oracle.gamma import GAMMA, GAMMA5

SMALL = [(2, 2, 2, 2), (2, 4, 2, 4), (4, 2, 2, 2)]


def test_gamma_algebra():
    for g in GAMMA:
        assert np.allclose(g, np.conj(g).T)
    for m in range(4):
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2.0 * (m == n) * np.eye(4))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))
    for g in GAMMA:
        assert np.allclose(GAMMA5 @ g + g @ GAMMA5, 0)


@pytest.mark.parametrize("dims", SMALL)
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_three_constructions_agree(dims, t_bc):
    u = synth.gauge_links(dims, 3)
    psi = synth.gaussian_source(dims, 7)
    d = wilson.dense_dw(u, dims, -2.0, 0.3, t_bc)
    y_dense = (d @ psi.ravel()).reshape(psi.shape)
    y_mf = wilson.apply_dw(u, psi, -2.0, 0.3, t_bc)
    h_sp = deflation.sparse_hw(u, dims, -2.0, 0.3, t_bc)
    y_sp = (h_sp @ psi.ravel()).reshape(psi.shape)
    vol = synth.volume(dims)
    sites = np.arange(vol)
    y_site = wilson.apply_dw_at_sites(u, psi, -2.0, 0.3, sites, t_bc).reshape(psi.shape)
    assert np.abs(y_dense - y_mf).max() < 1e-13
    assert np.abs(y_site - y_mf).max() < 1e-13
    assert np.abs(wilson.apply_gamma5(y_mf) - y_sp).max() < 1e-13


@pytest.mark.parametrize("dims", SMALL)
def test_gamma5_hermiticity(dims):
    u = synth.gauge_links(dims, 4)
    for mu in (0.0, 0.3, 1.0):
        h = wilson.dense_hw(u, dims, -2.0, mu)
        hm = wilson.dense_hw(u, dims, -2.0, -mu)
        assert np.abs(np.conj(h).T - hm).max() < 1e-14
    h0 = wilson.dense_hw(u, dims, -2.0, 0.0)
    assert np.abs(h0 - np.conj(h0).T).max() < 1e-14
    # mu != 0 really is non-Hermitian
    h3 = wilson.dense_hw(u, dims, -2.0, 0.3)
    assert np.abs(h3 - np.conj(h3).T).max() > 1e-2


def test_hop_structure_free_diagonal():
    """Diagonal blocks are the identity (m_q = 0, kappa form); kappa = 1/4 at m_W = -2."""
    dims = (2, 4, 2, 4)
    u = synth.gauge_links(dims, 5)
    d = wilson.dense_dw(u, dims, -2.0, 0.3)
    vol = synth.volume(dims)
    for s in range(vol):
        blk = d[12 * s:12 * s + 12, 12 * s:12 * s + 12]
        assert np.allclose(blk, np.eye(12))
    assert wilson.kappa(-2.0) == 0.25


def test_gauge_covariance():
    dims = (4, 2, 4, 2)
    u = synth.gauge_links(dims, 6)
    g = synth.random_su3_field(dims, 8)
    psi = synth.gaussian_source(dims, 9)
    ug = wilson.gauge_transform(u, g)
    lhs = wilson.apply_hw(ug, wilson.gauge_transform_spinor(psi, g), -2.0, 0.3)
    rhs = wilson.gauge_transform_spinor(wilson.apply_hw(u, psi, -2.0, 0.3), g)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_translation_covariance():
    dims = (4, 4, 2, 4)
    u = synth.gauge_links(dims, 10)
    psi = synth.gaussian_source(dims, 11)
    # shift by one site in y (axis 2 of [t][z][y][x]); spatial shifts commute with BCs
    us = np.roll(u, 1, axis=3)
    ps = np.roll(psi, 1, axis=2)
    lhs = wilson.apply_dw(us, ps, -2.0, 0.3)
    rhs = np.roll(wilson.apply_dw(u, psi, -2.0, 0.3), 1, axis=2)
    assert np.abs(lhs - rhs).max() < 1e-13


@pytest.mark.parametrize("t_bc", [-1, 1])
def test_free_field_momentum_space(t_bc):
    dims = (4, 2, 2, 4)
    u = synth.unit_links(dims)
    psi = synth.gaussian_source(dims, 12)
    y = wilson.apply_dw(u, psi, -2.0, 0.3, t_bc)
    yf = freefield.apply_dw_free(psi, dims, -2.0, 0.3, t_bc)
    assert np.abs(y - yf).max() < 1e-13


def test_free_field_spectrum_closed_form():
    dims = (2, 2, 2, 4)
    u = synth.unit_links(dims)
    d = wilson.dense_dw(u, dims, -2.0, 0.3)
    ev = np.linalg.eigvals(d)
    ref = freefield.dw_free_spectrum(dims, -2.0, 0.3)
    key = lambda z: (round(z.real, 8), round(z.imag, 8))
    a = sorted(ev, key=key)
    b = sorted(ref, key=key)
    assert np.abs(np.array(a) - np.array(b)).max() < 1e-10


def test_periodic_time_free_zero_modes():
    """Periodic time at m_W = -2 has exact free zero modes: sign is undefined there."""
    assert freefield.hw_free_gap((4, 4, 4, 4), -2.0, 0.0, t_bc=1) < 1e-12
    assert freefield.hw_free_gap((4, 4, 4, 4), -2.0, 0.0, t_bc=-1) > 0.3
