"""Pins for the oracle's dense matrix sign function (no GPU).

Definition: sign(A) = R diag(sign Re lambda) R^-1 (Section 1). Pins: a 2x2 closed form,
the Hermitian case (eigh), agreement of eig and scaled Newton, sign^2 = I, commutation,
sign(H_W(mu))^H = sign(H_W(-mu)), the Ginsparg-Wilson relation of D_ov = 1 + gamma5 sign(H_W),
and the free-field closed form.
"""
import numpy as np
import pytest

import synth
from oracle import freefield, matsign, wilson
from oracle.gamma import GAMMA5


def test_two_by_two_closed_form():
    # upper triangular, eigenvalues a > 0 > c: f(T)_12 = b (f(a) - f(c)) / (a - c)
    for a, b, c in [(2.0, 1.0, -0.5), (0.3, -2.0 + 1j, -4.0), (1.0 + 0.5j, 3.0, -1.0 - 2j)]:
        t = np.array([[a, b], [0, c]], dtype=np.complex128)
        ref = np.array([[1, 2 * b / (a - c)], [0, -1]])
        assert np.abs(matsign.sign_eig(t) - ref).max() < 1e-13
        s, _ = matsign.sign_newton(t)
        assert np.abs(s - ref).max() < 1e-13


def test_hermitian_eigh():
    rng = np.random.default_rng(1)
    g = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    h = g + np.conj(g).T
    s1 = matsign.sign_hermitian(h)
    s2 = matsign.sign_eig(h)
    s3, _ = matsign.sign_newton(h)
    assert np.abs(s1 - s2).max() < 1e-11
    assert np.abs(s1 - s3).max() < 1e-11


@pytest.fixture(scope="module")
def small_hw():
    dims = (2, 2, 2, 4)
    u = synth.gauge_links(dims, 21)
    return dims, u, wilson.dense_hw(u, dims, -2.0, 0.3), wilson.dense_hw(u, dims, -2.0, -0.3)


def test_sign_invariants(small_hw):
    dims, u, h, hm = small_hw
    s = matsign.sign_eig(h)
    sn, _ = matsign.sign_newton(h)
    n = h.shape[0]
    assert np.abs(s - sn).max() < 1e-11
    assert np.abs(s @ s - np.eye(n)).max() < 1e-11
    assert np.abs(s @ h - h @ s).max() < 1e-11
    smi = matsign.sign_eig(hm)
    assert np.abs(np.conj(s).T - smi).max() < 1e-11


def test_ginsparg_wilson(small_hw):
    dims, u, h, _ = small_hw
    vol = synth.volume(dims)
    g5 = np.kron(np.eye(vol), np.kron(GAMMA5, np.eye(3)))
    dov = np.eye(h.shape[0]) + g5 @ matsign.sign_eig(h)
    lhs = g5 @ dov + dov @ g5
    rhs = dov @ g5 @ dov
    assert np.abs(lhs - rhs).max() < 1e-11


def test_free_field_sign_closed_form():
    dims = (2, 2, 2, 4)
    u = synth.unit_links(dims)
    psi = synth.gaussian_source(dims, 22)
    for mu in (0.0, 0.3):
        h = wilson.dense_hw(u, dims, -2.0, mu)
        x_dense = matsign.sign_eig(h, psi.ravel()).reshape(psi.shape)
        x_free = freefield.sign_hw_free(psi, dims, -2.0, mu)
        assert np.abs(x_dense - x_free).max() < 1e-11


def test_ill_posed_detected():
    dims = (2, 2, 2, 4)
    h = wilson.dense_hw(synth.unit_links(dims), dims, -2.0, 0.0, t_bc=1)
    with pytest.raises(matsign.IllPosed):
        matsign.sign_eig(h)
