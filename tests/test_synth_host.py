"""The seeded input generators shared by both sides (no GPU): shapes and canonical layouts, the
SU(3) property the FP16 12-real links rely on (row 3 = conj(row 1 x row 2) holds only for unitary
matrices of determinant 1), the traceless Hermitian generator's spread, and reproducibility."""
import numpy as np

import synth


def test_links_are_su3_in_the_canonical_layout():
    dims = (2, 4, 6, 8)
    u = synth.gauge_links(dims, 3)
    assert u.shape == (4, 8, 6, 4, 2, 3, 3) and u.dtype == np.complex128 and u.flags["C_CONTIGUOUS"]
    m = u.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(np.einsum("nab,ncb->nac", m, m.conj()) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(m) - 1.0).max() < 1e-13
    # the third row is conj(row 1 x row 2), as the 12-real format reconstructs it
    r3 = np.conj(np.cross(m[:, 0, :], m[:, 1, :]))
    assert np.abs(r3 - m[:, 2, :]).max() < 1e-13


def test_link_spread_follows_eps():
    """U = exp(i eps H): the eigenvalue phases of U are eps times the eigenvalues of the same H (the
    draws do not depend on eps, and eps |w| stays below pi here), so their mean modulus scales
    linearly in eps; eps = 0 is the free field."""
    dims = (4, 4, 4, 4)
    assert np.abs(synth.gauge_links(dims, 0, eps=0.0) - synth.unit_links(dims)).max() < 1e-14
    spread = []
    for eps in (0.1, 0.5):
        w = np.linalg.eigvals(synth.gauge_links(dims, 0, eps=eps).reshape(-1, 3, 3))
        assert np.abs(np.abs(w) - 1.0).max() < 1e-13
        spread.append(np.abs(np.angle(w)).mean())
    assert abs(spread[1] / spread[0] - 5.0) < 1e-9
    assert 0.1 < spread[0] < 0.2  # mean |eigenvalue| of the traceless Hermitian H is about 1.4


def test_gauge_transformations_are_su3():
    g = synth.random_su3_field((2, 2, 2, 4), 9).reshape(-1, 3, 3)
    assert np.abs(np.einsum("nab,ncb->nac", g, g.conj()) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(g) - 1.0).max() < 1e-13


def test_sources_shapes_and_statistics():
    dims = (4, 4, 4, 8)
    b = synth.gaussian_source(dims, 1000)
    bb = synth.gaussian_source(dims, 1000, nrhs=3)
    assert b.shape == (8, 4, 4, 4, 4, 3) and bb.shape == (3, 8, 4, 4, 4, 4, 3)
    assert np.array_equal(bb[0], b)  # the first source of a batch is the single source of that seed
    n = b.size
    # i.i.d. N(0,1) real and imaginary parts: E|b_i|^2 = 2 (within a few standard errors)
    assert abs(np.mean(np.abs(bb) ** 2) - 2.0) < 5 * 2.0 / np.sqrt(3 * n)
    assert np.array_equal(synth.ones_source(dims), np.ones_like(b))


def test_reproducible_and_seed_dependent():
    dims = (2, 2, 2, 2)
    assert np.array_equal(synth.gauge_links(dims, 5), synth.gauge_links(dims, 5))
    assert not np.array_equal(synth.gauge_links(dims, 5), synth.gauge_links(dims, 6))
    assert np.array_equal(synth.gaussian_source(dims, 7), synth.gaussian_source(dims, 7))
    assert synth.volume(dims) == 16
