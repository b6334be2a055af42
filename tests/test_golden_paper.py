"""Pins from the values the paper prints (tests/golden/paper_values.txt, read through the
`paper` fixture): the matrix dimension Section 6 gives for each lattice, the parameter set of
Fig. 1 against Section 5's choice of the Neuberger scale and Theorem 1, and the parameters of
the timed configuration. No GPU.
"""
import math

import numpy as np
import pytest

import synth
from oracle import deflation, rational, wilson


@pytest.mark.parametrize("L", [4, 6, 8, 10])
def test_matrix_dimension_of_each_lattice(paper, L):
    """Section 6: n = 3,072 / 15,552 / 49,152 / 120,000 for 4^4 / 6^4 / 8^4 / 10^4, i.e. 12
    complex values per site (4 spins x 3 colours). A wrong spin or colour count, or a field of
    the wrong shape, changes n."""
    dims = (L,) * 4
    b = synth.ones_source(dims)
    assert b.size == int(paper["n_%d" % L])
    y = wilson.apply_hw(synth.gauge_links(dims, 0), b, paper["m_W"], paper["mu"])
    assert y.shape == b.shape and np.all(np.isfinite(y))


def test_sparse_operator_dimension_4444(paper):
    """The assembled H_W at 4^4 is n_4 x n_4, with the same action as the matrix-free operator
    on the paper's source b = (1, ..., 1)."""
    dims = (4, 4, 4, 4)
    u = synth.gauge_links(dims, 0)
    h = deflation.sparse_hw(u, dims, paper["m_W"], paper["mu"])
    n = int(paper["n_4"])
    assert h.shape == (n, n)
    b = synth.ones_source(dims)
    y = wilson.apply_hw(u, b, paper["m_W"], paper["mu"])
    assert np.abs(h @ b.ravel() - y.ravel()).max() < 1e-13


def test_fig1_scale_is_the_optimal_one(paper):
    """Fig. 1 uses c = 1/sqrt(10) with the Zolotarev interval [1, 10]. Section 5's optimal scale
    for a spectrum on [m - r, m + r] = [a, b], c = ((m + r)(m - r))^(-1/2), gives exactly that."""
    a, b = paper["fig1_zolotarev_a"], paper["fig1_zolotarev_b"]
    m, r = rational.circle_from_gap(a, b)
    assert (m - r, m + r) == (a, b)
    c, d = rational.scale_and_d(m, r)
    assert abs(c * c - paper["fig1_neuberger_c_sq"]) < 1e-15
    assert abs(d - math.sqrt(b / a)) < 1e-14


def test_fig1_neuberger_on_real_interval_and_circle(paper):
    """Fig. 1's Neuberger approximation (s = 10, c = 1/sqrt(10)): on [1, 10] the worst error is at
    both ends, 1 - tanh(2s atanh(c)) = 2 / (delta^(2s) + 1) with delta = (d + 1)/(d - 1); on the
    circle through 1 and 10 it stays within Theorem 1's 2 / (delta^(2s) - 1) and reaches it."""
    s = int(paper["fig1_s"])
    a, b = paper["fig1_zolotarev_a"], paper["fig1_zolotarev_b"]
    c = math.sqrt(paper["fig1_neuberger_c_sq"])
    w, sg = rational.neuberger_scaled(s, c)
    x = np.linspace(a, b, 100001)
    err = np.abs(rational.rational_eval(x, w, sg) - 1.0)
    d = math.sqrt(b / a)
    delta = (d + 1) / (d - 1)
    ends = 1.0 - math.tanh(2 * s * math.atanh(c * a))
    assert abs(ends - 2 / (delta ** (2 * s) + 1)) < 1e-15
    assert abs(err.max() - ends) < 1e-9 * ends
    assert abs(err[0] - err[-1]) < 1e-12  # g_s(ct) is symmetric under t -> ab/t
    th = np.linspace(0, 2 * np.pi, 20001)
    t = (a + b) / 2 + (b - a) / 2 * np.exp(1j * th)
    bound = 2 / (delta ** (2 * s) - 1)
    e_circ = np.abs(rational.rational_eval(t, w, sg) - 1.0).max()
    assert e_circ <= bound * (1 + 1e-7) and e_circ >= 0.999 * bound


def test_fig1_zolotarev_is_better_on_the_axis_and_worse_off_it(paper):
    """Fig. 1's point (Section 5): with the same s = 10, Zolotarev on [1, 10] beats Neuberger on the
    real interval by orders of magnitude but not on the circle through 1 and 10, where Neuberger's
    error is Theorem 1's bound."""
    s = int(paper["fig1_s"])
    a, b = paper["fig1_zolotarev_a"], paper["fig1_zolotarev_b"]
    wz, sz, ez = rational.zolotarev(s, a, b)
    wn, sn = rational.neuberger_scaled(s, math.sqrt(paper["fig1_neuberger_c_sq"]))
    x = np.linspace(a, b, 100001)
    en_real = np.abs(rational.rational_eval(x, wn, sn) - 1.0).max()
    ez_real = np.abs(np.real(rational.rational_eval(x, wz, sz)) - 1.0).max()
    assert ez_real < 1e-4 * en_real
    th = np.linspace(0, 2 * np.pi, 20001)
    t = (a + b) / 2 + (b - a) / 2 * np.exp(1j * th)
    en_circ = np.abs(rational.rational_eval(t, wn, sn) - 1.0).max()
    ez_circ = np.abs(rational.rational_eval(t, wz, sz) - 1.0).max()
    assert ez_circ > 10 * en_circ


def test_timed_configuration_uses_the_paper_parameters(paper):
    """The timed workload and the 4^4 test problem run at the paper's m_W and mu, to the accuracy
    its timings target."""
    import bench

    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert wl["mus"] == (paper["mu"],)
    assert wl["tol"] == paper["target_accuracy"]
    assert bench.M_W == paper["m_W"]
