"""Pins for the oracle's rational approximations (no GPU).

Neuberger/Kenney-Laub (Eqs. neuberger_mit_c, pfe_s): closed form = partial fractions =
tanh(2s atanh t), g_s(t) = g_s(1/t). Theorem 1 by sampling its circle. The pole count
(Eq. no_of_poles) with c, d by sampling C(m, r). The Fig. 1 parameter set. Jacobi elliptic
functions against scipy. Zolotarev: the n = 1 closed form and equioscillation.
"""
import math

import numpy as np
import pytest
import scipy.special as ss

from oracle import rational


@pytest.mark.parametrize("s", [1, 5, 10, 20])
def test_neuberger_three_forms(s):
    rng = np.random.default_rng(s)
    t = 0.9 * (rng.uniform(-1, 1, 200) + 1j * rng.uniform(-1, 1, 200)) / math.sqrt(2)
    w, sg = rational.neuberger_pfe(s)
    assert np.all(sg < 0)
    a = rational.g_closed(t, s)
    b = rational.rational_eval(t, w, sg)
    c = rational.g_tanh(t, s)
    assert np.abs(a - b).max() < 1e-11
    assert np.abs(a - c).max() < 1e-11
    t2 = 1.5 + rng.uniform(0, 3, 50) + 1j * rng.uniform(-1, 1, 50)
    assert np.abs(rational.g_closed(t2, s) - rational.g_closed(1 / t2, s)).max() < 1e-12


@pytest.mark.parametrize("s,eps", [(10, 1e-6), (5, 1e-3), (20, 1e-10)])
def test_theorem1_circle(s, eps):
    m, r = rational.theorem1_circle(s, eps)
    th = np.linspace(0, 2 * np.pi, 20001)
    t = m + r * np.exp(1j * th)
    err = np.abs(rational.g_closed(t, s) - 1.0)
    assert err.max() <= eps * (1 + 1e-7) + 2e-15  # + rounding of the closed form
    assert err.max() >= 0.99 * eps  # the bound is attained on the circle
    # interior points are better
    assert np.abs(rational.g_closed(m + 0.5 * r, s) - 1.0) < eps


@pytest.mark.parametrize("alpha,beta,eps", [(0.05, 2.5, 1e-8), (0.1, 2.6, 1e-10), (0.2, 3.0, 1e-6)])
def test_pole_count_and_scale(alpha, beta, eps):
    s, c, w, sg = rational.neuberger_for_spectrum(alpha, beta, eps)
    m, r = rational.circle_from_gap(alpha, beta)
    th = np.linspace(0, 2 * np.pi, 4001)
    t = m + r * np.exp(1j * th)
    err = np.abs(rational.rational_eval(t, w, sg) - 1.0)
    assert err.max() <= eps * (1 + 1e-6)
    # one pole fewer misses the target somewhere on the circle
    w2, sg2 = rational.neuberger_scaled(s - 1, c)
    assert np.abs(rational.rational_eval(t, w2, sg2) - 1.0).max() > eps
    # mirror circle
    assert np.abs(rational.rational_eval(-t, w, sg) + 1.0).max() <= eps * (1 + 1e-6)


def test_pole_count_example():
    # gap 0.05, largest modulus 2.5, eps 1e-8: d = sqrt(50)
    _, d = rational.scale_and_d(*rational.circle_from_gap(0.05, 2.5))
    assert abs(d - math.sqrt(50.0)) < 1e-12
    assert 33.0 < rational.pole_count(1e-8, d) < 34.0


def test_fig1_neuberger_parameters():
    """Fig. 1: s = 10, c = 1/sqrt(10) on [1, 10]: worst real-axis error at both ends."""
    s, c = 10, 1 / math.sqrt(10)
    x = np.linspace(1, 10, 100001)
    w, sg = rational.neuberger_scaled(s, c)
    err = np.abs(rational.rational_eval(x, w, sg) - 1.0)
    ref = 1.0 - math.tanh(20 * math.atanh(c))
    assert abs(err.max() - ref) < 1e-15 + 1e-9 * ref
    assert abs(err[0] - err[-1]) < 1e-12  # g_s(ct) symmetric under t -> 10/t


def test_elliptic_against_scipy():
    for m in (0.1, 0.5, 0.9, 0.999, 1 - 1e-6):
        assert abs(rational.ellipk(m) - ss.ellipk(m)) < 1e-12 * ss.ellipk(m)
        for u in (0.1, 0.7, 1.3, 0.9 * ss.ellipk(m)):
            sn, cn, dn = rational.ellipj(u, m)
            ref = ss.ellipj(u, m)
            assert abs(sn - ref[0]) < 1e-12 and abs(cn - ref[1]) < 1e-12 and abs(dn - ref[2]) < 1e-12


def test_zolotarev_n1_closed_form():
    # n = 1: c_1 = k, r(x) = M x/(x^2 + k); extremes 1/(2 sqrt k) at sqrt(k), 1/(1+k) at the ends
    for k in (0.01, 0.1, 0.5):
        c = rational.zolotarev_c(1, k)
        assert abs(c[0] - k) < 1e-13
        w, sg, err = rational.zolotarev(1, k, 1.0)
        fmax, fmin = 1 / (2 * math.sqrt(k)), 1 / (1 + k)
        assert abs(w[0] - 2 / (fmax + fmin)) < 1e-10
        assert abs(sg[0] + k) < 1e-13
        assert abs(err - (fmax - fmin) / (fmax + fmin)) < 1e-10


@pytest.mark.parametrize("n,a,b", [(4, 1.0, 10.0), (10, 1.0, 10.0), (8, 0.05, 2.6)])
def test_zolotarev_equioscillation(n, a, b):
    w, sg, err = rational.zolotarev(n, a, b)
    assert np.all(sg < 0)
    x = np.exp(np.linspace(math.log(a), math.log(b), 400001))
    e = np.real(rational.rational_eval(x, w, sg)) - 1.0
    assert abs(np.abs(e).max() - err) < 1e-3 * err + 1e-15
    # alternation points: runs of samples with |e| > 0.98 err, consecutive runs of opposite sign
    sg_big = np.sign(e[np.abs(e) > 0.98 * err])
    runs = 1 + int(np.count_nonzero(sg_big[1:] != sg_big[:-1]))
    assert runs >= 2 * n + 1
    # odd function
    assert np.abs(rational.rational_eval(-x[:100], w, sg) + rational.rational_eval(x[:100], w, sg)).max() < 1e-12


def test_zolotarev_beats_neuberger_on_real_interval():
    a, b, n = 0.05, 2.6, 20
    wz, sz, ez = rational.zolotarev(n, a, b)
    c, _ = rational.scale_and_d(*rational.circle_from_gap(a, b))
    wn, sn = rational.neuberger_scaled(n, c)
    x = np.exp(np.linspace(math.log(a), math.log(b), 20001))
    en = np.abs(rational.rational_eval(x, wn, sn) - 1).max()
    assert ez < en
    assert ez < 1e-10
