"""Rational approximations to sign(t) (test infrastructure, oracle only).

Neuberger / Kenney-Laub (Section 5, Eqs. neuberger_mit_c and pfe_s):
  g_s(t) = ((t+1)^{2s} - (t-1)^{2s}) / ((t+1)^{2s} + (t-1)^{2s}) = tanh(2 s atanh t)  (|t| < 1)
         = t sum_{i=1}^{s} w_i / (t^2 - sigma_i),
  w_i = (1/s) cos^-2(pi (i - 1/2) / (2s)),  sigma_i = -tan^2(pi (i - 1/2) / (2s)),
  sign(t) ~ g_s(c t).
Theorem 1: |g_s(t) - sign(t)| <= eps on the circle C_{s,eps} (and its mirror) with
  delta = (2/eps + 1)^{1/(2s)}, radius R = 2 delta/(delta^2 - 1), centre M = (delta^2+1)/(delta^2-1).
Scale and pole count for a spectrum inside C(m, r) u C(-m, r) (text after Theorem 1,
Eq. no_of_poles): c = ((m+r)(m-r))^{-1/2}, d = ((m+r)/(m-r))^{1/2},
  s >= log(eps/(eps+2)) / (2 log((d-1)/(d+1))).
Circle heuristic (Section 6): m = (alpha+beta)/2, r = (beta-alpha)/2 from the deflation
gap alpha and the largest |lambda| beta.

Zolotarev (Section 5 cites the best approximation on [-b,-a] u [a,b] without printing
coefficients). Reading: the classical Zolotarev solution of type (2n-1, 2n) on
[k, 1], k = a/b, k' = sqrt(1 - k^2), K' = K(k'):
  r(x) = M x prod_{j=1}^{n-1} (x^2 + c_{2j}) / prod_{j=1}^{n} (x^2 + c_{2j-1}),
  c_l = k^2 sn^2(l K'/(2n); k') / cn^2(l K'/(2n); k'),
with M chosen so that the relative error equioscillates, rescaled to [a, b]. The Jacobi
elliptic functions use the arithmetic-geometric-mean method of Abramowitz & Stegun 16.4.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- Neuberger / Kenney-Laub
def neuberger_pfe(s: int):
    """(omega[s], sigma[s]) of Eq. pfe_s, unscaled (c = 1)."""
    i = np.arange(1, s + 1, dtype=np.float64)
    th = np.pi / (2 * s) * (i - 0.5)
    return 1.0 / (s * np.cos(th) ** 2), -np.tan(th) ** 2


def neuberger_scaled(s: int, c: float):
    """Coefficients of g_s(c t) = t sum omega'_i/(t^2 - sigma'_i): omega/c, sigma/c^2."""
    w, sg = neuberger_pfe(s)
    return w / c, sg / (c * c)


def g_closed(t, s: int):
    """g_s(t) from the (t+1)^{2s} closed form (Eq. neuberger_mit_c)."""
    t = np.asarray(t, dtype=np.complex128)
    p = (t + 1) ** (2 * s)
    q = (t - 1) ** (2 * s)
    return (p - q) / (p + q)


def g_tanh(t, s: int):
    """g_s(t) = tanh(2 s atanh t), valid for |t| < 1."""
    return np.tanh(2 * s * np.arctanh(np.asarray(t, dtype=np.complex128)))


def rational_eval(t, omega, sigma):
    """t sum_i omega_i / (t^2 - sigma_i)."""
    t = np.asarray(t, dtype=np.complex128)
    tt = t[..., None] ** 2
    return t * np.sum(np.asarray(omega) / (tt - np.asarray(sigma)), axis=-1)


def theorem1_circle(s: int, eps: float):
    """(centre M, radius R) of C_{s,eps} in Theorem 1."""
    delta = (2.0 / eps + 1.0) ** (1.0 / (2 * s))
    return (delta * delta + 1) / (delta * delta - 1), 2 * delta / (delta * delta - 1)


def scale_and_d(m: float, r: float):
    """c and d for a spectrum in C(m, r) u C(-m, r)."""
    return ((m + r) * (m - r)) ** -0.5, ((m + r) / (m - r)) ** 0.5


def pole_count(eps: float, d: float) -> float:
    """Right-hand side of Eq. no_of_poles (real; round up for s)."""
    return math.log(eps / (eps + 2)) / (2 * math.log((d - 1) / (d + 1)))


def circle_from_gap(alpha: float, beta: float):
    """Section 6 heuristic: m = (alpha+beta)/2, r = (beta-alpha)/2."""
    return 0.5 * (alpha + beta), 0.5 * (beta - alpha)


def neuberger_for_spectrum(alpha: float, beta: float, eps: float):
    """(s, c, omega', sigma') from the gap alpha, largest modulus beta and target eps."""
    m, r = circle_from_gap(alpha, beta)
    c, d = scale_and_d(m, r)
    s = int(math.ceil(pole_count(eps, d) - 1e-12))
    w, sg = neuberger_scaled(s, c)
    return s, c, w, sg


# ---------------------------------------------------------------- Jacobi elliptic (A&S 16.4)
def _agm_tables(m: float, tol: float = 1e-16):
    a, b, c = 1.0, math.sqrt(1.0 - m), math.sqrt(m)
    aa, cc = [a], [c]
    while abs(c) > tol * abs(a) and len(aa) < 64:
        a, b, c = 0.5 * (a + b), math.sqrt(a * b), 0.5 * (a - b)
        aa.append(a)
        cc.append(c)
    return aa, cc


def ellipk(m: float) -> float:
    """Complete elliptic integral K(m) = pi / (2 AGM(1, sqrt(1-m))), parameter m = k^2."""
    aa, _ = _agm_tables(m)
    return math.pi / (2.0 * aa[-1])


def ellipj(u: float, m: float):
    """(sn, cn, dn)(u | m) by the descending AGM recursion of A&S 16.4.3."""
    aa, cc = _agm_tables(m)
    nsteps = len(aa) - 1
    phi = (2.0 ** nsteps) * aa[-1] * u
    phis = [phi]
    for i in range(nsteps, 0, -1):
        phi = 0.5 * (phi + math.asin(cc[i] / aa[i] * math.sin(phi)))
        phis.append(phi)
    p0 = phis[-1]
    p1 = phis[-2] if len(phis) > 1 else p0
    sn, cn = math.sin(p0), math.cos(p0)
    dn = cn / math.cos(p1 - p0) if len(phis) > 1 else 1.0
    return sn, cn, dn


# ---------------------------------------------------------------- Zolotarev
def zolotarev_c(n: int, k: float):
    """c_l, l = 1..2n-1, for the interval [k, 1]."""
    mp = 1.0 - k * k
    kp = ellipk(mp)
    c = []
    for l in range(1, 2 * n):
        sn, cn, _ = ellipj(l * kp / (2 * n), mp)
        c.append(k * k * sn * sn / (cn * cn))
    return np.array(c)


def _zolo_unnormalised(x, c, n):
    x = np.asarray(x, dtype=np.float64)
    num = np.ones_like(x)
    den = np.ones_like(x)
    for j in range(1, n):
        num = num * (x * x + c[2 * j - 1])
    for j in range(1, n + 1):
        den = den * (x * x + c[2 * j - 2])
    return x * num / den


def zolotarev(n: int, a: float, b: float, samples: int = 200001):
    """Zolotarev best approximation on [-b,-a] u [a,b] as (omega[n], sigma[n], max_err).

    M is set from the extreme values of the unnormalised function on a dense log grid
    of [k, 1] (each extremum refined by golden-section search).
    """
    k = a / b
    c = zolotarev_c(n, k)
    xs = np.exp(np.linspace(math.log(k), 0.0, samples))
    f = _zolo_unnormalised(xs, c, n)

    def refine(i, sign):
        lo = xs[max(i - 1, 0)]
        hi = xs[min(i + 1, len(xs) - 1)]
        g = (math.sqrt(5) - 1) / 2
        for _ in range(80):
            x1 = hi - g * (hi - lo)
            x2 = lo + g * (hi - lo)
            f1 = sign * _zolo_unnormalised(x1, c, n)
            f2 = sign * _zolo_unnormalised(x2, c, n)
            if f1 > f2:
                hi = x2
            else:
                lo = x1
        return float(_zolo_unnormalised(0.5 * (lo + hi), c, n))

    fmax = max(refine(int(np.argmax(f)), 1.0), float(f.max()))
    fmin = min(refine(int(np.argmin(f)), -1.0), float(f.min()))
    mnorm = 2.0 / (fmax + fmin)
    err = (fmax - fmin) / (fmax + fmin)
    # partial fractions of r(x) = x sum_j A_j / (x^2 + c_{2j-1})
    poles = np.array([c[2 * j - 2] for j in range(1, n + 1)])
    zeros = np.array([c[2 * j - 1] for j in range(1, n)])
    amp = np.empty(n)
    for j in range(n):
        num = np.prod(zeros - poles[j]) if n > 1 else 1.0
        den = np.prod(np.delete(poles, j) - poles[j]) if n > 1 else 1.0
        amp[j] = mnorm * num / den
    return amp * b, -poles * b * b, err
