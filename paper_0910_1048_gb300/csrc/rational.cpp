// Rational approximations g(t) = t sum_i omega_i / (t^2 - sigma_i) of sign(t) (host, FP64).
//
// Neuberger / Kenney-Laub, Section 5, Eq. pfe_s:
//   omega_i = (1/s) cos^-2(pi (i - 1/2) / (2s)),  sigma_i = -tan^2(pi (i - 1/2) / (2s)),
//   used as sign(t) ~ g_s(c t), i.e. omega_i / c and sigma_i / c^2.
// Scale and pole count for a spectrum in C(m, r) u C(-m, r), text after Theorem 1 and
// Eq. no_of_poles:  c = ((m+r)(m-r))^{-1/2},  d = ((m+r)/(m-r))^{1/2},
//   s >= log(eps/(eps+2)) / (2 log((d-1)/(d+1))),
// with the circle from the deflation gap alpha and largest modulus beta (Section 6):
//   m = (alpha+beta)/2, r = (beta-alpha)/2.
// Zolotarev (cited in Section 5, coefficients not printed): on [k, 1], k = lo/hi,
//   r(x) = M x prod_{j<n} (x^2 + c_{2j}) / prod_{j<=n} (x^2 + c_{2j-1}),
//   c_l = k^2 sn^2(l K'/(2n); k') / cn^2(l K'/(2n); k'),  k' = sqrt(1 - k^2), K' = K(k'),
// M from the extreme values on [k, 1] (equioscillation), then rescaled to [lo, hi].
// Jacobi elliptic functions by the AGM / descending Landen method (Abramowitz & Stegun 16.4).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace ovl {

namespace {

const double kPi = 3.14159265358979323846;

struct Agm {
  std::vector<double> a, c;
};

Agm agm(double m) {
  Agm t;
  double a = 1.0, b = std::sqrt(1.0 - m), c = std::sqrt(m);
  t.a.push_back(a);
  t.c.push_back(c);
  while (std::fabs(c) > 1e-16 * std::fabs(a) && t.a.size() < 64) {
    double an = 0.5 * (a + b), bn = std::sqrt(a * b), cn = 0.5 * (a - b);
    a = an;
    b = bn;
    c = cn;
    t.a.push_back(a);
    t.c.push_back(c);
  }
  return t;
}

double ellip_k(double m) {
  Agm t = agm(m);
  return kPi / (2.0 * t.a.back());
}

void ellip_sn_cn(double u, double m, double* sn, double* cn) {
  Agm t = agm(m);
  int nst = (int)t.a.size() - 1;
  double phi = std::ldexp(t.a.back() * u, nst);
  for (int i = nst; i >= 1; --i) phi = 0.5 * (phi + std::asin(t.c[i] / t.a[i] * std::sin(phi)));
  *sn = std::sin(phi);
  *cn = std::cos(phi);
}

double zolo_unnorm(double x, const std::vector<double>& c, int n) {
  double num = 1.0, den = 1.0;
  for (int j = 1; j < n; ++j) num *= x * x + c[2 * j - 1];
  for (int j = 1; j <= n; ++j) den *= x * x + c[2 * j - 2];
  return x * num / den;
}

double golden_extreme(const std::vector<double>& c, int n, double lo, double hi, double sign) {
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  for (int it = 0; it < 100; ++it) {
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    if (sign * zolo_unnorm(x1, c, n) > sign * zolo_unnorm(x2, c, n))
      hi = x2;
    else
      lo = x1;
  }
  return zolo_unnorm(0.5 * (lo + hi), c, n);
}

}  // namespace

void neuberger(int s, double c, double* omega, double* sigma) {
  for (int i = 1; i <= s; ++i) {
    double th = kPi / (2.0 * s) * (i - 0.5);
    double co = std::cos(th), ta = std::tan(th);
    omega[i - 1] = 1.0 / (s * co * co) / c;
    sigma[i - 1] = -(ta * ta) / (c * c);
  }
}

// eps-circle bound of Theorem 1 for s poles and d: |g_s(ct) - 1| <= 2/(((d+1)/(d-1))^{2s} - 1)
double neuberger_bound(int s, double d) {
  double q = std::pow((d + 1.0) / (d - 1.0), 2.0 * s);
  return 2.0 / (q - 1.0);
}

void neuberger_for_spectrum(double lo, double hi, double eps, int* s_out, double* c_out, double* d_out) {
  double m = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
  double c = 1.0 / std::sqrt((m + r) * (m - r));
  double d = std::sqrt((m + r) / (m - r));
  double sreal = std::log(eps / (eps + 2.0)) / (2.0 * std::log((d - 1.0) / (d + 1.0)));
  int s = (int)std::ceil(sreal - 1e-12);
  *s_out = std::max(s, 1);
  *c_out = c;
  *d_out = d;
}

double zolotarev(int n, double lo, double hi, double* omega, double* sigma) {
  double k = lo / hi;
  double mp = 1.0 - k * k;
  double kp = ellip_k(mp);
  std::vector<double> c(2 * n - 1);
  for (int l = 1; l < 2 * n; ++l) {
    double sn, cn;
    ellip_sn_cn(l * kp / (2.0 * n), mp, &sn, &cn);
    c[l - 1] = k * k * sn * sn / (cn * cn);
  }
  // extreme values of the unnormalised function on [k, 1] (log grid + golden refinement)
  const int ns = 100001;
  double lk = std::log(k);
  double fmax = -1e300, fmin = 1e300;
  int imax = 0, imin = 0;
  std::vector<double> xs(ns);
  for (int i = 0; i < ns; ++i) {
    xs[i] = std::exp(lk * (1.0 - (double)i / (ns - 1)));
    double f = zolo_unnorm(xs[i], c, n);
    if (f > fmax) fmax = f, imax = i;
    if (f < fmin) fmin = f, imin = i;
  }
  auto lohi = [&](int i, double* a, double* b) {
    *a = xs[std::max(i - 1, 0)];
    *b = xs[std::min(i + 1, ns - 1)];
    if (*a > *b) std::swap(*a, *b);
  };
  double a, b;
  lohi(imax, &a, &b);
  fmax = std::max(fmax, golden_extreme(c, n, a, b, 1.0));
  lohi(imin, &a, &b);
  fmin = std::min(fmin, golden_extreme(c, n, a, b, -1.0));
  double mnorm = 2.0 / (fmax + fmin);
  double err = (fmax - fmin) / (fmax + fmin);
  for (int j = 0; j < n; ++j) {
    double pj = c[2 * j];
    double num = 1.0, den = 1.0;
    for (int l = 1; l < n; ++l) num *= c[2 * l - 1] - pj;
    for (int l = 0; l < n; ++l)
      if (l != j) den *= c[2 * l] - pj;
    omega[j] = mnorm * num / den * hi;
    sigma[j] = -pj * hi * hi;
  }
  return err;
}

}  // namespace ovl

extern "C" ovl_status ovl_rational_coeffs(int32_t kind, int32_t s, double lo, double hi, double eps, int32_t s_cap,
                                          double* omega, double* sigma, int32_t* s_out, double* err_out) {
  ovl::clear_error();
  if (!(lo > 0) || !(hi > lo) || !omega || !sigma || s_cap < 1) {
    ovl::set_error("ovl_rational_coeffs: need 0 < lo < hi and output arrays");
    return OVL_EINVAL;
  }
  if (kind == OVL_RAT_NEUBERGER) {
    int sn;
    double c, d;
    if (!(eps > 0) && s <= 0) {
      ovl::set_error("ovl_rational_coeffs: Neuberger needs eps > 0 or s > 0");
      return OVL_EINVAL;
    }
    ovl::neuberger_for_spectrum(lo, hi, eps > 0 ? eps : 1e-8, &sn, &c, &d);
    if (s > 0) sn = s;
    if (sn > s_cap) {
      ovl::set_error("ovl_rational_coeffs: %d poles needed, capacity %d", sn, s_cap);
      return OVL_EINVAL;
    }
    ovl::neuberger(sn, c, omega, sigma);
    if (s_out) *s_out = sn;
    if (err_out) *err_out = ovl::neuberger_bound(sn, d);
    return OVL_OK;
  }
  if (kind == OVL_RAT_ZOLOTAREV) {
    if (s < 1 || s > s_cap) {
      ovl::set_error("ovl_rational_coeffs: Zolotarev needs 1 <= s <= s_cap");
      return OVL_EINVAL;
    }
    double err = ovl::zolotarev(s, lo, hi, omega, sigma);
    if (s_out) *s_out = s;
    if (err_out) *err_out = err;
    return OVL_OK;
  }
  ovl::set_error("ovl_rational_coeffs: unknown kind %d", kind);
  return OVL_EINVAL;
}
