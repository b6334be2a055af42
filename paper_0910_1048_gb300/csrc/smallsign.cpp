// y = sign(H_k) e_1 for the tridiagonal matrix of two-sided Lanczos (host, FP64).
//
// Algorithm 4 ends with x = x_P + beta V_k f(H_k) e_1; Section 2 evaluates f on the small
// projected matrix by an eigendecomposition or Roberts' Newton iteration, an O(k^3) term
// (Proposition 2). Two faster routes are implemented here.
//
// Eigenvector route (O(k^2), accurate to about cond(Z)^2 u):
//  1. Diagonal similarity S = D^-1 H_k D with d_1 = 1, d_{j+1} = d_j delta_j / gamma_j,
//     gamma_j = sqrt(beta_j delta_j), makes S complex symmetric (S^T = S) with diagonal
//     alpha and off-diagonal gamma. sign(H_k) e_1 = D sign(S) e_1.
//  2. Implicit shifted QR on S with complex orthogonal plane rotations G (G^T G = I,
//     c^2 + s^2 = 1) and Wilkinson shifts: S = Z Lambda Z^T, Z = G_1 ... G_N.
//     Only the first row of Z is accumulated; the rotations are stored.
//  3. sign(S) e_1 = Z (sign(Re Lambda) .* Z^T e_1), applying the stored rotations in
//     reverse order (O(N) = O(k^2)).
// Complex orthogonal rotations are not unitary; the result is therefore checked
// (sign(S)^2 e_1 = e_1 and H_k y = sign(H_k) H_k e_1) and, if a check fails, recomputed
// by scaled Newton on the dense k x k matrix (the paper's Roberts iteration, O(k^3)).
//
// Rational route, the default (more accurate; O(k^2) for the Ritz values, O(s k) per evaluation): Roberts'
// unscaled Newton iterate is exactly the Kenney-Laub function g_s of Section 5, whose
// partial fractions (Eq. pfe_s) give
//     sign(H_k) e_1 ~ g_s(c H_k) e_1 = c H_k sum_i omega_i (c^2 H_k^2 - sigma_i)^-1 e_1,
// s solves with the pentadiagonal H_k^2 (banded LU with partial pivoting). c and s are chosen
// from the Ritz values mu (right half plane representatives) so that every Ritz value meets
//     2 |(c mu - 1)/(c mu + 1)|^{2s} <= eps      (the proof of Theorem 1),
// and the result is accepted when the involution residual |g(cH) y - e_1| is small.
#include <algorithm>
#include <complex>
#include <thread>
#include <vector>

#include "common.h"

namespace ovl {

using cz = std::complex<double>;

// Number of small-sign evaluations the calling thread runs side by side (set by a driver that
// evaluates several right-hand sides at once); each gets its share of the host threads.
thread_local int g_sign_concurrency = 1;
void set_sign_concurrency(int n) { g_sign_concurrency = std::max(1, n); }

namespace {

// Principal square root of a + ib (branch cut on the negative real axis, like std::sqrt) from
// the half-angle identities: with r = |z|, t = sqrt((r + |a|) / 2), sqrt(z) = (t, b / 2t) for
// a >= 0 and (|b| / 2t, sign(b) t) for a < 0.
inline cz csqrt_fast(cz z) {
  const double a = z.real(), b = z.imag();
  if (a == 0.0 && b == 0.0) return cz(0.0, 0.0);
  const double r = std::sqrt(a * a + b * b);
  const double t = std::sqrt(0.5 * (r + std::fabs(a)));
  if (a >= 0.0) return cz(t, b / (2.0 * t));
  return cz(std::fabs(b) / (2.0 * t), std::copysign(t, b));
}


struct Rot {
  int p;
  cz c, s;
};

// G w on indices (p, p+1):  (c w_p + s w_q, -s w_p + c w_q)
inline void rot_apply(const Rot& r, cz* w) {
  cz a = w[r.p], b = w[r.p + 1];
  w[r.p] = r.c * a + r.s * b;
  w[r.p + 1] = -r.s * a + r.c * b;
}
// G^T w:  (c w_p - s w_q, s w_p + c w_q)
inline void rot_apply_t(const Rot& r, cz* w) {
  cz a = w[r.p], b = w[r.p + 1];
  w[r.p] = r.c * a - r.s * b;
  w[r.p + 1] = r.s * a + r.c * b;
}

struct CsqlResult {
  std::vector<cz> lam;
  std::vector<Rot> rots;
  bool ok = false;
};

CsqlResult cs_qr(std::vector<cz> d, std::vector<cz> e) {
  CsqlResult res;
  const int k = (int)d.size();
  const double eps = 1e-15;
  long long budget = 60LL * k + 100;
  res.rots.reserve((size_t)k * 8);
  // |e_i| <= eps (|d_i| + |d_i+1|) in squared magnitudes (no square roots in the scan)
  auto negligible = [&](int i) { return std::norm(e[i]) <= eps * eps * (std::norm(d[i]) + std::norm(d[i + 1])); };
  int hi = k - 1;
  while (hi > 0) {
    if (negligible(hi - 1)) {
      e[hi - 1] = 0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && !negligible(lo - 1)) --lo;
    if (lo > 0) e[lo - 1] = 0;
    if (--budget < 0) return res;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
    cz a = d[hi - 1], b = d[hi], ee = e[hi - 1];
    cz half = 0.5 * (a - b);
    cz disc = csqrt_fast(half * half + ee * ee);
    cz m1 = 0.5 * (a + b) + disc, m2 = 0.5 * (a + b) - disc;
    cz shift = std::abs(m1 - b) < std::abs(m2 - b) ? m1 : m2;
    cz x = d[lo] - shift, z = e[lo];
    for (int p = lo; p < hi; ++p) {
      const int q = p + 1;
      cz rho = std::sqrt(x * x + z * z);
      double scale = std::sqrt(std::norm(x) + std::norm(z));
      if (!(std::abs(rho) > 1e-8 * scale) || scale == 0.0) return res;  // (near) isotropic: give up
      cz c = x / rho, s = -z / rho;
      if (std::norm(c) + std::norm(s) > 1e8) return res;  // too far from unitary
      if (p > lo) e[p - 1] = rho;
      cz dp = d[p], dq = d[q], ep = e[p];
      cz c2 = c * c, s2 = s * s, cs = c * s;
      d[p] = dp * c2 - 2.0 * ep * cs + dq * s2;
      d[q] = dp * s2 + 2.0 * ep * cs + dq * c2;
      e[p] = cs * (dp - dq) + ep * (c2 - s2);
      if (q < hi) {
        z = -s * e[q];
        e[q] = c * e[q];
        x = e[p];
      }
      res.rots.push_back(Rot{p, c, s});
    }
  }
  res.lam = d;
  res.ok = true;
  return res;
}

// Dense complex LU inverse with partial pivoting (in place). Returns false if singular.
bool invert(std::vector<cz>& a, int n) {
  std::vector<int> piv(n);
  std::vector<cz> inv((size_t)n * n, cz(0));
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int pr = col;
    double best = std::abs(a[(size_t)col * n + col]);
    for (int r = col + 1; r < n; ++r)
      if (std::abs(a[(size_t)r * n + col]) > best) best = std::abs(a[(size_t)r * n + col]), pr = r;
    if (best == 0.0) return false;
    if (pr != col) {
      for (int c = 0; c < n; ++c) {
        std::swap(a[(size_t)pr * n + c], a[(size_t)col * n + c]);
        std::swap(inv[(size_t)pr * n + c], inv[(size_t)col * n + c]);
      }
    }
    cz pinv = 1.0 / a[(size_t)col * n + col];
    for (int c = 0; c < n; ++c) {
      a[(size_t)col * n + c] *= pinv;
      inv[(size_t)col * n + c] *= pinv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      cz f = a[(size_t)r * n + col];
      if (f == cz(0)) continue;
      cz* ar = &a[(size_t)r * n];
      cz* ac = &a[(size_t)col * n];
      cz* ir = &inv[(size_t)r * n];
      cz* ic = &inv[(size_t)col * n];
      for (int c = 0; c < n; ++c) {
        ar[c] -= f * ac[c];
        ir[c] -= f * ic[c];
      }
    }
  }
  a.swap(inv);
  return true;
}

}  // namespace

// Dense Roberts-Newton with determinantal scaling on the tridiagonal H (O(k^3)).
ovl_status small_sign_newton(int k, const cz* al, const cz* be, const cz* de, cz* y) {
  std::vector<cz> x((size_t)k * k, cz(0));
  for (int i = 0; i < k; ++i) {
    x[(size_t)i * k + i] = al[i];
    if (i + 1 < k) {
      x[(size_t)i * k + i + 1] = be[i];
      x[(size_t)(i + 1) * k + i] = de[i];
    }
  }
  bool scaling = true;
  for (int it = 0; it < 100; ++it) {
    std::vector<cz> xi = x;
    // log |det X| from an LU of a copy (partial pivoting)
    double logdet = 0.0;
    if (scaling) {
      std::vector<cz> lu = x;
      for (int col = 0; col < k; ++col) {
        int pr = col;
        double best = std::abs(lu[(size_t)col * k + col]);
        for (int r = col + 1; r < k; ++r)
          if (std::abs(lu[(size_t)r * k + col]) > best) best = std::abs(lu[(size_t)r * k + col]), pr = r;
        if (best == 0.0) {
          set_error("small_sign: singular projected matrix");
          return OVL_EILLPOSED;
        }
        if (pr != col)
          for (int c = 0; c < k; ++c) std::swap(lu[(size_t)pr * k + c], lu[(size_t)col * k + c]);
        cz piv = lu[(size_t)col * k + col];
        logdet += std::log(std::abs(piv));
        for (int r = col + 1; r < k; ++r) {
          cz f = lu[(size_t)r * k + col] / piv;
          if (f == cz(0)) continue;
          for (int c = col; c < k; ++c) lu[(size_t)r * k + c] -= f * lu[(size_t)col * k + c];
        }
      }
    }
    if (!invert(xi, k)) {
      set_error("small_sign: singular Newton iterate");
      return OVL_EILLPOSED;
    }
    double zeta = scaling ? std::exp(-logdet / k) : 1.0;
    double num = 0, den = 0;
    for (size_t i = 0; i < x.size(); ++i) {
      cz nx = 0.5 * (zeta * x[i] + xi[i] / zeta);
      num += std::norm(nx - x[i]);
      den += std::norm(nx);
      x[i] = nx;
    }
    double change = std::sqrt(num / den);
    if (change < 1e-2) scaling = false;
    if (change < 1e-14) break;
  }
  for (int i = 0; i < k; ++i) y[i] = x[(size_t)i * k];
  return OVL_OK;
}

ovl_status small_sign_ql(int k, const cz* al, const cz* be, const cz* de, cz* y, double* check) {
  // 1. symmetrising diagonal similarity
  std::vector<cz> dg(k), gm(k > 1 ? k - 1 : 0), dscale(k);
  dscale[0] = 1.0;
  for (int i = 0; i < k; ++i) dg[i] = al[i];
  for (int i = 0; i + 1 < k; ++i) {
    cz g = std::sqrt(be[i] * de[i]);
    if (g == cz(0)) {
      set_error("small_sign: zero off-diagonal");
      return OVL_EINVAL;
    }
    gm[i] = g;
    dscale[i + 1] = dscale[i] * de[i] / g;
  }
  // 2. implicit QR with complex orthogonal rotations
  CsqlResult r = cs_qr(dg, gm);
  if (!r.ok) return OVL_ENOCONV;
  double lmax = 0;
  for (auto& l : r.lam) lmax = std::max(lmax, std::abs(l));
  for (auto& l : r.lam)
    if (std::abs(l.real()) <= 1e-14 * lmax) {
      set_error("small_sign: Ritz value on the imaginary axis");
      return OVL_EILLPOSED;
    }
  // first row of Z = Z^T e_1
  std::vector<cz> u(k, cz(0));
  u[0] = 1.0;
  for (const Rot& g : r.rots) rot_apply_t(g, u.data());
  auto apply_sign_s = [&](std::vector<cz>& w) {  // w <- Z sign(L) Z^T w
    for (const Rot& g : r.rots) rot_apply_t(g, w.data());
    for (int i = 0; i < k; ++i) w[i] *= (r.lam[i].real() >= 0 ? 1.0 : -1.0);
    for (auto it = r.rots.rbegin(); it != r.rots.rend(); ++it) rot_apply(*it, w.data());
  };
  std::vector<cz> ys(k);
  for (int i = 0; i < k; ++i) ys[i] = (r.lam[i].real() >= 0 ? 1.0 : -1.0) * u[i];
  for (auto it = r.rots.rbegin(); it != r.rots.rend(); ++it) rot_apply(*it, ys.data());
  // 3. checks: sign(S)^2 e1 = e1 and H y = sign(H) (H e1)
  std::vector<cz> w2 = ys;
  apply_sign_s(w2);
  double err1 = std::abs(w2[0] - 1.0);
  for (int i = 1; i < k; ++i) err1 = std::max(err1, std::abs(w2[i]));
  for (int i = 0; i < k; ++i) y[i] = dscale[i] * ys[i];
  std::vector<cz> he1(k, cz(0));  // D^-1 H e1 = (alpha_1, delta_1 / d_2, 0...)
  he1[0] = al[0];
  if (k > 1) he1[1] = de[0] / dscale[1];
  apply_sign_s(he1);
  double err2 = 0, nrm = 0;
  for (int i = 0; i < k; ++i) {
    cz hy = al[i] * y[i];
    if (i > 0) hy += de[i - 1] * y[i - 1];
    if (i + 1 < k) hy += be[i] * y[i + 1];
    cz rhs = dscale[i] * he1[i];
    err2 = std::max(err2, std::abs(hy - rhs));
    nrm = std::max(nrm, std::abs(hy));
  }
  double err = std::max(err1, err2 / std::max(nrm, 1e-300));
  if (check) *check = err;
  if (!(err < 1e-9)) return OVL_ENOCONV;
  return OVL_OK;
}

namespace {

// Eigenvalues only of the complex symmetric tridiagonal with diagonal d and squared off-diagonal
// e2 (the eigenvalues depend on the squares alone). Implicitly shifted QR sweeps from the top of the
// unreduced block to its bottom, deflating there, in the root-free form of Pal, Walker and Kahan
// (Parlett, The Symmetric Eigenvalue Problem, Section 8.15): the sweep carries gamma = c (d - shift)
// - s gamma' and p = gamma^2 / c with c, s the squares of the rotation's cosine and sine, so a
// rotation takes one reciprocal and no square root. The algebra holds for complex symmetric
// matrices with complex orthogonal rotations (c + s = 1); a rotation whose r = p + e^2 cancels
// (an isotropic column, where the complex symmetric QR breaks down) gives up.
bool cs_eigs(std::vector<cz> d, std::vector<cz> e2, std::vector<cz>& lam) {
  const int k = (int)d.size();
  const double eps2 = 1e-30;  // (1e-15)^2
  long long budget = 60LL * k + 100;
  // |e_i| <= eps (|d_i| + |d_i+1|), tested as |e_i^2|^2 <= eps^4 (|d_i|^2 + |d_i+1|^2)^2
  auto negligible = [&](int i) {
    const double t = std::norm(d[i]) + std::norm(d[i + 1]);
    return std::norm(e2[i]) <= eps2 * eps2 * t * t;
  };
  int hi = k - 1;
  while (hi > 0) {
    if (negligible(hi - 1)) {
      e2[hi - 1] = 0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && !negligible(lo - 1)) --lo;
    if (lo > 0) e2[lo - 1] = 0;
    if (--budget < 0) return false;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
    const cz a = d[hi - 1], b = d[hi];
    const cz half = 0.5 * (a - b);
    const cz disc = csqrt_fast(half * half + e2[hi - 1]);
    const cz m1 = 0.5 * (a + b) + disc, m2 = 0.5 * (a + b) - disc;
    const cz shift = std::norm(m1 - b) < std::norm(m2 - b) ? m1 : m2;
    cz c = 1.0, s = 0.0;
    cz gam = d[lo] - shift;
    cz p = gam * gam;
    for (int i = lo; i < hi; ++i) {
      const cz bb = e2[i];
      const cz r = p + bb;
      const double nr = std::norm(r);
      if (!(nr > 1e-32 * (std::norm(p) + std::norm(bb)))) return false;  // cancellation, or not finite
      const cz inv_r = std::conj(r) * (1.0 / nr);
      if (i > lo) e2[i - 1] = s * r;
      const cz oldc = c, oldgam = gam;
      c = p * inv_r;
      s = bb * inv_r;
      const cz alpha = d[i + 1];
      gam = c * (alpha - shift) - s * oldgam;
      d[i] = oldgam + (alpha - gam);
      const double nc = std::norm(c);
      p = nc > 0.0 ? gam * gam * std::conj(c) * (1.0 / nc) : oldc * bb;
    }
    e2[hi - 1] = s * p;
    d[hi] = shift + gam;
  }
  lam = d;
  return true;
}

// Ritz values of H_k: its complex symmetric similar S has the squared off-diagonal beta_j delta_j.
bool ritz_values(int k, const cz* al, const cz* be, const cz* de, std::vector<cz>& lam) {
  std::vector<cz> dg(al, al + k), g2(k - 1);
  for (int i = 0; i + 1 < k; ++i) {
    g2[i] = be[i] * de[i];
    if (g2[i] == cz(0)) return false;
  }
  return cs_eigs(dg, g2, lam);
}

// (c, s): fewest poles with 2 |(c mu - 1)/(c mu + 1)|^{2s} <= eps over the Ritz values.
bool choose_scale(const std::vector<cz>& lam, double eps, int s_max, double* c_out, int* s_out) {
  std::vector<cz> mu;
  double amin = 1e300, amax = 0;
  for (cz l : lam) {
    cz m = l.real() >= 0 ? l : -l;
    if (!(m.real() > 0)) return false;
    mu.push_back(m);
    amin = std::min(amin, std::abs(m));
    amax = std::max(amax, std::abs(m));
  }
  // q(c) = max over mu of |c mu - 1| / |c mu + 1|, compared in squares (q2 = q^2)
  double best_q2 = 1.0, best_c = 1.0;
  const int ng = 160;
  for (int t = 0; t <= ng; ++t) {
    double c = std::exp(std::log(1.0 / amax) + (std::log(1.0 / amin) - std::log(1.0 / amax)) * t / ng);
    double q2 = 0;
    for (cz m : mu) {
      const double xr = c * m.real(), xi = c * m.imag();
      const double num = (xr - 1.0) * (xr - 1.0) + xi * xi, den = (xr + 1.0) * (xr + 1.0) + xi * xi;
      q2 = std::max(q2, num / den);
    }
    if (q2 < best_q2) best_q2 = q2, best_c = c;
  }
  if (!(best_q2 < 1.0)) return false;
  double sr = std::log(eps / 2.0) / std::log(best_q2);  // 2 q^{2s} <= eps
  int s = std::max(1, (int)std::ceil(sr));
  if (s > s_max) return false;
  *c_out = best_c;
  *s_out = s;
  return true;
}

// |re| + |im|: the pivoting magnitude of the tridiagonal solves (no square root).
inline double abs1(cz z) { return std::fabs(z.real()) + std::fabs(z.imag()); }
inline cz cinv(cz z) { return std::conj(z) * (1.0 / std::norm(z)); }

// Solve (c H + z) x = b in place (b -> x) for tridiagonal H (diag al, super be, sub de) by
// Gaussian elimination with partial pivoting (one row interchange at most per step; the
// interchange fills a second superdiagonal). d, du, dl, du2 are scratch of length k.
// Returns false if a pivot is zero.
inline bool tri_solve(int k, const cz* al, const cz* be, const cz* de, double c, cz z, cz* b, cz* d, cz* du, cz* dl,
                      cz* du2) {
  for (int i = 0; i < k; ++i) {
    d[i] = c * al[i] + z;
    if (i + 1 < k) {
      du[i] = c * be[i];
      dl[i] = c * de[i];
    }
    du2[i] = 0.0;
  }
  for (int i = 0; i + 1 < k; ++i) {
    if (abs1(d[i]) >= abs1(dl[i])) {
      if (d[i] == cz(0.0)) return false;
      const cz f = dl[i] * cinv(d[i]);
      d[i + 1] -= f * du[i];
      b[i + 1] -= f * b[i];
    } else {  // interchange rows i and i+1
      const cz f = d[i] * cinv(dl[i]);
      d[i] = dl[i];
      const cz t = d[i + 1];
      d[i + 1] = du[i] - f * t;
      if (i + 2 < k) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du2[i];
      }
      du[i] = t;
      const cz bi = b[i];
      b[i] = b[i + 1];
      b[i + 1] = bi - f * b[i + 1];
    }
  }
  if (d[k - 1] == cz(0.0)) return false;
  b[k - 1] *= cinv(d[k - 1]);
  if (k > 1) b[k - 2] = (b[k - 2] - du[k - 2] * b[k - 1]) * cinv(d[k - 2]);
  for (int i = k - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) * cinv(d[i]);
  return true;
}

// out = g_s(c H) v = c H sum_i omega_i (c^2 H^2 - sigma_i)^-1 v (Eq. pfe_s). With sigma_i =
// -t_i^2 (t_i = tan theta_i > 0) each shifted matrix factors into tridiagonal ones,
// c^2 H^2 + t_i^2 = (c H - i t_i)(c H + i t_i), so each pole costs two tridiagonal solves
// (no cancellation: the factors are applied one after the other). Returns false if a solve
// meets a zero pivot.
bool rational_apply(int k, const cz* al, const cz* be, const cz* de, double c, int s, const cz* v, cz* out) {
  // the s shifted solves are independent: split them over host threads, each summing its
  // own shifts in order, then add the per-thread sums in thread order (deterministic)
  const int hw = std::max(1, (int)std::thread::hardware_concurrency() / std::max(1, g_sign_concurrency));
  const int nth = std::max(1, std::min({hw, 16, s, (int)((size_t)s * k / 40000 + 1)}));
  std::vector<std::vector<cz>> part(nth, std::vector<cz>(k, 0.0));
  std::vector<char> ok(nth, 1);
  auto work = [&](int tid) {
    std::vector<cz>& acc = part[tid];
    std::vector<cz> x(k), d(k), du(k), dl(k), du2(k);
    for (int sh = 1 + tid; sh <= s; sh += nth) {
      const double th = 3.14159265358979323846 / (2.0 * s) * (sh - 0.5);
      const double om = 1.0 / (s * std::cos(th) * std::cos(th));
      const double t = std::tan(th);  // sigma = -t^2
      std::copy(v, v + k, x.begin());
      if (!tri_solve(k, al, be, de, c, cz(0.0, -t), x.data(), d.data(), du.data(), dl.data(), du2.data()) ||
          !tri_solve(k, al, be, de, c, cz(0.0, t), x.data(), d.data(), du.data(), dl.data(), du2.data())) {
        ok[tid] = 0;
        return;
      }
      for (int i = 0; i < k; ++i) acc[i] += om * x[i];
    }
  };
  if (nth == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 1; t < nth; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& t : th) t.join();
  }
  for (int t = 0; t < nth; ++t)
    if (!ok[t]) return false;
  std::vector<cz> acc(k, 0.0);
  for (int t = 0; t < nth; ++t)
    for (int i = 0; i < k; ++i) acc[i] += part[t][i];
  for (int i = 0; i < k; ++i) {
    cz t = al[i] * acc[i];
    if (i > 0) t += de[i - 1] * acc[i - 1];
    if (i + 1 < k) t += be[i] * acc[i + 1];
    out[i] = c * t;
  }
  return true;
}

}  // namespace

// Rational route with a (c, s) hint; hint->s == 0 means "compute from the Ritz values".
// Returns OVL_OK when the involution residual is below tol_inv.
ovl_status small_sign_rational(int k, const cz* al, const cz* be, const cz* de, cz* y, double* hint_c, int* hint_s,
                               double* inv_res, int* ritz_count) {
  const double eps = 1e-15, tol_inv = 1e-11;
  const int s_max = 4000;
  // attempts: the cached (c, s); the same c with 50% more poles (new Ritz values closer to
  // the imaginary axis usually need only a few more); (c, s) from freshly computed Ritz values
  const bool had_hint = *hint_s > 0;
  for (int attempt = had_hint ? 0 : 2; attempt < 3; ++attempt) {
    if (attempt == 1) *hint_s = std::min(s_max, (*hint_s * 3 + 1) / 2);
    if (attempt == 2) {
      if (ritz_count) ++*ritz_count;
      std::vector<cz> lam;
      if (!ritz_values(k, al, be, de, lam)) return OVL_ENOCONV;
      double lmax = 0;
      for (cz l : lam) lmax = std::max(lmax, std::abs(l));
      for (cz l : lam)
        if (std::abs(l.real()) <= 1e-14 * lmax) {
          set_error("small_sign: Ritz value on the imaginary axis");
          return OVL_EILLPOSED;
        }
      if (!choose_scale(lam, eps, s_max, hint_c, hint_s)) return OVL_ENOCONV;
    }
    std::vector<cz> e1(k, 0.0), chk(k);
    e1[0] = 1.0;
    if (!rational_apply(k, al, be, de, *hint_c, *hint_s, e1.data(), y) ||
        !rational_apply(k, al, be, de, *hint_c, *hint_s, y, chk.data()))
      continue;  // a singular shifted factor: try the next (c, s)
    double r = std::abs(chk[0] - 1.0);
    for (int i = 1; i < k; ++i) r = std::max(r, std::abs(chk[i]));
    if (inv_res) *inv_res = r;
    if (r <= tol_inv) return OVL_OK;
  }
  return OVL_ENOCONV;
}

// method 0 auto (rational, then QL eigenvectors, then Newton up to k = kNewtonMaxK: its O(k^3)
// steps would dominate a solve beyond), 1 QL only, 2 Newton only, 3 rational only.
// hint_c/hint_s (may be null) carry (c, s) between calls on growing H_k.
constexpr int kNewtonMaxK = 200;
ovl_status small_sign(int k, const cz* al, const cz* be, const cz* de, cz* y, int method, double* hint_c = nullptr,
                      int* hint_s = nullptr, int* ritz_count = nullptr) {
  if (k < 1) {
    set_error("small_sign: k < 1");
    return OVL_EINVAL;
  }
  if (k == 1) {
    if (al[0].real() == 0.0) {
      set_error("small_sign: eigenvalue on the imaginary axis");
      return OVL_EILLPOSED;
    }
    y[0] = al[0].real() > 0 ? 1.0 : -1.0;
    return OVL_OK;
  }
  if (method == 0 || method == 3) {
    double c = hint_c ? *hint_c : 0.0;
    int sp = hint_s ? *hint_s : 0;
    ovl_status s = small_sign_rational(k, al, be, de, y, &c, &sp, nullptr, ritz_count);
    if (hint_c && s == OVL_OK) *hint_c = c;
    if (hint_s) *hint_s = s == OVL_OK ? sp : 0;
    if (s == OVL_OK || method == 3 || s == OVL_EILLPOSED) return s;
  }
  if (method != 2) {
    double chk = 0;
    ovl_status s = small_sign_ql(k, al, be, de, y, &chk);
    if (s == OVL_OK || method == 1 || s == OVL_EILLPOSED) return s;
  }
  if (method == 0 && k > kNewtonMaxK) {
    set_error("small_sign: no route reached the accuracy check at k = %d (H_k too close to singular "
              "or to the imaginary axis)", k);
    return OVL_ENOCONV;
  }
  return small_sign_newton(k, al, be, de, y);
}

}  // namespace ovl

extern "C" ovl_status ovl_small_sign(int32_t k, const void* alpha, const void* beta, const void* delta, void* y,
                                     int32_t method) {
  ovl::clear_error();
  if (k < 1 || !alpha || !y || (k > 1 && (!beta || !delta)) || method < 0 || method > 3) {
    ovl::set_error("ovl_small_sign: invalid arguments");
    return OVL_EINVAL;
  }
  return ovl::small_sign(k, (const ovl::cz*)alpha, (const ovl::cz*)beta, (const ovl::cz*)delta, (ovl::cz*)y, method);
}
