/*
 * Plain FP64 CPU two-sided Lanczos for x = sign(H_W(mu)) b (Algorithm 4) — TEST INFRASTRUCTURE
 * ONLY (oracle). Only the tests, smoke() and bench.py's cpu_baseline / reference legs load it;
 * the CUDA library neither links nor calls it, and the two share no code.
 *
 * Written from the paper: H_W = gamma5 D_W(mu) (Section 1), with D_W in the reading used by the
 * whole oracle (the paper defers it to its reference [Bloch:2006cd]):
 *   (D_W psi)(x) = psi(x) - kappa sum_nu [ e^{+mu d_nu,4} (1 - g_nu) U_nu(x) psi(x+nu)
 *                                        + e^{-mu d_nu,4} (1 + g_nu) U_nu(x-nu)^H psi(x-nu) ],
 *   kappa = 1/(2 m_W + 8), chiral gamma matrices, time hops across the boundary times t_bc.
 * The spin factors (1 -/+ g_nu) are applied as full 4x4 matrices and the colour factor as a
 * full 3x3 product: the definition written out, nothing folded or projected.
 *
 * The two-sided Lanczos process (Section 2.2, Eqs. 2sided1/2sided2) in the oracle's reading:
 * v_1 = r / ||r||, w_1 = r~ / conj(r~^H v_1) (so v_1^H w_1 = 1); per step j
 *   alpha_j = w_j^H A v_j,
 *   vh = A v_j - alpha_j v_j - beta_{j-1} v_{j-1},  wh = A^H w_j - conj(alpha_j) w_j - conj(delta_{j-1}) w_{j-1},
 *   ip = wh^H vh, delta_j = sqrt|ip|, beta_j = ip / delta_j, v_{j+1} = vh / delta_j, w_{j+1} = wh / conj(beta_j),
 * breakdown when |ip| < 1e-14 ||vh|| ||wh||. A^H = H_W(-mu) (gamma5-hermiticity).
 * The small sign(H_k) e_1 and the combine are left to the Python side (numpy), as are the
 * deflation split and the sources.
 *
 * Layouts: links U[4][V][3][3], spinors [V][4][3] complex128 (re, im interleaved); site index
 * ((t Lz + z) Ly + y) Lx + x. Work over sites is split across OpenMP threads.
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stddef.h>
#include <stdint.h>

typedef double complex zc;

/* chiral basis: g_k = [[0, -i s_k], [i s_k, 0]] (k = 1..3), g_4 = [[0, 1], [1, 0]] */
static void gamma_matrix(int nu, zc g[4][4]) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) g[a][b] = 0;
  /* Pauli matrices s_1, s_2, s_3 */
  zc s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  if (nu == 3) {
    g[0][2] = g[1][3] = g[2][0] = g[3][1] = 1;
    return;
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      g[a][2 + b] = -I * s[nu][a][b];
      g[2 + a][b] = I * s[nu][a][b];
    }
}

int ovlref_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
}

/* out = H_W(mu) in = gamma5 D_W(mu) in. */
void ovlref_apply_hw(const int32_t* dims, int32_t t_bc, double m_w, double mu, const zc* U, const zc* in,
                     zc* out) {
  const long lx = dims[0], ly = dims[1], lz = dims[2], lt = dims[3];
  const long vol = lx * ly * lz * lt;
  const double kappa = 1.0 / (2.0 * m_w + 8.0);
  zc pm[4][4][4], pp[4][4][4]; /* 1 - g_nu, 1 + g_nu */
  for (int nu = 0; nu < 4; ++nu) {
    zc g[4][4];
    gamma_matrix(nu, g);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        pm[nu][a][b] = (a == b ? 1.0 : 0.0) - g[a][b];
        pp[nu][a][b] = (a == b ? 1.0 : 0.0) + g[a][b];
      }
  }
  const long ext[4] = {lx, ly, lz, lt};
#pragma omp parallel for schedule(static)
  for (long s = 0; s < vol; ++s) {
    long c[4];
    c[0] = s % lx;
    c[1] = (s / lx) % ly;
    c[2] = (s / (lx * ly)) % lz;
    c[3] = s / (lx * ly * lz);
    zc acc[4][3];
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) acc[a][i] = in[s * 12 + a * 3 + i];
    for (int nu = 0; nu < 4; ++nu) {
      long cf[4] = {c[0], c[1], c[2], c[3]}, cb[4] = {c[0], c[1], c[2], c[3]};
      cf[nu] = (c[nu] + 1) % ext[nu];
      cb[nu] = (c[nu] + ext[nu] - 1) % ext[nu];
      const long sf = ((cf[3] * lz + cf[2]) * ly + cf[1]) * lx + cf[0];
      const long sb = ((cb[3] * lz + cb[2]) * ly + cb[1]) * lx + cb[0];
      double ef = 1.0, eb = 1.0;
      if (nu == 3) {
        ef = exp(mu);
        eb = exp(-mu);
        if (c[3] == lt - 1) ef *= t_bc;
        if (c[3] == 0) eb *= t_bc;
      }
      const zc* uf = U + ((long)nu * vol + s) * 9;  /* U_nu(x) */
      const zc* ub = U + ((long)nu * vol + sb) * 9; /* U_nu(x - nu) */
      zc tf[4][3], tb[4][3];
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
          zc f = 0, b = 0;
          for (int j = 0; j < 3; ++j) {
            f += uf[i * 3 + j] * in[sf * 12 + a * 3 + j];
            b += conj(ub[j * 3 + i]) * in[sb * 12 + a * 3 + j];
          }
          tf[a][i] = f;
          tb[a][i] = b;
        }
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
          zc f = 0, b = 0;
          for (int bb = 0; bb < 4; ++bb) {
            f += pm[nu][a][bb] * tf[bb][i];
            b += pp[nu][a][bb] * tb[bb][i];
          }
          acc[a][i] -= kappa * (ef * f + eb * b);
        }
    }
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) out[s * 12 + a * 3 + i] = (a < 2 ? 1.0 : -1.0) * acc[a][i];
  }
}

/* a^H b: 64 fixed chunks summed in order, so the result does not depend on the thread count. */
#define VDOT_CHUNKS 64
static zc vdot(long n, const zc* a, const zc* b) {
  double pr[VDOT_CHUNKS], pi[VDOT_CHUNKS];
#pragma omp parallel for schedule(static)
  for (int c = 0; c < VDOT_CHUNKS; ++c) {
    const long lo = n * c / VDOT_CHUNKS, hi = n * (c + 1) / VDOT_CHUNKS;
    double re = 0, im = 0;
    for (long i = lo; i < hi; ++i) {
      zc p = conj(a[i]) * b[i];
      re += creal(p);
      im += cimag(p);
    }
    pr[c] = re;
    pi[c] = im;
  }
  double re = 0, im = 0;
  for (int c = 0; c < VDOT_CHUNKS; ++c) {
    re += pr[c];
    im += pi[c];
  }
  return re + I * im;
}

static double norm(long n, const zc* a) { return sqrt(creal(vdot(n, a, a))); }

/* Start of the process from (r, r~): V[0] = v_1, W[0] = w_1; returns ||r|| in *beta0.
 * Returns 0, or 1 when ||r|| = 0 or r~^H v_1 = 0 (no process). */
int ovlref_lanczos_start(long n, const zc* r, const zc* rt, zc* V, zc* W, double* beta0) {
  const double b0 = norm(n, r);
  *beta0 = b0;
  if (!(b0 > 0)) return 1;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) V[i] = r[i] / b0;
  const zc d = vdot(n, rt, V);
  if (d == 0) return 1;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) W[i] = rt[i] / conj(d);
  return 0;
}

/* Steps j = *k_io + 1 .. *k_io + nsteps (1-based) of the process. V holds columns v_1..v_{kcap}
 * ([kcap][n]); W two rotating shadow vectors ([2][n], w_j in slot (j-1) % 2); av, aw scratch [n];
 * alpha, beta, delta [kcap] (complex; delta real). Step j computes alpha_j and, if j < kcap, the
 * pair beta_j, delta_j and v_{j+1}, w_{j+1}. On return *k_io is the number of completed steps.
 * Returns 0, or 1 on breakdown (then *k_io = the step whose alpha is the last one). */
int ovlref_lanczos_steps(const int32_t* dims, int32_t t_bc, double m_w, double mu, const zc* U, long n, int kcap,
                         zc* V, zc* W, zc* av, zc* aw, zc* alpha, zc* beta, zc* delta, int* k_io, int nsteps) {
  int j0 = *k_io;
  for (int j = j0 + 1; j <= j0 + nsteps && j <= kcap; ++j) {
    zc* v = V + (long)(j - 1) * n;
    zc* w = W + (long)((j - 1) % 2) * n;
    zc* wprev = W + (long)(j % 2) * n; /* w_{j-1}; overwritten by w_{j+1} below */
    const zc* vprev = j > 1 ? V + (long)(j - 2) * n : NULL;
    ovlref_apply_hw(dims, t_bc, m_w, mu, U, v, av);
    ovlref_apply_hw(dims, t_bc, m_w, -mu, U, w, aw);
    const zc a = vdot(n, w, av);
    alpha[j - 1] = a;
    *k_io = j;
    if (j == kcap) break;
    const zc bprev = j > 1 ? beta[j - 2] : 0, dprev = j > 1 ? delta[j - 2] : 0;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
      zc x = av[i] - a * v[i];
      zc y = aw[i] - conj(a) * w[i];
      if (vprev) {
        x -= bprev * vprev[i];
        y -= conj(dprev) * wprev[i];
      }
      av[i] = x;
      aw[i] = y;
    }
    const zc ip = vdot(n, aw, av);
    if (cabs(ip) < 1e-14 * norm(n, av) * norm(n, aw)) return 1;
    const double d = sqrt(cabs(ip));
    const zc bt = ip / d;
    delta[j - 1] = d;
    beta[j - 1] = bt;
    zc* vnext = V + (long)j * n;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
      vnext[i] = av[i] / d;
      wprev[i] = aw[i] / conj(bt);
    }
  }
  return 0;
}

/* x += c * sum_{j < k} y_j V[j]  (the combine x = x_P + beta V_k y with c = beta). */
void ovlref_combine(long n, int k, const zc* V, const zc* y, double c, zc* x) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    zc s = 0;
    for (int j = 0; j < k; ++j) s += y[j] * V[(long)j * n + i];
    x[i] += c * s;
  }
}
