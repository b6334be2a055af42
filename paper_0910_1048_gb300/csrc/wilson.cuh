// Site-level Wilson hop arithmetic shared by the stencil kernels.
//
// (D_W psi)(x) = psi(x) - kappa sum_nu [ e^{+mu d_nu,t} (1 - g_nu) U_nu(x) psi(x+nu)
//                                      + e^{-mu d_nu,t} (1 + g_nu) U_nu(x-nu)^H psi(x-nu) ]
// (the reading of the paper's H_W = gamma5 D_W, Section 1, with the notation of its
// reference [Bloch:2006cd]); t hops that wrap the time boundary carry t_bc.
//
// Chiral basis: g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]]. Writing
// g_nu = [[0, M], [N, 0]] on (upper, lower) spin pairs, (1 -/+ g_nu) psi is determined by
// the half spinor h = upper -/+ M lower: (1 - g) psi = (h, -N h), (1 + g) psi = (h, N h).
// Only h (2 spins x 3 colours) is multiplied by the link.
#pragma once

#include <cmath>

#include "common.h"

#if defined(__CUDACC__)
#include <cuda_fp16.h>
#endif

namespace ovl {

template <class R> struct Spin { cplx<R> c[4][3]; };
template <class R> struct Half { cplx<R> c[2][3]; };
template <class R> struct Mat3 { cplx<R> m[3][3]; };

// Half spinor h of (1 - g_mu) p (FWD) or (1 + g_mu) p (!FWD).
template <int MU, bool FWD, class R>
OVL_HD void project(const Spin<R>& p, Half<R>& h) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (MU == 0) {  // M l = (-i p3, -i p2)
      h.c[0][a] = FWD ? p.c[0][a] + times_i(p.c[3][a]) : p.c[0][a] + times_mi(p.c[3][a]);
      h.c[1][a] = FWD ? p.c[1][a] + times_i(p.c[2][a]) : p.c[1][a] + times_mi(p.c[2][a]);
    } else if (MU == 1) {  // M l = (-p3, p2)
      h.c[0][a] = FWD ? p.c[0][a] + p.c[3][a] : p.c[0][a] - p.c[3][a];
      h.c[1][a] = FWD ? p.c[1][a] - p.c[2][a] : p.c[1][a] + p.c[2][a];
    } else if (MU == 2) {  // M l = (-i p2, i p3)
      h.c[0][a] = FWD ? p.c[0][a] + times_i(p.c[2][a]) : p.c[0][a] + times_mi(p.c[2][a]);
      h.c[1][a] = FWD ? p.c[1][a] + times_mi(p.c[3][a]) : p.c[1][a] + times_i(p.c[3][a]);
    } else {  // M l = (p2, p3)
      h.c[0][a] = FWD ? p.c[0][a] - p.c[2][a] : p.c[0][a] + p.c[2][a];
      h.c[1][a] = FWD ? p.c[1][a] - p.c[3][a] : p.c[1][a] + p.c[3][a];
    }
  }
}

// a*b + c, one fused operation on host and device.
template <class R>
OVL_HD R mad(R a, R b, R c) {
#if defined(__CUDA_ARCH__)
  return fma(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// a += f * rot(h) with rot = identity (ROT 0), i (1), -1 (2), -i (3): two fused operations.
template <int ROT, class R>
OVL_HD void acc_rot(cplx<R>& a, R f, const cplx<R>& h) {
  const R vr = ROT == 0 ? h.re : ROT == 1 ? -h.im : ROT == 2 ? -h.re : h.im;
  const R vi = ROT == 0 ? h.im : ROT == 1 ? h.re : ROT == 2 ? -h.im : -h.re;
  a.re = mad(f, vr, a.re);
  a.im = mad(f, vi, a.im);
}

// acc += f (h, -/+ N h): the full spinor of the projected hop, with the hop coefficient f
// folded into the accumulation.
template <int MU, bool FWD, class R>
OVL_HD void reconstruct_add(Spin<R>& acc, const Half<R>& h, R f) {
  // lower rows: N h takes (h1, h0) for MU 0, 1 and (h0, h1) for MU 2, 3
  constexpr int i2 = MU < 2 ? 1 : 0, i3 = MU < 2 ? 0 : 1;
  // rotation applied to each: MU 0: FWD (-i, -i) / BWD (i, i); MU 1: (-1, 1) / (1, -1);
  // MU 2: (-i, i) / (i, -i); MU 3: (-1, -1) / (1, 1)
  constexpr int r2 = MU == 0 ? (FWD ? 3 : 1) : MU == 1 ? (FWD ? 2 : 0) : MU == 2 ? (FWD ? 3 : 1) : (FWD ? 2 : 0);
  constexpr int r3 = MU == 0 ? (FWD ? 3 : 1) : MU == 1 ? (FWD ? 0 : 2) : MU == 2 ? (FWD ? 1 : 3) : (FWD ? 2 : 0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc_rot<0>(acc.c[0][a], f, h.c[0][a]);
    acc_rot<0>(acc.c[1][a], f, h.c[1][a]);
    acc_rot<r2>(acc.c[2][a], f, h.c[i2][a]);
    acc_rot<r3>(acc.c[3][a], f, h.c[i3][a]);
  }
}

// out = U h (DAG false) or U^H h (DAG true), colour multiply of both half-spinor rows as
// chains of fused multiply-adds (the first product seeds the chain).
template <bool DAG, class R>
OVL_HD void su3_mul(const Mat3<R>& u, const Half<R>& h, Half<R>& out) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // m_b = U[a][b] or conj(U[b][a]); out = sum_b m_b h_b
      const R sg = DAG ? (R)-1 : (R)1;  // sign of Im m_b
      cplx<R> m = DAG ? u.m[0][a] : u.m[a][0];
      const cplx<R>& x = h.c[s][0];
      R re = m.re * x.re;
      R im = m.re * x.im;
      re = mad(-sg * m.im, x.im, re);
      im = mad(sg * m.im, x.re, im);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        m = DAG ? u.m[b][a] : u.m[a][b];
        const cplx<R>& y = h.c[s][b];
        re = mad(m.re, y.re, mad(-sg * m.im, y.im, re));
        im = mad(m.re, y.im, mad(sg * m.im, y.re, im));
      }
      out.c[s][a] = mk<R>(re, im);
    }
  }
}

// ------------------------------------------------------------------ link loads
template <int LF, class R>
OVL_HD void load_link(const Links& U, int mu, int site, int vol, Mat3<R>& u) {
  if (LF == LINK_F64) {
    const double2* p = U.f64 + (size_t)mu * 9 * vol + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = p[(size_t)k * vol];
      u.m[k / 3][k % 3] = mk<R>((R)v.x, (R)v.y);
    }
  } else if (LF == LINK_F32) {
    const float2* p = U.f32 + (size_t)mu * 9 * vol + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float2 v = p[(size_t)k * vol];
      u.m[k / 3][k % 3] = mk<R>((R)v.x, (R)v.y);
    }
  } else {
#if defined(__CUDA_ARCH__)
    const uint32_t* p = U.f16 + (size_t)mu * 6 * vol + site;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      uint32_t bits = p[(size_t)k * vol];
      __half2 hv = *reinterpret_cast<__half2*>(&bits);
      float2 f = __half22float2(hv);
      u.m[k / 3][k % 3] = mk<R>((R)f.x, (R)f.y);
    }
    // third row of an SU(3) matrix: conj(row0 x row1)
    u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
    u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
    u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
#endif
  }
}

// ------------------------------------------------------------------ neighbours
struct Nbr {
  int f[4], b[4];  // forward / backward neighbour site per direction
  int t;           // time coordinate (for the boundary sign)
};

OVL_HD void neighbours(const Geom& g, int s, Nbr& n) {
  int x = s % g.lx;
  int r = s / g.lx;
  int y = r % g.ly;
  r /= g.ly;
  int z = r % g.lz;
  int t = r / g.lz;
  n.t = t;
  n.f[0] = (x == g.lx - 1) ? s - (g.lx - 1) : s + 1;
  n.b[0] = (x == 0) ? s + (g.lx - 1) : s - 1;
  n.f[1] = (y == g.ly - 1) ? s - (g.ly - 1) * g.sy : s + g.sy;
  n.b[1] = (y == 0) ? s + (g.ly - 1) * g.sy : s - g.sy;
  n.f[2] = (z == g.lz - 1) ? s - (g.lz - 1) * g.sz : s + g.sz;
  n.b[2] = (z == 0) ? s + (g.lz - 1) * g.sz : s - g.sz;
  n.f[3] = (t == g.lt - 1) ? s - (g.lt - 1) * g.st : s + g.st;
  n.b[3] = (t == 0) ? s + (g.lt - 1) * g.st : s - g.st;
}

// Hop coefficients: spatial -kappa; time forward -kappa e^{mu}, backward -kappa e^{-mu},
// each times t_bc where the hop wraps the time boundary.
template <class R>
struct HopCoef {
  R ks, ktf, ktb;
};

// acc += one hop term: forward (FWD, from site x + mu with U_mu(x)) or backward (from x - mu with
// U_mu(x - mu)^H), coefficient k, input p loaded by `ld`.
template <int MU, bool FWD, int LF, class R, class Load>
OVL_HD void hop_one(const Geom& g, const Links& U, int s, const Nbr& n, R k, Load ld, Spin<R>& acc) {
  Mat3<R> u;
  Half<R> h, hu;
  Spin<R> p;
  ld(FWD ? n.f[MU] : n.b[MU], p);
  project<MU, FWD>(p, h);
  load_link<LF>(U, MU, FWD ? s : n.b[MU], g.vol, u);
  su3_mul<!FWD>(u, h, hu);
  reconstruct_add<MU, FWD>(acc, hu, k);
}

// acc += hop terms for one direction (forward and backward).
template <int MU, int LF, class R, class Load>
OVL_HD void hop_dir(const Geom& g, const Links& U, int s, const Nbr& n, R kf, R kb, Load ld, Spin<R>& acc) {
  hop_one<MU, true, LF>(g, U, s, n, kf, ld, acc);
  hop_one<MU, false, LF>(g, U, s, n, kb, ld, acc);
}

// out = D_W psi at site s (psi loaded through `ld`), coefficients c.
template <int LF, class R, class Load>
OVL_HD void dslash_site(const Geom& g, const Links& U, int s, const HopCoef<R>& c, Load ld, Spin<R>& out) {
  Nbr n;
  neighbours(g, s, n);
  ld(s, out);
  hop_dir<0, LF>(g, U, s, n, c.ks, c.ks, ld, out);
  hop_dir<1, LF>(g, U, s, n, c.ks, c.ks, ld, out);
  hop_dir<2, LF>(g, U, s, n, c.ks, c.ks, ld, out);
  R ktf = (n.t == g.lt - 1) ? (R)g.t_bc * c.ktf : c.ktf;
  R ktb = (n.t == 0) ? (R)g.t_bc * c.ktb : c.ktb;
  hop_dir<3, LF>(g, U, s, n, ktf, ktb, ld, out);
}

// The same operator for G right-hand sides at once (the first `nact` of them active): each link is
// loaded once per site and applied to every source of the group, so a batch of sources reads the
// links G times less often. out[r] = D_W psi_r at site s.
template <int MU, bool FWD, int LF, int G, class R, class Load>
OVL_HD void hop_one_g(const Geom& g, const Links& U, int s, const Nbr& n, R k, const Load (&ld)[G], int nact,
                      Spin<R> (&acc)[G]) {
  Mat3<R> u;
  load_link<LF>(U, MU, FWD ? s : n.b[MU], g.vol, u);
#pragma unroll
  for (int r = 0; r < G; ++r) {
    if (r < nact) {
      Half<R> h, hu;
      Spin<R> p;
      ld[r](FWD ? n.f[MU] : n.b[MU], p);
      project<MU, FWD>(p, h);
      su3_mul<!FWD>(u, h, hu);
      reconstruct_add<MU, FWD>(acc[r], hu, k);
    }
  }
}

template <int MU, int LF, int G, class R, class Load>
OVL_HD void hop_dir_g(const Geom& g, const Links& U, int s, const Nbr& n, R kf, R kb, const Load (&ld)[G], int nact,
                      Spin<R> (&acc)[G]) {
  hop_one_g<MU, true, LF, G>(g, U, s, n, kf, ld, nact, acc);
  hop_one_g<MU, false, LF, G>(g, U, s, n, kb, ld, nact, acc);
}

template <int LF, int G, class R, class Load>
OVL_HD void dslash_site_g(const Geom& g, const Links& U, int s, const HopCoef<R>& c, const Load (&ld)[G], int nact,
                          Spin<R> (&out)[G]) {
  Nbr n;
  neighbours(g, s, n);
#pragma unroll
  for (int r = 0; r < G; ++r)
    if (r < nact) ld[r](s, out[r]);
  hop_dir_g<0, LF, G>(g, U, s, n, c.ks, c.ks, ld, nact, out);
  hop_dir_g<1, LF, G>(g, U, s, n, c.ks, c.ks, ld, nact, out);
  hop_dir_g<2, LF, G>(g, U, s, n, c.ks, c.ks, ld, nact, out);
  R ktf = (n.t == g.lt - 1) ? (R)g.t_bc * c.ktf : c.ktf;
  R ktb = (n.t == 0) ? (R)g.t_bc * c.ktb : c.ktb;
  hop_dir_g<3, LF, G>(g, U, s, n, ktf, ktb, ld, nact, out);
}

template <class R>
OVL_HD void gamma5_inplace(Spin<R>& p) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p.c[2][a] = -p.c[2][a];
    p.c[3][a] = -p.c[3][a];
  }
}

template <class R>
OVL_HD HopCoef<R> hop_coef(double m_w, double mu) {
  double kap = 1.0 / (2.0 * m_w + 8.0);
  HopCoef<R> c;
  c.ks = (R)(-kap);
  c.ktf = (R)(-kap * std::exp(mu));
  c.ktb = (R)(-kap * std::exp(-mu));
  return c;
}

}  // namespace ovl
