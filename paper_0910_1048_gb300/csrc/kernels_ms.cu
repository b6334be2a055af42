// Multishift BiCG kernels (Algorithm 3 on M = A^2, A = H_W(mu); Section 5's rational sign).
//
// One iteration k is four launches:
//   pair1:  t = A p,  t~ = A^H p~                                   (A^H = H_W(-mu))
//   pair2:  q = A t - s1 p = (M - s1) p,  q~ = A^H t~ - s1 p~;  alpha_k = rho / (p~^H q);
//           last block: zeta^i_{k+1}, alpha^i_k for every live shift
//   update: r -= alpha_k q,  r~ -= conj(alpha_k) q~;  rho' = r~^H r, |r|;
//           last block: beta_k = rho'/rho, beta^i_k = beta_k (zeta^i_{k+1}/zeta^i_k)^2,
//           shifts with |zeta^i_{k+1}| |r| <= tol |r_0| are retired after this step
//   dirs:   X += sum_i omega_i alpha^i_k p^i;  p^i = zeta^i_{k+1} r + beta^i_k p^i;
//           p = r + beta_k p,  p~ = r~ + conj(beta_k) p~
// The shifted recurrences follow from the BiCG residual polynomials: r_k = R_k(M0) r_0 with
// R_{k+1}(t) = (1 + a_k b_{k-1}/a_{k-1} - a_k t) R_k(t) - (a_k b_{k-1}/a_{k-1}) R_{k-1}(t), and the
// residual of (M0 - d) x = r_0 in the same Krylov space is R_k(d)^-1 r_k, i.e. zeta = 1/R_k(d).
#include "devutil.cuh"
#include "kernels.h"

namespace ovl {

template <class R>
__device__ __forceinline__ size_t voff(int rhs, size_t n) { return (size_t)rhs * n; }

// start: r = b - R L^H b, r~ = b - L R^H b, x_P; p = r, p~ = r~, p^i = r, X = 0
template <class R>
__global__ void __launch_bounds__(kBlock) k_ms_start(Geom g, MsDev ms, MsVecs v, const double2* b, int m,
                                                     const double2* Rv, const double2* Lv, const double* lam_sign,
                                                     const double2* dots) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)12 * g.vol;
  double acc[4] = {0, 0, 0, 0};
  if (s < g.vol) {
    const double2* dr = dots + (size_t)rhs * 2 * m;
    for (int c = 0; c < 12; ++c) {
      zd bv = ldc<double>(b, (size_t)rhs * n + (size_t)s * 12 + c);
      zd r = bv, rt = bv, x = mk(0.0, 0.0);
      for (int i = 0; i < m; ++i) {
        zd ci = ldc<double>(dr, i), di = ldc<double>(dr, m + i);
        zd ri = ldc<double>(Rv, (size_t)i * n + (size_t)c * g.vol + s);
        zd li = ldc<double>(Lv, (size_t)i * n + (size_t)c * g.vol + s);
        r = r - ci * ri;
        x = x + lam_sign[i] * (ci * ri);
        rt = rt - di * li;
      }
      const size_t e = voff<R>(rhs, n) + (size_t)c * g.vol + s;
      if (v.xp) stc<double>(v.xp, e, x);
      if (v.r64) stc<double>(v.r64, e, r);
      if (v.xs)
        for (int i = 0; i < ms.s; ++i) stc<double>(v.xs, ((size_t)rhs * ms.s + i) * n + (size_t)c * g.vol + s, mk(0.0, 0.0));
      stc<double>(v.X, e, mk(0.0, 0.0));
      cplx<R> rr = mk<R>((R)r.re, (R)r.im), rtt = mk<R>((R)rt.re, (R)rt.im);
      stc<R>((T*)v.r, e, rr);
      stc<R>((T*)v.p, e, rr);
      stc<R>((T*)v.rt, e, rtt);
      stc<R>((T*)v.pt, e, rtt);
      for (int i = 0; i < ms.s; ++i) stc<R>((T*)v.ps, ((size_t)rhs * ms.s + i) * n + (size_t)c * g.vol + s, rr);
      // rho and |r| from the stored (rounded) vectors, so the recurrences start consistent
      zd rd = mk((double)rr.re, (double)rr.im), rtd = mk((double)rtt.re, (double)rtt.im);
      zd ip = cdot(rtd, rd);
      acc[0] += ip.re;
      acc[1] += ip.im;
      acc[2] += norm2(rd);
    }
  }
  block_sum<4>(acc);
  double* part = ms.part + (size_t)rhs * ms.nblk * 4;
  if (publish_partials<4>(acc, part, ms.count + rhs)) {
    reduce_partials<4>(part, gridDim.x, acc);
    const int t = lin_tid();
    double2* sd = ms.seed + (size_t)rhs * 8;
    if (t == 0) {
      double rn = sqrt(acc[2]);
      sd[0] = make_double2(acc[0], acc[1]);  // rho
      sd[1] = make_double2(0, 0);
      sd[2] = make_double2(1, 0);  // alpha_{-1}
      sd[3] = make_double2(0, 0);  // beta_{-1}
      sd[4] = make_double2(rn, rn);
      sd[5] = make_double2(0, 0);
      ms.k[rhs] = 0;
      ms.status[rhs] = acc[2] == 0.0 ? 3 : ((acc[0] != 0.0 || acc[1] != 0.0) ? 0 : 1);
    }
    for (int i = t; i < ms.s; i += lin_nthreads()) {
      double2* z = ms.zeta + ((size_t)rhs * ms.s + i) * 3;
      z[0] = z[1] = z[2] = make_double2(1, 0);
      ms.active[(size_t)rhs * ms.s + i] = 1;
      ms.ash[(size_t)rhs * ms.s + i] = make_double2(0, 0);
      ms.bsh[(size_t)rhs * ms.s + i] = make_double2(0, 0);
    }
  }
}

// Every FP64 instruction is slow on GB300's narrow FP64 pipe, so the last blocks' recurrences keep
// their dependent chains short (one division per shift, comparisons on squares). Blocks have at
// least as many threads as shifts (s <= 127), so thread t holds shift t.
struct MsAlphaIn {
  zd rho, akm, bkm;  // rho_k, alpha_{k-1}, beta_{k-1}
  int act;           // shift t: 0 retired, 1 live, 2 last direction update done
  zd zm, z0;         // zeta^t_{k-1}, zeta^t_k
  double dsig;       // sigma_t - sigma_1
};

__device__ __forceinline__ MsAlphaIn ms_alpha_inputs(const MsDev& ms, int rhs) {
  MsAlphaIn in{};
  const double2* sd = ms.seed + (size_t)rhs * 8;
  const int t = lin_tid();
  in.rho = ldc<double>(sd, 0);
  in.akm = ldc<double>(sd, 2);
  in.bkm = ldc<double>(sd, 3);
  if (t < ms.s) {
    const size_t si = (size_t)rhs * ms.s + t;
    in.act = ms.active[si];
    const double2* z = ms.zeta + si * 3;
    in.zm = ldc<double>(z, 0);
    in.z0 = ldc<double>(z, 1);
    in.dsig = ms.dsig[t];
  }
  return in;
}

// last block of pair2: alpha_k, then zeta^i_{k+1} and alpha^i_k of the live shifts
__device__ __forceinline__ void ms_alpha_and_shifts(MsDev& ms, int rhs, const double (&pv)[4], const MsAlphaIn& in) {
  __shared__ zd alpha_sh;
  __shared__ int bad;
  const int t = lin_tid();
  double2* sd = ms.seed + (size_t)rhs * 8;
  if (t == 0) {
    zd den = mk(pv[0], pv[1]);
    double dd = norm2(den);
    bad = !(dd > 0.0) || !(dd < 1e300);
    zd alpha = bad ? mk(0.0, 0.0) : (1.0 / dd) * (in.rho * conj(den));
    alpha_sh = alpha;
    if (bad) ms.status[rhs] = 1;
    sd[1] = make_double2(alpha.re, alpha.im);
  }
  __syncthreads();
  if (bad) return;
  const zd ak = alpha_sh, akm = in.akm, bkm = in.bkm;
  for (int i = t; i < ms.s; i += lin_nthreads()) {
    const size_t si = (size_t)rhs * ms.s + i;
    double2* z = ms.zeta + si * 3;
    const bool mine = i == t;
    int act = mine ? in.act : ms.active[si];
    if (act == 2) ms.active[si] = act = 0;
    if (!act) continue;
    const zd zm = mine ? in.zm : ldc<double>(z, 0), z0 = mine ? in.z0 : ldc<double>(z, 1);
    const double ds = mine ? in.dsig : ms.dsig[i];
    zd d1 = mk(1.0 - ak.re * ds, -ak.im * ds);
    zd den = akm * zm * d1 + ak * bkm * (zm - z0);
    zd num = z0 * zm * akm;
    const double dn = norm2(den), z0n = norm2(z0);
    const zd nc = num * conj(den);
    zd zp = mk(0.0, 0.0), ai = mk(0.0, 0.0);
    const double prod = dn * z0n;
    if (prod > 1e-300 && prod < 1e300) {  // zeta^i_{k+1} = num / den, alpha^i_k = alpha_k zeta^i_{k+1} / zeta^i_k
      const double inv = 1.0 / prod;
      zp = (z0n * inv) * nc;
      ai = ak * (inv * (nc * conj(z0)));
    } else {  // the same with one division each (a product outside the safe range)
      if (dn > 0) zp = (1.0 / dn) * nc;
      if (z0n > 0) ai = ak * ((1.0 / z0n) * (zp * conj(z0)));
    }
    z[2] = make_double2(zp.re, zp.im);
    ms.ash[si] = make_double2(ai.re, ai.im);
  }
}

// pair1 (MODE 0): t = A p, t~ = A^H p~.  pair2 (MODE 1): q = A t - s1 p, q~ = A^H t~ - s1 p~, p~^H q.
template <class R, int LF, int MODE>
__global__ void __launch_bounds__(2 * kPairSites) k_ms_pair(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm, MsDev ms,
                                                            MsVecs v) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (MODE == 0 && blockIdx.x == 0 && lin_tid() == 0 && ms.status[rhs] == 4) ms.status[rhs] = 2;
  if (ms.status[rhs] != 0) return;
  const size_t n = (size_t)12 * g.vol;
  const int s = blockIdx.x * kPairSites + threadIdx.x;
  const bool is_t = threadIdx.y == 1;
  const T* in = (const T*)(MODE == 0 ? (is_t ? v.pt : v.p) : (is_t ? v.tt : v.t)) + voff<R>(rhs, n);
  T* out = (T*)(MODE == 0 ? (is_t ? v.tt : v.t) : (is_t ? v.qt : v.q)) + voff<R>(rhs, n);
  const double s1d = ms.sig1v ? ms.sig1v[rhs] : ms.sigma1;
  R s1v[1];
  scalars_in<R, 1>(&s1d, s1v);
  Red<R> acc[2];
  if (s < g.vol) {
    Spin<R> o;
    dslash_site<LF, R>(g, U, s, is_t ? cm : cp, Loader<R, true>{in, g.vol, false}, o);
    const R s1 = s1v[0];
    const T* pp = (const T*)(is_t ? v.pt : v.p) + voff<R>(rhs, n);
    const T* ptl = (const T*)v.pt + voff<R>(rhs, n);
    // MODE 1: every load before the first store (stores that might alias would otherwise
    // serialise twelve memory round trips)
    cplx<R> pv[12], tv[12];
    if (MODE == 1) {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        pv[c] = ldc<R>(pp, (size_t)c * g.vol + s);
        tv[c] = is_t ? mk<R>(0, 0) : ldc<R>(ptl, (size_t)c * g.vol + s);
      }
    }
    cplx<R> a = mk<R>(0, 0);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      cplx<R> x = o.c[c / 3][c % 3];
      if (c >= 6) x = -x;  // gamma5
      if (MODE == 1) {
        x = x - s1 * pv[c];
        if (!is_t) a = a + cdot(tv[c], x);
      }
      stc<R>(out, (size_t)c * g.vol + s, x);
    }
    acc[0].add(a.re);
    acc[1].add(a.im);
  }
  if (MODE == 0) return;
  double tot[2];
  block_reduce<R, 2>(acc, tot);
  double* part = ms.part + (size_t)rhs * ms.nblk * 4;
  double pv[4] = {tot[0], tot[1], 0, 0};
  if (publish_partials<4>(pv, part, ms.count + rhs)) {
    // (the inputs are loaded after the sum here: held across it they cost the whole stencil
    // kernel registers, 80 -> 106, and occupancy)
    reduce_partials<4>(part, gridDim.x, pv);
    ms_alpha_and_shifts(ms, rhs, pv, ms_alpha_inputs(ms, rhs));
  }
}

// pair1 / pair2 with 8 threads per site (small lattices): see pair_split.
template <class R, int LF, int MODE>
__global__ void __launch_bounds__(8 * kSplitSites) k_ms_pair_split(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm,
                                                                   MsDev ms, MsVecs v) {
  using T = typename V2<R>::T;
  __shared__ SplitSmem<R> sm;
  const int rhs = blockIdx.y;
  if (MODE == 0 && blockIdx.x == 0 && lin_tid() == 0 && ms.status[rhs] == 4) ms.status[rhs] = 2;
  if (ms.status[rhs] != 0) return;
  const size_t n = (size_t)12 * g.vol;
  const T* in0 = (const T*)(MODE == 0 ? v.p : v.t) + voff<R>(rhs, n);
  const T* in1 = (const T*)(MODE == 0 ? v.pt : v.tt) + voff<R>(rhs, n);
  const double s1d = ms.sig1v ? ms.sig1v[rhs] : ms.sigma1;
  R s1v[1];
  scalars_in<R, 1>(&s1d, s1v);
  const R s1 = s1v[0];
  Red<R> acc[2];
  // each thread finishes one spin (three colours) of its site: see pair_split
  pair_split<R, LF>(g, U, cp, cm, in0, in1, sm, [&](int which, int s, int sp, cplx<R> (&o)[3]) {
    T* out = (T*)(MODE == 0 ? (which ? v.tt : v.t) : (which ? v.qt : v.q)) + voff<R>(rhs, n);
    const T* pp = (const T*)(which ? v.pt : v.p) + voff<R>(rhs, n);
    const T* ptl = (const T*)v.pt + voff<R>(rhs, n);
    const R g5 = sp >= 2 ? (R)-1 : (R)1;
    cplx<R> pv[3], tv[3];  // loads first (see k_ms_pair)
    if (MODE == 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pv[a] = ldc<R>(pp, (size_t)(sp * 3 + a) * g.vol + s);
        tv[a] = which ? mk<R>(0, 0) : ldc<R>(ptl, (size_t)(sp * 3 + a) * g.vol + s);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> x = g5 * o[a];
      if (MODE == 1) {
        x = x - s1 * pv[a];
        if (!which) {
          acc[0].dot2(tv[a].re, x.re, tv[a].im, x.im);
          acc[1].dot2(tv[a].re, x.im, -tv[a].im, x.re);
        }
      }
      stc<R>(out, (size_t)(sp * 3 + a) * g.vol + s, x);
    }
  });
  if (MODE == 0) return;
  double tot[2];
  block_reduce<R, 2>(acc, tot);
  double* part = ms.part + (size_t)rhs * ms.nblk * 4;
  double pv[4] = {tot[0], tot[1], 0, 0};
  if (publish_partials<4>(pv, part, ms.count + rhs)) {
    // (the inputs are loaded after the sum here: held across it they cost the whole stencil
    // kernel registers, 80 -> 106, and occupancy)
    reduce_partials<4>(part, gridDim.x, pv);
    ms_alpha_and_shifts(ms, rhs, pv, ms_alpha_inputs(ms, rhs));
  }
}

// update: r -= alpha q, r~ -= conj(alpha) q~; rho' = r~^H r, |r|^2 (elt elements per thread)
template <class R>
__global__ void __launch_bounds__(kVecBlock) k_ms_update(Geom g, MsDev ms, MsVecs v, int elt) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (ms.status[rhs] != 0) return;
  const size_t n = (size_t)12 * g.vol;
  double2* sd = ms.seed + (size_t)rhs * 8;
  R akr[2];
  scalars_in<R, 2>((const double*)(sd + 1), akr);
  const cplx<R> a = mk<R>(akr[0], akr[1]), ac = mk<R>(akr[0], -akr[1]);
  T* r = (T*)v.r + voff<R>(rhs, n);
  T* rt = (T*)v.rt + voff<R>(rhs, n);
  const T* q = (const T*)v.q + voff<R>(rhs, n);
  const T* qt = (const T*)v.qt + voff<R>(rhs, n);
  Red<R> red[3];
  for (int k = 0; k < elt; ++k) {
    const size_t e = ((size_t)blockIdx.x * elt + k) * blockDim.x + threadIdx.x;
    if (e >= n) break;
    cplx<R> x = cmsub(ldc<R>(r, e), a, ldc<R>(q, e));
    cplx<R> y = cmsub(ldc<R>(rt, e), ac, ldc<R>(qt, e));
    stc<R>(r, e, x);
    stc<R>(rt, e, y);
    red[0].add(fma(y.re, x.re, y.im * x.im));  // (y^H x).re
    red[1].add(fma(y.re, x.im, -(y.im * x.re)));
    red[2].add(fma(x.re, x.re, x.im * x.im));
  }
  double acc[3];
  block_reduce<R, 3>(red, acc);
  double* part = ms.part + (size_t)rhs * ms.nblk * 4;
  double pv[4] = {acc[0], acc[1], acc[2], 0};
  if (publish_partials<4>(pv, part, ms.count + rhs)) {
    // this block's inputs first (their latency overlaps the sum): rho_k, |r_0|, shift t's state
    const int t = lin_tid();
    const double tl = ms.tolv ? ms.tolv[rhs] : ms.tol;
    const zd rho = ldc<double>(sd, 0);
    const double r0 = sd[4].x;
    int act0 = 0;
    zd z1 = mk(0.0, 0.0), z2 = mk(0.0, 0.0);
    if (t < ms.s) {
      const size_t si = (size_t)rhs * ms.s + t;
      act0 = ms.active[si];
      z1 = ldc<double>(ms.zeta + si * 3, 1);
      z2 = ldc<double>(ms.zeta + si * 3, 2);
    }
    reduce_partials<4>(part, gridDim.x, pv);
    __shared__ zd beta_sh;
    __shared__ double r2_sh;
    __shared__ int live;
    if (t == 0) {
      zd rhon = mk(pv[0], pv[1]);
      double rr = norm2(rho);
      zd beta = rr > 0 ? (1.0 / rr) * (rhon * conj(rho)) : mk(0.0, 0.0);
      double rn = sqrt(pv[2]);
      beta_sh = beta;
      r2_sh = pv[2];
      live = 0;
      sd[0] = make_double2(rhon.re, rhon.im);
      sd[2] = sd[1];  // alpha_{k-1} <- alpha_k
      sd[3] = make_double2(beta.re, beta.im);
      sd[5] = make_double2(beta.re, beta.im);
      sd[4].y = rn;
      ms.k[rhs] += 1;
      // breakdown of the BiCG recurrence (rho' = 0 while r is not small) or non-finite values
      if (!(rn < 1e300) || !(norm2(rhon) < 1e300) || (norm2(rhon) == 0.0 && rn > tl * sd[4].x))
        ms.status[rhs] = 1;
    }
    __syncthreads();
    const zd beta = beta_sh;
    const double r2 = r2_sh, lim = (tl * r0) * (tl * r0);
    int mylive = 0;
    for (int i = t; i < ms.s; i += lin_nthreads()) {
      const size_t si = (size_t)rhs * ms.s + i;
      const bool mine = i == t;
      if (!(mine ? act0 : ms.active[si])) continue;
      double2* z = ms.zeta + si * 3;
      const zd z0 = mine ? z1 : ldc<double>(z, 1), zp = mine ? z2 : ldc<double>(z, 2);
      double z0n = norm2(z0);
      zd ratio = z0n > 0 ? (1.0 / z0n) * (zp * conj(z0)) : mk(0.0, 0.0);
      zd bi = beta * (ratio * ratio);
      ms.bsh[si] = make_double2(bi.re, bi.im);
      z[0] = make_double2(z0.re, z0.im);
      z[1] = make_double2(zp.re, zp.im);
      if (norm2(zp) * r2 <= lim)  // |zeta^i_{k+1}| |r_{k+1}| <= tol |r_0|, on squares
        ms.active[si] = 2;  // this step's direction update is its last
      else
        mylive = 1;
    }
    if (mylive) atomicOr(&live, 1);
    __syncthreads();
    if (t == 0 && !live && ms.status[rhs] == 0) ms.status[rhs] = 4;
  }
}

// dirs: X += sum_i omega_i alpha^i p^i; p^i = zeta^i r + beta^i p^i; p, p~ updates.
// FP64 kernels accumulate X term by term in double. FP32 kernels sum the iteration's terms
// over the shifts in float-float and add that sum to the FP64 X once (the FP64 pipe is 1/64 of
// the FP32 rate); with per-shift solutions kept (refinement), x^(i) is held in float-float
// (re hi, re lo, im hi, im lo: the 16 bytes of a complex double) during the pass, so the
// increments alpha^i p^i need no FP64 arithmetic; it is converted to FP64 in place afterwards.
// XS: per-shift solutions kept (v.xs set), a compile-time choice so that neither path's
// instructions are issued predicated-off in the other (predicated-off FP64 instructions still hold
// the FP64 pipe).
template <class R, bool XS>
__global__ void __launch_bounds__(kVecBlock) k_ms_dirs(Geom g, MsDev ms, MsVecs v) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  const int st = ms.status[rhs];
  if (st != 0 && st != 4) return;
  const size_t n = (size_t)12 * g.vol;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // one vector element per thread
  // the shift coefficients in the kernel's own precision (FP32 kernels convert them once per
  // block here, not per element: a double -> float conversion runs on the FP64 pipe)
  using T2 = typename V2<R>::T;
  __shared__ T2 coefx[kMaxShifts], coefz[kMaxShifts], coefb[kMaxShifts], coefa[kMaxShifts];
  __shared__ int act[kMaxShifts];
  for (int i = threadIdx.x; i < ms.s; i += blockDim.x) {
    const size_t si = (size_t)rhs * ms.s + i;
    act[i] = ms.active[si];
    const zd ai = ldc<double>(ms.ash, si);
    const double2 z = ms.zeta[si * 3 + 1], b = ms.bsh[si];  // zeta_{k+1} after the rotation in update
    coefa[i].x = (R)ai.re;
    coefa[i].y = (R)ai.im;
    coefx[i].x = (R)(ms.omega[i] * ai.re);
    coefx[i].y = (R)(ms.omega[i] * ai.im);
    coefz[i].x = (R)z.x;
    coefz[i].y = (R)z.y;
    coefb[i].x = (R)b.x;
    coefb[i].y = (R)b.y;
  }
  __syncthreads();
  R bkr[2];
  scalars_in<R, 2>((const double*)(ms.seed + (size_t)rhs * 8 + 5), bkr);
  if (e >= n) return;
  const cplx<R> b = mk<R>(bkr[0], bkr[1]), bc = mk<R>(bkr[0], -bkr[1]);
  const T* r = (const T*)v.r + voff<R>(rhs, n);
  const T* rt = (const T*)v.rt + voff<R>(rhs, n);
  T* p = (T*)v.p + voff<R>(rhs, n);
  T* pt = (T*)v.pt + voff<R>(rhs, n);
  T* ps = (T*)v.ps + (size_t)rhs * ms.s * n;
  double2* X = v.X + voff<R>(rhs, n);
  {
    const cplx<R> rv = ldc<R>(r, e);
    zd xa = XS ? mk(0.0, 0.0) : ldc<double>(X, e);  // X is not used when x^(i) are kept
    Red<R> sre, sim;  // FP32: this iteration's sum over the shifts
    for (int i = 0; i < ms.s; ++i) {
      if (!act[i]) continue;
      T* pi = ps + (size_t)i * n;
      const cplx<R> pv = ldc<R>(pi, e);
      if constexpr (XS) {  // keep x^(i) itself: x^(i) += alpha^i p^i
        const T2 ca = coefa[i];
        if constexpr (sizeof(R) == 8) {
          double2* xi = v.xs + ((size_t)rhs * ms.s + i) * n;
          stc<double>(xi, e, ldc<double>(xi, e) + mk(ca.x, ca.y) * pv);
        } else {
          float4* xi = reinterpret_cast<float4*>(v.xs + ((size_t)rhs * ms.s + i) * n);
          const cplx<R> inc = mk<R>(ca.x, ca.y) * pv;
          float4 x4 = xi[e];
          const FF re = ff_add(FF{x4.x, x4.y}, FF{inc.re, 0.f}), im = ff_add(FF{x4.z, x4.w}, FF{inc.im, 0.f});
          xi[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
      } else {
        const T2 cx = coefx[i];
        if constexpr (sizeof(R) == 8) {
          xa = xa + mk(cx.x, cx.y) * pv;
        } else {
          const cplx<R> c = mk<R>(cx.x, cx.y);
          sre.add(fma(c.re, pv.re, -(c.im * pv.im)));
          sim.add(fma(c.re, pv.im, c.im * pv.re));
        }
      }
      if (act[i] == 1) {
        const T2 cz = coefz[i], cb = coefb[i];
        cplx<R> nv = mk<R>(cz.x, cz.y) * rv + mk<R>(cb.x, cb.y) * pv;
        stc<R>(pi, e, nv);
      }
    }
    if constexpr (!XS) {
      if constexpr (sizeof(R) == 4) {
        xa.re += sre.get();
        xa.im += sim.get();
      }
      stc<double>(X, e, xa);
    }
    if (st == 0) {
      stc<R>(p, e, rv + b * ldc<R>(p, e));
      stc<R>(pt, e, ldc<R>(rt, e) + bc * ldc<R>(pt, e));
    }
  }
}

cudaError_t launch_ms_start(const Geom& g, bool f64, const MsDev& ms, const MsVecs& v, const double2* b, int m,
                            const double2* R, const double2* L, const double* lam_sign, double2* dots, cudaStream_t st) {
  dim3 grid((g.vol + kBlock - 1) / kBlock, ms.nrhs);
  if (m > 0) {
    cudaError_t e = launch_defl_dots(g, ms.nrhs, m, b, R, L, ms.part, ms.count, dots, st);
    if (e != cudaSuccess) return e;
  }
  if (f64)
    k_ms_start<double><<<grid, kBlock, 0, st>>>(g, ms, v, b, m, R, L, lam_sign, dots);
  else
    k_ms_start<float><<<grid, kBlock, 0, st>>>(g, ms, v, b, m, R, L, lam_sign, dots);
  return cudaGetLastError();
}

bool ms_pair_split(const Geom& g, int key) {
  const int tv = tuned_pair_variant(g.vol, key);
  return tv < 0 ? use_split(g) : (tv == 1 || tv == 4 || tv == 5);  // 0, 2, 3, 6, 7, 8: one thread per site
}

template <class R, int LF>
static cudaError_t ms_step_t(const Geom& g, const Links& U, double m_w, double mu, const MsDev& ms, const MsVecs& v,
                             cudaStream_t st, cudaEvent_t* ev) {
  dim3 grid(vec_blocks(g), ms.nrhs);
  dim3 pgrid((g.vol + kPairSites - 1) / kPairSites, ms.nrhs), pblock(kPairSites, 2);
  HopCoef<R> cp = hop_coef<R>(m_w, mu), cm = hop_coef<R>(m_w, -mu);
  dim3 sgrid((g.vol + kSplitSites - 1) / kSplitSites, ms.nrhs), sblock(kSplitSites, 8);
  const bool split = ms_pair_split(g, sizeof(R) == 8 ? 0 : LF);
  const int elt = vec_elts(g, ms.nrhs, sizeof(R) == 8);
  cudaError_t e;
  if (ev && (e = record_timing(ev[0], st))) return e;
  e = split ? launch_plain(k_ms_pair_split<R, LF, 0>, sgrid, sblock, st, g, U, cp, cm, ms, v)
            : launch_plain(k_ms_pair<R, LF, 0>, pgrid, pblock, st, g, U, cp, cm, ms, v);
  if (e) return e;
  if (ev && (e = record_timing(ev[1], st))) return e;
  e = split ? launch_plain(k_ms_pair_split<R, LF, 1>, sgrid, sblock, st, g, U, cp, cm, ms, v)
            : launch_plain(k_ms_pair<R, LF, 1>, pgrid, pblock, st, g, U, cp, cm, ms, v);
  if (e) return e;
  if ((e = launch_plain(k_ms_update<R>, dim3(vec_blocks(g, elt), ms.nrhs), dim3(kVecBlock), st, g, ms, v, elt))) return e;
  if (ev && (e = record_timing(ev[2], st))) return e;
  if ((e = v.xs ? launch_plain(k_ms_dirs<R, true>, grid, dim3(kVecBlock), st, g, ms, v)
                : launch_plain(k_ms_dirs<R, false>, grid, dim3(kVecBlock), st, g, ms, v)))
    return e;
  if (ev && (e = record_timing(ev[3], st))) return e;
  return cudaGetLastError();
}

cudaError_t launch_ms_step(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu, const MsDev& ms,
                           const MsVecs& v, cudaStream_t st, cudaEvent_t* ev) {
  if (f64) return ms_step_t<double, LINK_F64>(g, U, m_w, mu, ms, v, st, ev);
  if (lf == LINK_F16R12) return ms_step_t<float, LINK_F16R12>(g, U, m_w, mu, ms, v, st, ev);
  return ms_step_t<float, LINK_F32>(g, U, m_w, mu, ms, v, st, ev);
}

__global__ void __launch_bounds__(kVecBlock) k_ms_residual_batch(int vol, int j0, int s, const double2* r64,
                                                                 const double2* t2, const double2* x,
                                                                 const double* sigma, double2* res, double* part,
                                                                 unsigned* count, double* out) {
  const size_t n = (size_t)12 * vol;
  const int j = blockIdx.y, jj = j0 + j, rhs = jj / s, i = jj % s;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0};
  if (e < n) {
    const size_t o = (size_t)j * n + e;
    zd a = ldc<double>(r64, (size_t)rhs * n + e) - (ldc<double>(t2, o) - sigma[i] * ldc<double>(x, o));
    stc<double>(res, o, a);
    acc[0] = norm2(a);
  }
  block_sum<1>(acc);
  if (publish_partials<1>(acc, part + (size_t)j * gridDim.x, count + j)) {
    reduce_partials<1>(part + (size_t)j * gridDim.x, gridDim.x, acc);
    if (lin_tid() == 0) out[j] = acc[0];
  }
}

cudaError_t launch_ms_residual_batch(const Geom& g, int j0, int gn, int s, const double2* r64, const double2* t2,
                                     const double2* x, const double* sigma, double2* res, double* part,
                                     unsigned* count, double* out, cudaStream_t st) {
  dim3 grid(vec_blocks(g), gn);
  k_ms_residual_batch<<<grid, kVecBlock, 0, st>>>(g.vol, j0, s, r64, t2, x, sigma, res, part, count, out);
  return cudaGetLastError();
}

__global__ void k_axpy_f64_masked(size_t n, const int* status, const double2* e, double2* x) {
  const int j = blockIdx.y;
  if (status[j] == 1) return;  // breakdown of this correction solve: keep x_j
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) stc<double>(x, (size_t)j * n + i, ldc<double>(x, (size_t)j * n + i) + ldc<double>(e, (size_t)j * n + i));
}

cudaError_t launch_axpy_f64_masked(const Geom& g, int gn, const int* status, const double2* e, double2* x,
                                   cudaStream_t st) {
  size_t n = (size_t)12 * g.vol;
  dim3 grid((unsigned)((n + 255) / 256), gn);
  k_axpy_f64_masked<<<grid, 256, 0, st>>>(n, status, e, x);
  return cudaGetLastError();
}

// Float-float complex (re hi, re lo, im hi, im lo) -> complex double, in place.
__global__ void k_ff_to_f64(size_t n, double2* x) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 f = reinterpret_cast<const float4*>(x)[i];
  x[i] = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w);
}

cudaError_t launch_ff_to_f64(size_t n, double2* x, cudaStream_t st) {
  k_ff_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x);
  return cudaGetLastError();
}

__global__ void k_ms_combine_shifts(size_t n, int s, const double* omega, const double2* xs, double2* X) {
  const int rhs = blockIdx.y;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  zd a = mk(0.0, 0.0);
  for (int j = 0; j < s; ++j) a = a + omega[j] * ldc<double>(xs, ((size_t)rhs * s + j) * n + i);
  stc<double>(X, (size_t)rhs * n + i, a);
}

cudaError_t launch_ms_combine_shifts(const Geom& g, int nrhs, int s, const double* omega, const double2* xs,
                                     double2* X, cudaStream_t st) {
  size_t n = (size_t)12 * g.vol;
  dim3 grid((unsigned)((n + 255) / 256), nrhs);
  k_ms_combine_shifts<<<grid, 256, 0, st>>>(n, s, omega, xs, X);
  return cudaGetLastError();
}

__global__ void k_ms_finish(int vol, const double2* ax, const double2* xp, double2* x) {
  const size_t n = (size_t)12 * vol;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (e >= n) return;
  zd a = ldc<double>(ax, (size_t)rhs * n + e);
  if (xp) a = a + ldc<double>(xp, (size_t)rhs * n + e);
  int c = (int)(e / vol), s = (int)(e % vol);
  x[(size_t)rhs * n + (size_t)s * 12 + c] = make_double2(a.re, a.im);
}

cudaError_t launch_ms_finish(const Geom& g, int nrhs, const double2* ax, const double2* xp, double2* x, cudaStream_t st) {
  size_t n = (size_t)12 * g.vol;
  dim3 grid((unsigned)((n + 255) / 256), nrhs);
  k_ms_finish<<<grid, 256, 0, st>>>(g.vol, ax, xp, x);
  return cudaGetLastError();
}

}  // namespace ovl
