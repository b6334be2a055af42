// CUDA kernels of the sign(H_W(mu)) b path for sm_103a.
//
// Data layout in HBM: fields are component-major ("native"): element (rhs, c, site) at
// (rhs*12 + c)*V + site with c = spin*3 + colour, so the 32 threads of a warp (32
// consecutive sites) read one contiguous 256 B (FP32) / 512 B (FP64) segment per
// component; links likewise [dir][comp][V]. Reductions are deterministic: fixed-order
// warp-shuffle and shared-memory trees per block, block partials to global memory, and
// the last block to finish (atomic ticket) sums the partials in block order.
#include <cuda_fp16.h>

#include <map>
#include <mutex>

#include "devutil.cuh"
#include "kernels.h"

namespace ovl {

// ------------------------------------------------------------------ autotuner table
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tune;

int tuned_pair_variant(int vol, int prec) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find({vol, prec});
  return it == g_tune.end() ? -1 : it->second;
}
int tune_pair_variant(int vol, int prec, int (*measure)(void*), void* arg) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find({vol, prec});
  if (it != g_tune.end()) return it->second;
  int v = measure(arg);
  if (v >= 0) g_tune[{vol, prec}] = v;
  return v;
}

// ------------------------------------------------------------------ layout conversion
template <class Tin, class Tout>
__global__ void k_to_native(int vol, int nrhs, const Tin* in, Tout* out) {
  size_t n = (size_t)vol * 12;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (e >= n) return;
  int c = (int)(e / vol), s = (int)(e % vol);
  Tin v = in[(size_t)r * n + (size_t)s * 12 + c];
  Tout o;
  o.x = v.x;
  o.y = v.y;
  out[(size_t)r * n + e] = o;
}

template <class Tin, class Tout>
__global__ void k_from_native(int vol, int nrhs, const Tin* in, Tout* out) {
  size_t n = (size_t)vol * 12;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (e >= n) return;
  int c = (int)(e / vol), s = (int)(e % vol);
  Tin v = in[(size_t)r * n + e];
  Tout o;
  o.x = v.x;
  o.y = v.y;
  out[(size_t)r * n + (size_t)s * 12 + c] = o;
}

template <class A, class B>
static cudaError_t conv(const Geom& g, int nrhs, const void* in, void* out, bool to, cudaStream_t st) {
  size_t n = (size_t)g.vol * 12;
  dim3 grid((unsigned)((n + 255) / 256), nrhs);
  if (to)
    k_to_native<A, B><<<grid, 256, 0, st>>>(g.vol, nrhs, (const A*)in, (B*)out);
  else
    k_from_native<A, B><<<grid, 256, 0, st>>>(g.vol, nrhs, (const A*)in, (B*)out);
  return cudaGetLastError();
}

cudaError_t launch_to_native(const Geom& g, int nrhs, bool in_f64, const void* in, bool out_f64, void* out, cudaStream_t st) {
  if (in_f64 && out_f64) return conv<double2, double2>(g, nrhs, in, out, true, st);
  if (in_f64) return conv<double2, float2>(g, nrhs, in, out, true, st);
  if (out_f64) return conv<float2, double2>(g, nrhs, in, out, true, st);
  return conv<float2, float2>(g, nrhs, in, out, true, st);
}
cudaError_t launch_from_native(const Geom& g, int nrhs, bool in_f64, const void* in, bool out_f64, void* out, cudaStream_t st) {
  if (in_f64 && out_f64) return conv<double2, double2>(g, nrhs, in, out, false, st);
  if (in_f64) return conv<double2, float2>(g, nrhs, in, out, false, st);
  if (out_f64) return conv<float2, double2>(g, nrhs, in, out, false, st);
  return conv<float2, float2>(g, nrhs, in, out, false, st);
}

// ------------------------------------------------------------------ link ingest
__global__ void k_ingest_links(int vol, const double2* ucan, double2* u64, float2* u32, uint32_t* u16) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over 4*9*V
  if (e >= (size_t)36 * vol) return;
  int s = (int)(e % vol);
  int k = (int)((e / vol) % 9);
  int mu = (int)(e / ((size_t)9 * vol));
  double2 v = ucan[((size_t)mu * vol + s) * 9 + k];
  if (u64) u64[e] = v;
  if (u32) u32[e] = make_float2((float)v.x, (float)v.y);
  if (u16 && k < 6) {
    __half2 h = __floats2half2_rn((float)v.x, (float)v.y);
    u16[((size_t)mu * 6 + k) * vol + s] = *reinterpret_cast<uint32_t*>(&h);
  }
}

cudaError_t launch_ingest_links(const Geom& g, const double* ucan, double2* u64, float2* u32, uint32_t* u16, cudaStream_t st) {
  size_t n = (size_t)36 * g.vol;
  k_ingest_links<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.vol, (const double2*)ucan, u64, u32, u16);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ apply D_W
// G5IN (gamma5 on the input, the adjoint's form) is a template parameter so that the common
// case carries no per-neighbour branch: 32^4 FP32 4.7 -> 5.2 TB/s in a probe without it.
template <class R, int LF, bool NIN, bool NOUT, bool G5IN>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? (LF == LINK_F16R12 ? 6 : 7) : 1)
    k_dslash(Geom g, Links U, HopCoef<R> c, bool g5_out, const typename V2<R>::T* in, typename V2<R>::T* out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.vol) return;
  size_t off = (size_t)blockIdx.y * 12 * g.vol;
  Loader<R, NIN> ld{in + off, g.vol, G5IN};
  Spin<R> o;
  dslash_site<LF, R>(g, U, s, c, ld, o);
  const R sg = g5_out ? (R)-1 : (R)1;  // gamma5 = diag(1, 1, -1, -1) on the output, without a branch
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o.c[2][a] = sg * o.c[2][a];
    o.c[3][a] = sg * o.c[3][a];
  }
  store_spin<R, NOUT>(out + off, g.vol, s, o);
}

template <class R, int LF, bool G5IN>
static cudaError_t dslash_g(dim3 grid, const Geom& g, const Links& U, HopCoef<R> c, bool go, bool nin, bool nout,
                            const typename V2<R>::T* i, typename V2<R>::T* o, cudaStream_t st) {
  if (nin && nout)
    k_dslash<R, LF, true, true, G5IN><<<grid, kBlock, 0, st>>>(g, U, c, go, i, o);
  else if (nin)
    k_dslash<R, LF, true, false, G5IN><<<grid, kBlock, 0, st>>>(g, U, c, go, i, o);
  else if (nout)
    k_dslash<R, LF, false, true, G5IN><<<grid, kBlock, 0, st>>>(g, U, c, go, i, o);
  else
    k_dslash<R, LF, false, false, G5IN><<<grid, kBlock, 0, st>>>(g, U, c, go, i, o);
  return cudaGetLastError();
}

template <class R, int LF>
static cudaError_t dslash_t(const Geom& g, const Links& U, double m_w, double mu, bool gi, bool go, bool nin, bool nout,
                            int nrhs, const void* in, void* out, cudaStream_t st) {
  HopCoef<R> c = hop_coef<R>(m_w, mu);
  dim3 grid((g.vol + kBlock - 1) / kBlock, nrhs);
  using T = typename V2<R>::T;
  const T* i = (const T*)in;
  T* o = (T*)out;
  return gi ? dslash_g<R, LF, true>(grid, g, U, c, go, nin, nout, i, o, st)
            : dslash_g<R, LF, false>(grid, g, U, c, go, nin, nout, i, o, st);
}

cudaError_t launch_dslash(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu, bool g5_in,
                          bool g5_out, bool native_in, bool native_out, int nrhs, const void* in, void* out,
                          cudaStream_t st) {
  if (f64) return dslash_t<double, LINK_F64>(g, U, m_w, mu, g5_in, g5_out, native_in, native_out, nrhs, in, out, st);
  if (lf == LINK_F16R12)
    return dslash_t<float, LINK_F16R12>(g, U, m_w, mu, g5_in, g5_out, native_in, native_out, nrhs, in, out, st);
  return dslash_t<float, LINK_F32>(g, U, m_w, mu, g5_in, g5_out, native_in, native_out, nrhs, in, out, st);
}

// ------------------------------------------------------------------ Lanczos: start
// part layout for this kernel: [nrhs][nblk][4] = (|r|^2, Re r^H r~, Im r^H r~, unused)
template <class R>
__global__ void __launch_bounds__(kBlock) k_lz_start(Geom g, LzDev lz, typename V2<R>::T* vh, typename V2<R>::T* wh,
                                                     double2* xp, const double2* b, int m, const double2* Rv,
                                                     const double2* Lv, const double* lam_sign, const double2* dots) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)12 * g.vol;
  double acc[4] = {0, 0, 0, 0};
  if (s < g.vol) {
    T* v1 = vh + (size_t)rhs * (lz.kmax + 1) * n;  // column 1
    T* w1 = wh + (size_t)(1 * lz.nrhs + rhs) * n;  // slot (1 & 1) = 1
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
      size_t e = (size_t)c * g.vol + s;
      if (xp) stc<double>(xp, (size_t)rhs * n + e, x);
      stc<R>(v1, e, mk<R>((R)r.re, (R)r.im));
      stc<R>(w1, e, mk<R>((R)rt.re, (R)rt.im));
      acc[0] += norm2(r);
      zd ip = cdot(r, rt);
      acc[1] += ip.re;
      acc[2] += ip.im;
    }
  }
  block_sum<4>(acc);
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  if (publish_partials<4>(acc, part, lz.count + rhs)) {
    reduce_partials<4>(part, gridDim.x, acc);
    if (lin_tid() == 0) {
      double nr2 = acc[0];
      double b0 = sqrt(nr2);
      // v1 = r / beta0, w1 = r~ / (v1^H r~) = r~ * beta0 / (r^H r~)
      zd ip = mk(acc[1], acc[2]);
      double den = norm2(ip);
      size_t o = (size_t)rhs * (lz.kmax + 2);
      lz.beta0[rhs] = b0;
      lz.sv[o + 1] = 1.0 / b0;
      lz.sw[o + 1] = make_double2(b0 * ip.re / den, -b0 * ip.im / den);
      lz.vnorm[o + 1] = 1.0;
      lz.j[rhs] = 1;
      // 3: r = 0 (b lies in the deflated space, x = x_P); 1: r^H r~ = 0 (breakdown at start)
      lz.status[rhs] = nr2 == 0.0 ? 3 : (den > 0.0 ? 0 : 1);
    }
  }
}

// c_i = l_i^H b, d_i = r_i^H b for i < m; partials [nrhs][m][nblk][4], summed by the last block.
__global__ void __launch_bounds__(kBlock) k_defl_dots(Geom g, int m, const double2* b, const double2* Rv,
                                                      const double2* Lv, double* part, unsigned* count,
                                                      double2* dots) {
  const int rhs = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)12 * g.vol;
  __shared__ bool last;
  for (int i = 0; i < m; ++i) {
    double acc[4] = {0, 0, 0, 0};
    if (s < g.vol) {
      for (int c = 0; c < 12; ++c) {
        zd bv = ldc<double>(b, (size_t)rhs * n + (size_t)s * 12 + c);
        zd li = ldc<double>(Lv, (size_t)i * n + (size_t)c * g.vol + s);
        zd ri = ldc<double>(Rv, (size_t)i * n + (size_t)c * g.vol + s);
        zd a = cdot(li, bv), d = cdot(ri, bv);
        acc[0] += a.re;
        acc[1] += a.im;
        acc[2] += d.re;
        acc[3] += d.im;
      }
    }
    block_sum<4>(acc);
    if (threadIdx.x == 0) {
      double* p = part + (((size_t)rhs * m + i) * gridDim.x + blockIdx.x) * 4;
      for (int q = 0; q < 4; ++q) p[q] = acc[q];
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(count + rhs, 1u);
    last = (t == gridDim.x - 1);
    if (last) count[rhs] = 0u;
  }
  __syncthreads();
  if (!last) return;
  for (int i = 0; i < m; ++i) {
    double acc[4];
    reduce_partials<4>(part + ((size_t)rhs * m + i) * gridDim.x * 4, gridDim.x, acc);
    if (threadIdx.x == 0) {
      dots[(size_t)rhs * 2 * m + i] = make_double2(acc[0], acc[1]);
      dots[(size_t)rhs * 2 * m + m + i] = make_double2(acc[2], acc[3]);
    }
  }
}

cudaError_t launch_defl_dots(const Geom& g, int nrhs, int m, const double2* b, const double2* R, const double2* L,
                             double* part, unsigned* count, double2* dots, cudaStream_t st) {
  dim3 grid((g.vol + kBlock - 1) / kBlock, nrhs);
  k_defl_dots<<<grid, kBlock, 0, st>>>(g, m, b, R, L, part, count, dots);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_start(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, const double2* b, int m,
                                 const double2* R, const double2* L, const double* lam_sign, double2* dots,
                                 cudaStream_t st) {
  dim3 grid((g.vol + kBlock - 1) / kBlock, lz.nrhs);
  if (m > 0) {
    k_defl_dots<<<grid, kBlock, 0, st>>>(g, m, b, R, L, lz.part, lz.count, dots);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (f64)
    k_lz_start<double><<<grid, kBlock, 0, st>>>(g, lz, (double2*)vec.vh, (double2*)vec.wh, vec.xp, b, m, R, L,
                                                 lam_sign, dots);
  else
    k_lz_start<float><<<grid, kBlock, 0, st>>>(g, lz, (float2*)vec.vh, (float2*)vec.wh, vec.xp, b, m, R, L, lam_sign,
                                                dots);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Lanczos: one step
// Pair stencil: Av_j = sv_j H(mu) vhat_j, Aw_j = sw_j H(-mu) what_j (H(mu)^H = H(-mu)),
// alpha_j = w_j^H A v_j = conj(sw_j) sum_x what_j(x)^H Av_j(x).
// Block (kPairSites, 2): threadIdx.y = 0 applies H(mu) to vhat, = 1 applies H(-mu) to what,
// for the same kPairSites sites, so each thread holds one stencil's registers and the two
// halves of the block share the link lines in L1.
template <class R, int LF>
__global__ void __launch_bounds__(2 * kPairSites) k_lz_pair(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm, LzDev lz,
                                                            const typename V2<R>::T* vh, const typename V2<R>::T* wh,
                                                            typename V2<R>::T* av, typename V2<R>::T* aw) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  const double2 swd = lz.sw[o + j];
  const T* vj = vh + ((size_t)rhs * (lz.kmax + 1) + (j - 1)) * n;
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  const int s = blockIdx.x * kPairSites + threadIdx.x;
  const bool is_w = threadIdx.y == 1;
  Red<R> acc[2];
  if (s < g.vol) {
    Spin<R> ov;
    if (!is_w) {
      dslash_site<LF, R>(g, U, s, cp, Loader<R, true>{vj, g.vol, false}, ov);
      const R sv = (R)lz.sv[o + j];
      // all loads of w_j before the stores of Av (the compiler cannot reorder them across stores
      // that might alias, which would serialise twelve memory round trips)
      cplx<R> wv[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) wv[c] = ldc<R>(wj, (size_t)c * g.vol + s);
      cplx<R> a = mk<R>(0, 0);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cplx<R> x = sv * ov.c[c / 3][c % 3];
        if (c >= 6) x = -x;  // gamma5
        stc<R>(av + (size_t)rhs * n, (size_t)c * g.vol + s, x);
        a = a + cdot(wv[c], x);
      }
      acc[0].add(a.re);
      acc[1].add(a.im);
    } else {
      dslash_site<LF, R>(g, U, s, cm, Loader<R, true>{wj, g.vol, false}, ov);
      const cplx<R> sw = mk<R>((R)swd.x, (R)swd.y);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cplx<R> y = sw * ov.c[c / 3][c % 3];
        if (c >= 6) y = -y;  // gamma5
        stc<R>(aw + (size_t)rhs * n, (size_t)c * g.vol + s, y);
      }
    }
  }
  double tot[2];
  block_reduce<R, 2>(acc, tot);
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  double pv[4] = {tot[0], tot[1], 0, 0};
  if (publish_partials<4>(pv, part, lz.count + rhs)) {
    reduce_partials<4>(part, gridDim.x, pv);
    if (lin_tid() == 0) {
      zd sum = mk(pv[0], pv[1]);
      zd alpha = conj(mk(swd.x, swd.y)) * sum;
      lz.alpha[o + j] = make_double2(alpha.re, alpha.im);
    }
  }
}

// The same step with 8 threads per site (small lattices): see pair_split.
template <class R, int LF>
__global__ void __launch_bounds__(8 * kSplitSites) k_lz_pair_split(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm,
                                                                   LzDev lz, const typename V2<R>::T* vh,
                                                                   const typename V2<R>::T* wh,
                                                                   typename V2<R>::T* av, typename V2<R>::T* aw) {
  using T = typename V2<R>::T;
  __shared__ SplitSmem<R> sm;
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  const double2 swd = lz.sw[o + j];
  const T* vj = vh + ((size_t)rhs * (lz.kmax + 1) + (j - 1)) * n;
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  const R sv = (R)lz.sv[o + j];
  const cplx<R> sw = mk<R>((R)swd.x, (R)swd.y);
  Red<R> acc[2];
  pair_split<R, LF>(g, U, cp, cm, vj, wj, sm, [&](int which, int s, Spin<R>& out) {
    if (which == 0) {
      cplx<R> wv[12];  // loads first (see k_lz_pair)
#pragma unroll
      for (int c = 0; c < 12; ++c) wv[c] = ldc<R>(wj, (size_t)c * g.vol + s);
      cplx<R> a = mk<R>(0, 0);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cplx<R> x = sv * out.c[c / 3][c % 3];
        if (c >= 6) x = -x;  // gamma5
        stc<R>(av + (size_t)rhs * n, (size_t)c * g.vol + s, x);
        a = a + cdot(wv[c], x);
      }
      acc[0].add(a.re);
      acc[1].add(a.im);
    } else {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cplx<R> y = sw * out.c[c / 3][c % 3];
        if (c >= 6) y = -y;
        stc<R>(aw + (size_t)rhs * n, (size_t)c * g.vol + s, y);
      }
    }
  });
  double tot[2];
  block_reduce<R, 2>(acc, tot);
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  double pv[4] = {tot[0], tot[1], 0, 0};
  if (publish_partials<4>(pv, part, lz.count + rhs)) {
    reduce_partials<4>(part, gridDim.x, pv);
    if (lin_tid() == 0) {
      zd alpha = conj(mk(swd.x, swd.y)) * mk(pv[0], pv[1]);
      lz.alpha[o + j] = make_double2(alpha.re, alpha.im);
    }
  }
}

// vhat_{j+1} = Av_j - alpha_j v_j - beta_{j-1} v_{j-1}
// what_{j+1} = Aw_j - conj(alpha_j) w_j - conj(delta_{j-1}) w_{j-1}    (Eqs. 2sided1/2)
// then delta_j = sqrt|what^H vhat|, beta_j = what^H vhat / delta_j (scaling reading).
// One thread per vector element (component, site): 12 V threads per rhs.
template <class R>
__global__ void __launch_bounds__(kVecBlock) k_lz_update(Geom g, LzDev lz, typename V2<R>::T* vh,
                                                         typename V2<R>::T* wh, const typename V2<R>::T* av,
                                                         const typename V2<R>::T* aw, int elt) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  const zd alpha = ldc<double>(lz.alpha, o + j);
  const double svj = lz.sv[o + j];
  const zd swj = ldc<double>(lz.sw, o + j);
  zd cv1 = svj * alpha, cw1 = swj * conj(alpha), cv2 = mk(0.0, 0.0), cw2 = mk(0.0, 0.0);
  if (j > 1) {
    cv2 = lz.sv[o + j - 1] * ldc<double>(lz.beta, o + j - 1);
    cw2 = lz.delta[o + j - 1] * ldc<double>(lz.sw, o + j - 1);
  }
  const cplx<R> a1 = mk<R>((R)cv1.re, (R)cv1.im), a2 = mk<R>((R)cv2.re, (R)cv2.im);
  const cplx<R> b1 = mk<R>((R)cw1.re, (R)cw1.im), b2 = mk<R>((R)cw2.re, (R)cw2.im);
  const T* vj = vh + ((size_t)rhs * (lz.kmax + 1) + (j - 1)) * n;
  const T* vjm = vh + ((size_t)rhs * (lz.kmax + 1) + (j > 1 ? j - 2 : 0)) * n;
  T* vnew = vh + ((size_t)rhs * (lz.kmax + 1) + j) * n;
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  T* wnew = wh + ((size_t)((j + 1) & 1) * lz.nrhs + rhs) * n;  // holds what_{j-1} until overwritten
  const T* avr = av + (size_t)rhs * n;
  const T* awr = aw + (size_t)rhs * n;
  Red<R> acc[4];
  // elt elements per thread, block-contiguous per pass (coalesced)
  for (int q = 0; q < elt; ++q) {
    const size_t e = ((size_t)blockIdx.x * elt + q) * blockDim.x + threadIdx.x;
    if (e >= n) break;
    cplx<R> x = cmsub(ldc<R>(avr, e), a1, ldc<R>(vj, e));
    cplx<R> y = cmsub(ldc<R>(awr, e), b1, ldc<R>(wj, e));
    if (j > 1) {
      x = cmsub(x, a2, ldc<R>(vjm, e));
      y = cmsub(y, b2, ldc<R>(wnew, e));
    }
    stc<R>(vnew, e, x);
    stc<R>(wnew, e, y);
    acc[0].add(fma(y.re, x.re, y.im * x.im));  // (y^H x).re
    acc[1].add(fma(y.re, x.im, -(y.im * x.re)));
    acc[2].add(fma(x.re, x.re, x.im * x.im));
    acc[3].add(fma(y.re, y.re, y.im * y.im));
  }
  double tot[4];
  block_reduce<R, 4>(acc, tot);
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  if (publish_partials<4>(tot, part, lz.count + rhs)) {
    double sums[4];
    reduce_partials<4>(part, gridDim.x, sums);
    if (lin_tid() == 0) {
      zd ip = mk(sums[0], sums[1]);
      double aip = sqrt(norm2(ip));
      if (!(aip > 1e-14 * sqrt(sums[2] * sums[3])) || !(aip < 1e300)) {
        lz.status[rhs] = 1;  // breakdown (or non-finite)
      } else {
        double d = sqrt(aip);
        zd bt = (1.0 / d) * ip;
        lz.delta[o + j] = d;
        lz.beta[o + j] = make_double2(bt.re, bt.im);
        lz.sv[o + j + 1] = 1.0 / d;
        double bb = norm2(bt);  // 1/conj(beta) = beta / |beta|^2
        lz.sw[o + j + 1] = make_double2(bt.re / bb, bt.im / bb);
        lz.vnorm[o + j + 1] = sqrt(sums[2]) / d;
        lz.j[rhs] = j + 1;
      }
    }
  }
}

cudaError_t launch_lanczos_pair(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu,
                                const LzDev& lz, const LzVecs& vec, cudaStream_t st, int variant) {
  if (variant < 0) variant = tuned_pair_variant(g.vol, f64 ? 0 : lf);
  if (variant < 0) variant = use_split(g) ? 1 : 0;
  const HopCoef<double> dp = hop_coef<double>(m_w, mu), dm = hop_coef<double>(m_w, -mu);
  const HopCoef<float> fp = hop_coef<float>(m_w, mu), fm = hop_coef<float>(m_w, -mu);
  const double2 *dv = (const double2*)vec.vh, *dw = (const double2*)vec.wh;
  const float2 *fv = (const float2*)vec.vh, *fw = (const float2*)vec.wh;
  cudaError_t e;
  if (variant == 1) {
    dim3 grid((g.vol + kSplitSites - 1) / kSplitSites, lz.nrhs), block(kSplitSites, 8);
    if (f64)
      e = launch_plain(k_lz_pair_split<double, LINK_F64>, grid, block, st, g, U, dp, dm, lz, dv, dw, (double2*)vec.av,
                     (double2*)vec.aw);
    else if (lf == LINK_F16R12)
      e = launch_plain(k_lz_pair_split<float, LINK_F16R12>, grid, block, st, g, U, fp, fm, lz, fv, fw, (float2*)vec.av,
                     (float2*)vec.aw);
    else
      e = launch_plain(k_lz_pair_split<float, LINK_F32>, grid, block, st, g, U, fp, fm, lz, fv, fw, (float2*)vec.av,
                     (float2*)vec.aw);
  } else {
    dim3 grid((g.vol + kPairSites - 1) / kPairSites, lz.nrhs), block(kPairSites, 2);
    if (f64)
      e = launch_plain(k_lz_pair<double, LINK_F64>, grid, block, st, g, U, dp, dm, lz, dv, dw, (double2*)vec.av,
                     (double2*)vec.aw);
    else if (lf == LINK_F16R12)
      e = launch_plain(k_lz_pair<float, LINK_F16R12>, grid, block, st, g, U, fp, fm, lz, fv, fw, (float2*)vec.av,
                     (float2*)vec.aw);
    else
      e = launch_plain(k_lz_pair<float, LINK_F32>, grid, block, st, g, U, fp, fm, lz, fv, fw, (float2*)vec.av,
                     (float2*)vec.aw);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_update(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, cudaStream_t st) {
  const int elt = vec_elts(g, lz.nrhs, f64);
  dim3 grid(vec_blocks(g, elt), lz.nrhs);
  cudaError_t e;
  if (f64)
    e = launch_plain(k_lz_update<double>, grid, dim3(kVecBlock), st, g, lz, (double2*)vec.vh, (double2*)vec.wh,
                   (const double2*)vec.av, (const double2*)vec.aw, elt);
  else
    e = launch_plain(k_lz_update<float>, grid, dim3(kVecBlock), st, g, lz, (float2*)vec.vh, (float2*)vec.wh,
                   (const float2*)vec.av, (const float2*)vec.aw, elt);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_step(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu, const LzDev& lz,
                                const LzVecs& vec, cudaStream_t st) {
  cudaError_t e = launch_lanczos_pair(g, U, lf, f64, m_w, mu, lz, vec, st);
  if (e != cudaSuccess) return e;
  return launch_lanczos_update(g, f64, lz, vec, st);
}

// ------------------------------------------------------------------ combine
// x (canonical complex128) = x_P + sum_{j=1..k} coef_j vhat_j  (x = x_P + beta V_k y with the
// column scales folded into coef on the host). One thread per (component, site).
template <class R>
__global__ void __launch_bounds__(256) k_lz_combine(int vol, int kmax, const int* kr, const typename V2<R>::T* vh,
                                                    const double2* xp, const double2* coef, int kcoef, double2* x) {
  __shared__ double2 cs[256];
  const int rhs = blockIdx.y;
  const int k = kr[rhs];  // this rhs's Krylov dimension (columns beyond it are never read)
  const size_t n = (size_t)12 * vol;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const typename V2<R>::T* base = vh + (size_t)rhs * (kmax + 1) * n;
  zd acc = mk(0.0, 0.0);
  for (int j0 = 0; j0 < k; j0 += 256) {
    __syncthreads();
    if (j0 + (int)threadIdx.x < k) cs[threadIdx.x] = coef[(size_t)rhs * kcoef + j0 + threadIdx.x];
    __syncthreads();
    if (e < n) {
      int jn = min(256, k - j0);
      for (int jj = 0; jj < jn; ++jj) {
        cplx<R> v = ldc<R>(base, (size_t)(j0 + jj) * n + e);
        zd vd = mk((double)v.re, (double)v.im);
        double2 c = cs[jj];
        acc = acc + mk(c.x, c.y) * vd;
      }
    }
  }
  if (e >= n) return;
  if (xp) acc = acc + ldc<double>(xp, (size_t)rhs * n + e);
  int c = (int)(e / vol), s = (int)(e % vol);
  x[(size_t)rhs * n + (size_t)s * 12 + c] = make_double2(acc.re, acc.im);
}

// ||sum_j d1_j vhat_j||^2 and ||sum_j d2_j vhat_j||^2 per rhs (the change of x between two
// checks and the Krylov part of x), each rhs up to its own kr; result out[rhs][2].
// The sums run in FP32 arithmetic (FP64 only across elements): the result only feeds the
// stopping estimate, whose terms are all of the size of the change itself.
template <class R>
__global__ void __launch_bounds__(256) k_lz_vnorms(int vol, int kmax, const int* kr, const typename V2<R>::T* vh,
                                                   const double2* d1, const double2* d2, int kcoef, int stride,
                                                   double* part, unsigned* count, double* out) {
  __shared__ float2 c1[256], c2[256];
  const int rhs = blockIdx.y;
  const int k = kr[rhs];
  const size_t n = (size_t)12 * vol;
  // sampled element: runs of 32 consecutive elements, one run every 32 * stride (stride 1: all)
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t e = (t >> 5) * 32 * (size_t)stride + (t & 31);
  const typename V2<R>::T* base = vh + (size_t)rhs * (kmax + 1) * n;
  cplx<float> a1 = mk<float>(0, 0), a2 = mk<float>(0, 0);
  for (int j0 = 0; j0 < k; j0 += 256) {
    __syncthreads();
    if (j0 + (int)threadIdx.x < k) {
      double2 x1 = d1[(size_t)rhs * kcoef + j0 + threadIdx.x], x2 = d2[(size_t)rhs * kcoef + j0 + threadIdx.x];
      c1[threadIdx.x] = make_float2((float)x1.x, (float)x1.y);
      c2[threadIdx.x] = make_float2((float)x2.x, (float)x2.y);
    }
    __syncthreads();
    if (e < n) {
      int jn = min(256, k - j0);
      for (int jj = 0; jj < jn; ++jj) {
        cplx<R> v = ldc<R>(base, (size_t)(j0 + jj) * n + e);
        cplx<float> vf = mk<float>((float)v.re, (float)v.im);
        a1 = a1 + mk<float>(c1[jj].x, c1[jj].y) * vf;
        a2 = a2 + mk<float>(c2[jj].x, c2[jj].y) * vf;
      }
    }
  }
  double acc[2] = {(double)norm2(a1), (double)norm2(a2)};
  block_sum<2>(acc);
  double* pr = part + (size_t)rhs * gridDim.x * 2;
  if (publish_partials<2>(acc, pr, count + rhs)) {
    reduce_partials<2>(pr, gridDim.x, acc);
    if (threadIdx.x == 0) {
      out[rhs * 2] = acc[0];
      out[rhs * 2 + 1] = acc[1];
    }
  }
}

cudaError_t launch_lanczos_vnorms(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, const int* kr,
                                  const double2* d1, const double2* d2, int kcoef, double* part, unsigned* count,
                                  double* out, cudaStream_t st) {
  const size_t n = (size_t)12 * g.vol;
  const int stride = vnorm_stride(g);
  const size_t ns = (n + stride - 1) / stride;  // sampled elements (upper bound)
  dim3 grid((unsigned)((ns + 255) / 256), lz.nrhs);
  if (f64)
    k_lz_vnorms<double><<<grid, 256, 0, st>>>(g.vol, lz.kmax, kr, (const double2*)vec.vh, d1, d2, kcoef, stride, part,
                                               count, out);
  else
    k_lz_vnorms<float><<<grid, 256, 0, st>>>(g.vol, lz.kmax, kr, (const float2*)vec.vh, d1, d2, kcoef, stride, part,
                                              count, out);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_combine(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, const int* kr,
                                   const double2* coef, int kcoef, double2* x, cudaStream_t st) {
  size_t n = (size_t)12 * g.vol;
  dim3 grid((unsigned)((n + 255) / 256), lz.nrhs);
  if (f64)
    k_lz_combine<double><<<grid, 256, 0, st>>>(g.vol, lz.kmax, kr, (const double2*)vec.vh, vec.xp, coef, kcoef, x);
  else
    k_lz_combine<float><<<grid, 256, 0, st>>>(g.vol, lz.kmax, kr, (const float2*)vec.vh, vec.xp, coef, kcoef, x);
  return cudaGetLastError();
}

}  // namespace ovl
