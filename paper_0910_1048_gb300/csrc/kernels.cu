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
#include <set>
#include <tuple>

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
void set_pair_variant(int vol, int prec, int variant) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (variant < 0)
    g_tune.erase({vol, prec});
  else
    g_tune[{vol, prec}] = variant;
}

// ------------------------------------------------------------------ one block per SM
// Launch geometry that puts exactly one block of a kernel on every SM: a request for more than half
// of an SM's shared memory (the kernels do not use it) keeps a second block of the same kernel off
// the SM, so a grid of one block per SM is spread evenly whatever order the hardware hands the
// blocks out in. (Left to the hardware, 648 equal blocks of the FP64 pair stencil at 12^4 gave the
// busiest SM 1.3 times the mean SM time.)
struct SmFill {
  int nsm = 0;   // SMs of the current device (0: query failed)
  int smem = 0;  // dynamic shared memory per block that admits one block per SM
};
static std::mutex g_fill_mu;
static SmFill sm_fill(int dev) {
  static std::map<int, SmFill> cache;
  std::lock_guard<std::mutex> lk(g_fill_mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  SmFill r;
  int per_sm = 0;
  if (cudaDeviceGetAttribute(&r.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return SmFill{};
  }
  r.smem = per_sm / 2 + 1024;
  cache[dev] = r;
  return r;
}
// Launch `kern` with one block per SM of the current device (grid (SM count, gy)), after allowing
// it the shared-memory request once per kernel and device.
// early = true: programmatic dependent launch (the blocks may start while the previous kernel of
// the stream runs; the kernel waits for it with griddepcontrol.wait before reading its results).
template <typename... KArgs, typename... Args>
static cudaError_t launch_sm_fill(void (*kern)(KArgs...), int gy, dim3 block, cudaStream_t st, bool early,
                                  Args... args) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const SmFill f = sm_fill(dev);
  if (f.nsm <= 0) return cudaErrorLaunchFailure;
  {
    static std::set<std::pair<const void*, int>> allowed;
    std::lock_guard<std::mutex> lk(g_fill_mu);
    if (!allowed.count({(const void*)kern, dev})) {
      if ((e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, f.smem)))
        return e;
      allowed.insert({(const void*)kern, dev});
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(f.nsm, gy);
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = f.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (early) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, args...);
}
static int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sm_fill(dev).nsm;
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

// The FP32 operator on a batch of sources, native layout in and out. A thread applies the links of
// its site to a group of G sources (each link loaded once per group), and the grid is ordered
// group-fastest (block b: site tile b / ngroups, group b % ngroups), so that the blocks of all
// groups of one site tile run together and a tile's link lines come from DRAM once and from L2
// for the other groups. G = 1 is the single-source kernel in that order.
template <int LF, bool G5IN, int G>
__global__ void __launch_bounds__(kBlock, G == 1 ? 7 : (G == 2 ? 4 : 2))
    k_dslash_group(Geom g, Links U, HopCoef<float> c, bool g5_out, int nrhs,
                                                         const float2* in, float2* out) {
  const int ngroups = (nrhs + G - 1) / G;
  const int tile = blockIdx.x / ngroups, grp = blockIdx.x % ngroups;
  const int s = tile * blockDim.x + threadIdx.x;
  if (s >= g.vol) return;
  const int r0 = grp * G;
  const int nact = min(G, nrhs - r0);
  const size_t n = (size_t)12 * g.vol;
  Loader<float, true> ld[G];
#pragma unroll
  for (int r = 0; r < G; ++r) ld[r] = Loader<float, true>{in + (size_t)(r0 + (r < nact ? r : 0)) * n, g.vol, G5IN};
  Spin<float> o[G];
  dslash_site_g<LF, G>(g, U, s, c, ld, nact, o);
  const float sg = g5_out ? -1.f : 1.f;
#pragma unroll
  for (int r = 0; r < G; ++r) {
    if (r < nact) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        o[r].c[2][a] = sg * o[r].c[2][a];
        o[r].c[3][a] = sg * o[r].c[3][a];
      }
      store_spin<float, true>(out + (size_t)(r0 + r) * n, g.vol, s, o[r]);
    }
  }
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

template <int LF, int G>
static cudaError_t dslash_group_g(const Geom& g, const Links& U, HopCoef<float> c, bool gi, bool go, int nrhs,
                                  const void* in, void* out, cudaStream_t st) {
  const unsigned tiles = (unsigned)((g.vol + kBlock - 1) / kBlock), ngroups = (unsigned)((nrhs + G - 1) / G);
  if (gi)
    k_dslash_group<LF, true, G><<<tiles * ngroups, kBlock, 0, st>>>(g, U, c, go, nrhs, (const float2*)in, (float2*)out);
  else
    k_dslash_group<LF, false, G><<<tiles * ngroups, kBlock, 0, st>>>(g, U, c, go, nrhs, (const float2*)in,
                                                                      (float2*)out);
  return cudaGetLastError();
}

// Sources per link load of the batched stencil (1, 2 or 4), chosen per (volume, links, batch) by
// timing the three on the first call (the real launch follows and rewrites `out`).
static std::mutex g_group_mu;
static std::map<std::tuple<int, int, int>, int> g_group;

template <int LF>
static cudaError_t dslash_group_t(const Geom& g, const Links& U, double m_w, double mu, bool gi, bool go, int nrhs,
                                  const void* in, void* out, cudaStream_t st) {
  const HopCoef<float> c = hop_coef<float>(m_w, mu);
  auto run = [&](int G) {
    return G == 4 ? dslash_group_g<LF, 4>(g, U, c, gi, go, nrhs, in, out, st)
                  : G == 2 ? dslash_group_g<LF, 2>(g, U, c, gi, go, nrhs, in, out, st)
                           : dslash_group_g<LF, 1>(g, U, c, gi, go, nrhs, in, out, st);
  };
  int G = 0;
  {
    std::lock_guard<std::mutex> lk(g_group_mu);
    auto it = g_group.find({g.vol, LF, nrhs});
    if (it != g_group.end()) G = it->second;
    if (!G) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
        float best = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep)
          for (int cand : {1, 2, 4}) {
            ok = ok && cudaEventRecord(a, st) == cudaSuccess && run(cand) == cudaSuccess &&
                 cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess;
            float ms = 0;
            if (ok && rep > 0 && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best) best = ms, G = cand;
          }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (!ok) G = 0;
      }
      cudaGetLastError();
      if (G) g_group[{g.vol, LF, nrhs}] = G;
    }
  }
  return run(G ? G : kLinkGroup);
}

cudaError_t launch_dslash(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu, bool g5_in,
                          bool g5_out, bool native_in, bool native_out, int nrhs, const void* in, void* out,
                          cudaStream_t st) {
  if (f64) return dslash_t<double, LINK_F64>(g, U, m_w, mu, g5_in, g5_out, native_in, native_out, nrhs, in, out, st);
  if (nrhs > 1 && native_in && native_out) {  // a batch: links once per group of sources
    if (lf == LINK_F16R12) return dslash_group_t<LINK_F16R12>(g, U, m_w, mu, g5_in, g5_out, nrhs, in, out, st);
    return dslash_group_t<LINK_F32>(g, U, m_w, mu, g5_in, g5_out, nrhs, in, out, st);
  }
  if (lf == LINK_F16R12)
    return dslash_t<float, LINK_F16R12>(g, U, m_w, mu, g5_in, g5_out, native_in, native_out, nrhs, in, out, st);
  return dslash_t<float, LINK_F32>(g, U, m_w, mu, g5_in, g5_out, native_in, native_out, nrhs, in, out, st);
}

// ------------------------------------------------------------------ Lanczos: start
// Offset of basis column j (1-based) of rhs: slot (j - 1) % vcols (every column with the full
// basis, a rotating window of three in the two-pass mode).
__device__ __forceinline__ size_t vcol(const LzDev& lz, int rhs, int j, size_t n) {
  return ((size_t)rhs * lz.vcols + (size_t)((j - 1) % lz.vcols)) * n;
}

// part layout for this kernel: [nrhs][nblk][4] = (|r|^2, Re r^H r~, Im r^H r~, |r~|^2)
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
    T* v1 = vh + vcol(lz, rhs, 1, n);  // column 1
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
      if (lz.xacc) {  // second pass: x = coef_1 vhat_1 (the stored, rounded vector)
        const cplx<R> s1 = ldc<R>(v1, e);
        stc<double>(lz.xacc, (size_t)rhs * n + e,
                    ldc<double>(lz.xcoef, (size_t)rhs * (lz.kmax + 2) + 1) * mk((double)s1.re, (double)s1.im));
      }
      acc[0] += norm2(r);
      zd ip = cdot(r, rt);
      acc[1] += ip.re;
      acc[2] += ip.im;
      acc[3] += norm2(rt);
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
      // 3: r = 0 (b lies in the deflated space, x = x_P); 1: |r^H r~| <= 1e-14 |r| |r~| (breakdown
      // at the start, the same relative test as every later step; j = 0: no Krylov part, x = x_P)
      const int st = nr2 == 0.0 ? 3 : (sqrt(den) > 1e-14 * sqrt(nr2 * acc[3]) && den < 1e300 ? 0 : 1);
      lz.status[rhs] = st;
      lz.j[rhs] = st == 1 ? 0 : 1;
      lz.pending[rhs] = 0;
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
// Last block of the pair stencil of step j: alpha_j = conj(sw_j) sum what_j^H A vhat_j (pv[0..1],
// the partials of the product with the scaled A v_j), and the coefficients of the update that
// follows, so that its threads only load them:
//   vhat_{j+1} = A v_j - (sv_j alpha_j) vhat_j - (sv_{j-1} beta_{j-1}) vhat_{j-1},
//   what_{j+1} = A^H w_j - (sw_j conj(alpha_j)) what_j - (delta_{j-1} sw_{j-1}) what_{j-1}.
// alpha_j = conj(sw_j) (sum of the partials), and the update coefficients in LzDev::ucoef order.
// The scalars of earlier steps that alpha_j's coefficients need (loaded ahead of the sum).
struct AlphaIn {
  zd sw;   // sw_j
  double sv;  // sv_j
  zd a2, b2;  // sv_{j-1} beta_{j-1}, delta_{j-1} sw_{j-1} (0 at j = 1)
};

__device__ __forceinline__ AlphaIn lz_alpha_inputs(const LzDev& lz, size_t o, int j) {
  AlphaIn in;
  const double2 swd = lz.sw[o + j];
  in.sw = mk(swd.x, swd.y);
  in.sv = lz.sv[o + j];
  in.a2 = in.b2 = mk(0.0, 0.0);
  if (j > 1) {
    in.a2 = lz.sv[o + j - 1] * ldc<double>(lz.beta, o + j - 1);
    in.b2 = lz.delta[o + j - 1] * ldc<double>(lz.sw, o + j - 1);
  }
  return in;
}

__device__ __forceinline__ zd lz_alpha_coeffs(const AlphaIn& in, const double (&pv)[4], double2 (&c)[4]) {
  const zd alpha = conj(in.sw) * mk(pv[0], pv[1]);
  const zd a1 = in.sv * alpha, b1 = in.sw * conj(alpha);
  c[0] = make_double2(a1.re, a1.im);
  c[1] = make_double2(in.a2.re, in.a2.im);
  c[2] = make_double2(b1.re, b1.im);
  c[3] = make_double2(in.b2.re, in.b2.im);
  return alpha;
}

__device__ __forceinline__ zd lz_alpha_coeffs(const LzDev& lz, size_t o, int j, double2 swd, const double (&pv)[4],
                                              double2 (&c)[4]) {
  AlphaIn in = lz_alpha_inputs(lz, o, j);
  in.sw = mk(swd.x, swd.y);
  return lz_alpha_coeffs(in, pv, c);
}

__device__ __forceinline__ void lz_alpha_store(const LzDev& lz, int rhs, size_t o, int j, zd alpha,
                                               const double2 (&c)[4]) {
  lz.alpha[o + j] = make_double2(alpha.re, alpha.im);
  double2* u = lz.ucoef + (size_t)rhs * 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) u[i] = c[i];
}

__device__ __forceinline__ void lz_alpha_finish(const LzDev& lz, int rhs, size_t o, int j, double2 swd,
                                                const double (&pv)[4]) {
  double2 c[4];
  const zd alpha = lz_alpha_coeffs(lz, o, j, swd, pv, c);
  lz_alpha_store(lz, rhs, o, j, alpha, c);
}

struct BetaVals {
  bool ok;    // false: breakdown (or a non-finite value)
  double d;   // delta_j
  double id;  // 1/delta_j = sv_{j+1}
  zd bt;      // beta_j
  zd swv;     // 1/conj(beta_j) = sw_{j+1}
  double vn;  // |v_{j+1}|
};

__device__ __forceinline__ BetaVals lz_beta_vals(const double (&sums)[4]) {
  // few FP64 operations in one dependent chain (each is slow on this GPU's FP64 pipe): with
  // r = |ip|^-1 and id = r^(1/2) = 1/delta_j, delta_j = |ip| id, beta_j = id ip, and
  // 1/conj(beta_j) = beta_j / |beta_j|^2 = id r ip (|beta_j|^2 = |ip|); the breakdown test on squares
  BetaVals b{};
  const zd ip = mk(sums[0], sums[1]);
  const double n2 = norm2(ip);
  b.ok = (n2 > 1e-28 * (sums[2] * sums[3])) && (n2 <= 1.7976931348623157e308);
  if (!b.ok) return b;
  const double r = rsqrt(n2), id = sqrt(r), idp = id * r;
  b.id = id;
  b.d = n2 * r * id;  // |ip| / delta_j = delta_j
  b.bt = id * ip;
  b.swv = mk(idp * ip.re, idp * ip.im);
  b.vn = sqrt(sums[2]) * id;
  return b;
}

// Stores the values of step j (b.ok) or marks the breakdown.
__device__ __forceinline__ void lz_beta_store(const LzDev& lz, int rhs, size_t o, int j, const BetaVals& b) {
  if (!b.ok) {
    lz.status[rhs] = 1;
    return;
  }
  lz.delta[o + j] = b.d;
  lz.beta[o + j] = make_double2(b.bt.re, b.bt.im);
  lz.sv[o + j + 1] = b.id;
  lz.sw[o + j + 1] = make_double2(b.swv.re, b.swv.im);
  lz.vnorm[o + j + 1] = b.vn;
}

// From sums = (what^H vhat re, im, |vhat|^2, |what|^2) of step j: delta_j = sqrt|what^H vhat|,
// beta_j = what^H vhat / delta_j, the next column scales and |v_{j+1}|; j advances. A relative
// breakdown (or a non-finite value) sets status 1 instead.
__device__ __forceinline__ void lz_beta_finish(const LzDev& lz, int rhs, size_t o, int j, const double (&sums)[4]) {
  const BetaVals b = lz_beta_vals(sums);
  lz_beta_store(lz, rhs, o, j, b);
  if (b.ok) lz.j[rhs] = j + 1;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Pair stencil: Av_j = sv_j H(mu) vhat_j, Aw_j = sw_j H(-mu) what_j (H(mu)^H = H(-mu)),
// alpha_j = w_j^H A v_j = conj(sw_j) sum_x what_j(x)^H Av_j(x).
// Block (PS, 2): threadIdx.y = 0 applies H(mu) to vhat, = 1 applies H(-mu) to what, for the same
// PS sites, so each thread holds one stencil's registers and the two halves of the block share
// the link lines in L1. PS (64, 48 or 32 sites) sets how evenly the blocks spread over the SMs:
// 12^4 FP64 with 64 sites is 324 blocks, three on 20 SMs and two on the other 132 (the SMs sat
// idle a third of the time under ncu); with 48 sites it is 432 blocks, 2.84 per SM.
// ONE_ROLE: one warp-uniform half per block instead (block (PS, 1), even blocks H(mu) vhat, odd
// blocks H(-mu) what), twice the blocks at half the size: 12^4 with 32 sites is 1296 one-warp
// blocks, at most 9 on an SM against a mean of 8.53 (with both halves per block: 5 against 4.26).
template <class R, int LF, int PS, bool ONE_ROLE = false>
__global__ void __launch_bounds__(ONE_ROLE ? PS : 2 * PS) k_lz_pair(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm, LzDev lz,
                                                            const typename V2<R>::T* vh, const typename V2<R>::T* wh,
                                                            typename V2<R>::T* av, typename V2<R>::T* aw) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  const double2 swd = lz.sw[o + j];
  const T* vj = vh + vcol(lz, rhs, j, n);
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  const int s = (ONE_ROLE ? (int)(blockIdx.x >> 1) : (int)blockIdx.x) * PS + threadIdx.x;
  const bool is_w = ONE_ROLE ? (blockIdx.x & 1) != 0 : threadIdx.y == 1;
  const double sd[3] = {lz.sv[o + j], swd.x, swd.y};
  R sc[3];
  scalars_in<R, 3>(sd, sc);
  Red<R> acc[2];
  if (s < g.vol) {
    Spin<R> ov;
    if (!is_w) {
      dslash_site<LF, R>(g, U, s, cp, Loader<R, true>{vj, g.vol, false}, ov);
      const R sv = sc[0];
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
      const cplx<R> sw = mk<R>(sc[1], sc[2]);
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
    if (lin_tid() == 0) lz_alpha_finish(lz, rhs, o, j, swd, pv);
  }
}

// The same step with 8 threads per site (small lattices): see pair_split. Each thread finishes
// one spin (three colours) of its site: scale, gamma5, store, and for the v half the partial of
// alpha_j. SITES sites per block, at least MINB blocks per SM.
template <class R, int LF, int MINB = 1, int SITES = kSplitSites>
__global__ void __launch_bounds__(8 * SITES, MINB) k_lz_pair_split(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm,
                                                                   LzDev lz, const typename V2<R>::T* vh,
                                                                   const typename V2<R>::T* wh,
                                                                   typename V2<R>::T* av, typename V2<R>::T* aw) {
  using T = typename V2<R>::T;
  __shared__ SplitSmem<R, SITES> sm;
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  const double2 swd = lz.sw[o + j];
  const T* vj = vh + vcol(lz, rhs, j, n);
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  const double sd[3] = {lz.sv[o + j], swd.x, swd.y};
  R sc[3];
  scalars_in<R, 3>(sd, sc);
  const R sv = sc[0];
  const cplx<R> sw = mk<R>(sc[1], sc[2]);
  Red<R> acc[2];
  pair_split<R, LF, SITES>(g, U, cp, cm, vj, wj, sm, [&](int which, int s, int sp, cplx<R> (&x)[3]) {
    const R g5 = sp >= 2 ? (R)-1 : (R)1;
    if (which == 0) {
      cplx<R> wv[3];  // loads first (see k_lz_pair)
#pragma unroll
      for (int a = 0; a < 3; ++a) wv[a] = ldc<R>(wj, (size_t)(sp * 3 + a) * g.vol + s);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const cplx<R> y = (g5 * sv) * x[a];
        stc<R>(av + (size_t)rhs * n, (size_t)(sp * 3 + a) * g.vol + s, y);
        acc[0].dot2(wv[a].re, y.re, wv[a].im, y.im);
        acc[1].dot2(wv[a].re, y.im, -wv[a].im, y.re);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) stc<R>(aw + (size_t)rhs * n, (size_t)(sp * 3 + a) * g.vol + s, g5 * (sw * x[a]));
    }
  });
  double tot[2];
  block_reduce<R, 2>(acc, tot);
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  double pv[4] = {tot[0], tot[1], 0, 0};
  if (publish_partials<4>(pv, part, lz.count + rhs)) {
    reduce_partials<4>(part, gridDim.x, pv);
    if (lin_tid() == 0) lz_alpha_finish(lz, rhs, o, j, swd, pv);
  }
}

// The pair step on one block per SM, all SMs with the same number of warps, whose warps claim
// tasks from a counter; task t applies H(mu) to vhat_j (t even) or H(-mu) to what_j (t odd) on the
// 32 sites of chunk t / 2. The FP64 stencil is bound by the FP64 pipe, so a grid finishes with its
// most loaded SM: at 12^4 ncu counted 140K / 164K / 214K active cycles (min / mean / max over the
// SMs) for 1296 one-warp blocks placed by the hardware. Here the 1296 tasks go to 152 x 9 warps
// (at most 9 per SM against a mean of 8.53), and on larger lattices, with several tasks per warp,
// a warp that finishes early claims the next. The alpha partial of a chunk goes to the chunk's own
// slot and k_lz_alpha_finish sums the slots in chunk order: the result does not depend on which
// warp ran which task.
constexpr int kDynMaxWarps = 12;  // warps per block at most

template <class R, int LF>
__global__ void __launch_bounds__(32 * kDynMaxWarps, 1) k_lz_pair_dyn(Geom g, Links U, HopCoef<R> cp, HopCoef<R> cm,
                                                                 LzDev lz, const typename V2<R>::T* vh,
                                                                 const typename V2<R>::T* wh,
                                                                 typename V2<R>::T* av, typename V2<R>::T* aw) {
  using T = typename V2<R>::T;
  // launched early (programmatic dependent launch): the blocks are resident while the previous
  // kernel finishes, and wait for it here (a no-op when launched the ordinary way)
  // Launched early (programmatic dependent launch) behind k_lz_settle, which finishes the previous
  // update: status and j are final before k_lz_settle starts (the update advanced j), so they are
  // read now; the column scales sv_j, sw_j are read after griddepcontrol.wait, which each warp runs
  // before its first epilogue, so the settle kernel's serial FP64 chain overlaps the stencil work.
  const int rhs = blockIdx.y;
  __shared__ int stat, jsh;
  if (threadIdx.x == 0) {
    stat = lz.status[rhs];
    jsh = lz.j[rhs];
  }
  __syncthreads();
  if (stat) return;
  const int j = jsh;
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  const T* vj = vh + vcol(lz, rhs, j, n);
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  R sc[3] = {0, 0, 0};
  bool waited = false, stop = false;
  const int lane = threadIdx.x & 31;
  const int nchunk = (g.vol + 31) >> 5;
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  // the scales of step j, once per warp, after the settle kernel has finished (see above); a
  // breakdown found there stops the warp (no stores), the counters are still reset at the end
  auto scales = [&]() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    waited = true;
    if (lz.status[rhs]) {
      stop = true;
      return;
    }
    const double2 swd = lz.sw[o + j];
    sc[0] = (R)lz.sv[o + j];
    sc[1] = (R)swd.x;
    sc[2] = (R)swd.y;
  };
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(lz.claim + rhs, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= 2 * nchunk) break;
    const int c = t >> 1, s = c * 32 + lane;
    const bool is_w = t & 1;
    Red<R> acc[2];
    const bool live = s < g.vol;
    Spin<R> ov;
    if (live) dslash_site<LF, R>(g, U, s, is_w ? cm : cp, Loader<R, true>{is_w ? wj : vj, g.vol, false}, ov);
    if (!waited) scales();  // warp-uniform: every lane reaches it, the status load is one value
    if (stop) break;
    if (live) {
      if (!is_w) {
        cplx<R> wv[12];  // all loads of w_j before the stores of Av (see k_lz_pair)
#pragma unroll
        for (int q = 0; q < 12; ++q) wv[q] = ldc<R>(wj, (size_t)q * g.vol + s);
        cplx<R> a = mk<R>(0, 0);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          cplx<R> x = sc[0] * ov.c[q / 3][q % 3];
          if (q >= 6) x = -x;  // gamma5
          stc<R>(av + (size_t)rhs * n, (size_t)q * g.vol + s, x);
          a = a + cdot(wv[q], x);
        }
        acc[0].add(a.re);
        acc[1].add(a.im);
      } else {
        const cplx<R> sw = mk<R>(sc[1], sc[2]);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          cplx<R> y = sw * ov.c[q / 3][q % 3];
          if (q >= 6) y = -y;  // gamma5
          stc<R>(aw + (size_t)rhs * n, (size_t)q * g.vol + s, y);
        }
      }
    }
    if (!is_w) {  // the chunk's partial of alpha_j, at the chunk's slot
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        acc[0].add(acc[0].shfl_xor(off));
        acc[1].add(acc[1].shfl_xor(off));
      }
      if (lane == 0) {
        double* pc = part + (size_t)c * 4;
        pc[0] = acc[0].get();
        pc[1] = acc[1].get();
        pc[2] = 0.0;
        pc[3] = 0.0;
      }
    }
  }
  // a warp that found no task has not waited yet: the kernel must not complete before the settle
  // kernel it was launched behind (later kernels rely on stream order)
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
  // the last block to finish resets the task counter (every block has stopped claiming by then);
  // the chunk partials are summed by k_lz_alpha_finish or by the FP64 update's blocks
  __syncthreads();
  if (lin_tid() == 0 && atomicAdd(lz.count + rhs, 1u) == gridDim.x - 1) {
    lz.count[rhs] = 0u;
    lz.claim[rhs] = 0u;
  }
}

// FP32 pair stencil for a batch with each site's links loaded once per group of G right-hand
// sides (dslash_site_g): block (kGroupSites, 2), threadIdx.y = 0 applies H(mu) to the group's vhat_j,
// = 1 applies H(-mu) to its what_j; the grid runs group-fastest (block b: site tile b / ngroups,
// group b % ngroups) so that the groups of a tile share its link lines in L2. Each rhs of the group
// gets its own alpha partials (one slot per tile) and the last tile block of the group finishes
// alpha for each. Right-hand sides that have stopped (status != 0) are computed with the others
// and not stored.
constexpr int kGroupSites = 32;

template <int LF, int G>
__global__ void __launch_bounds__(2 * kGroupSites) k_lz_pair_group(Geom g, Links U, HopCoef<float> cp,
                                                                  HopCoef<float> cm, LzDev lz, const float2* vh,
                                                                  const float2* wh, float2* av, float2* aw) {
  const int ngroups = (lz.nrhs + G - 1) / G;
  const int tile = blockIdx.x / ngroups, grp = blockIdx.x % ngroups, ntiles = gridDim.x / ngroups;
  const int r0 = grp * G, nact = min(G, lz.nrhs - r0);
  const int s = tile * kGroupSites + threadIdx.x;
  const bool is_w = threadIdx.y == 1;
  const size_t n = (size_t)12 * g.vol;
  // per-rhs state, staged once per block (FP64 -> FP32 conversions run on the FP64 pipe)
  __shared__ int st[G], js[G];
  __shared__ float scl[G][3];
  if (lin_tid() < nact) {
    const int r = r0 + lin_tid();
    const int jr = lz.j[r];
    const size_t o = (size_t)r * (lz.kmax + 2);
    st[lin_tid()] = lz.status[r];
    js[lin_tid()] = jr;
    const double2 swd = lz.sw[o + jr];
    scl[lin_tid()][0] = (float)lz.sv[o + jr];
    scl[lin_tid()][1] = (float)swd.x;
    scl[lin_tid()][2] = (float)swd.y;
  }
  __syncthreads();
  bool any = false;
  for (int r = 0; r < nact; ++r) any |= st[r] == 0;
  if (!any) return;
  Loader<float, true> ld[G];
#pragma unroll
  for (int r = 0; r < G; ++r) {
    // a stopped rhs may hold j = 0 (breakdown at the start): any valid column does for its loads
    const int rr = r0 + (r < nact ? r : 0), jr = max(js[r < nact ? r : 0], 1);
    const float2* base = is_w ? wh + ((size_t)(jr & 1) * lz.nrhs + rr) * n : vh + vcol(lz, rr, jr, n);
    ld[r] = Loader<float, true>{base, g.vol, false};
  }
  Red<float> acc[2 * G];
  if (s < g.vol) {
    Spin<float> o[G];
    dslash_site_g<LF, G>(g, U, s, is_w ? cm : cp, ld, nact, o);
#pragma unroll
    for (int r = 0; r < G; ++r) {
      if (r >= nact || st[r] != 0) continue;
      const int rr = r0 + r;
      if (!is_w) {
        const float2* wj = wh + ((size_t)(js[r] & 1) * lz.nrhs + rr) * n;
        cplx<float> wv[12];  // loads before the stores (see k_lz_pair)
#pragma unroll
        for (int q = 0; q < 12; ++q) wv[q] = ldc<float>(wj, (size_t)q * g.vol + s);
        cplx<float> a = mk<float>(0, 0);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          cplx<float> x = scl[r][0] * o[r].c[q / 3][q % 3];
          if (q >= 6) x = -x;  // gamma5
          stc<float>(av + (size_t)rr * n, (size_t)q * g.vol + s, x);
          a = a + cdot(wv[q], x);
        }
        acc[2 * r].add(a.re);
        acc[2 * r + 1].add(a.im);
      } else {
        const cplx<float> sw = mk<float>(scl[r][1], scl[r][2]);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          cplx<float> y = sw * o[r].c[q / 3][q % 3];
          if (q >= 6) y = -y;  // gamma5
          stc<float>(aw + (size_t)rr * n, (size_t)q * g.vol + s, y);
        }
      }
    }
  }
  double tot[2 * G];
  block_reduce<float, 2 * G>(acc, tot);
  __shared__ bool last;
  if (lin_tid() == 0) {
    for (int r = 0; r < nact; ++r) {
      double* pr = lz.part + ((size_t)(r0 + r) * lz.nblk + tile) * 4;
      pr[0] = tot[2 * r];
      pr[1] = tot[2 * r + 1];
      pr[2] = 0.0;
      pr[3] = 0.0;
    }
    __threadfence();
    last = atomicAdd(lz.count + r0, 1u) == (unsigned)ntiles - 1;
    if (last) lz.count[r0] = 0u;
  }
  __syncthreads();
  if (!last) return;
  for (int r = 0; r < nact; ++r) {  // block-uniform loop: reduce_partials synchronises the block
    if (st[r] != 0) continue;
    const int rr = r0 + r;
    double pv[4];
    reduce_partials<4>(lz.part + (size_t)rr * lz.nblk * 4, ntiles, pv);
    if (lin_tid() == 0) {
      const size_t o = (size_t)rr * (lz.kmax + 2);
      lz_alpha_finish(lz, rr, o, js[r], lz.sw[o + js[r]], pv);
    }
  }
}

// vhat_{j+1} = Av_j - alpha_j v_j - beta_{j-1} v_{j-1}
// what_{j+1} = Aw_j - conj(alpha_j) w_j - conj(delta_{j-1}) w_{j-1}    (Eqs. 2sided1/2)
// then delta_j = sqrt|what^H vhat|, beta_j = what^H vhat / delta_j (scaling reading).
// Element-parallel, grid-stride: each thread takes two elements per pass, both loaded before
// either is used. FP64 grids have one pass (256 elements per block): FP64 makes this kernel bound
// by the FP64 pipe, and only many short blocks, which the hardware hands to whichever SM is free,
// give every SM the same share (324 blocks of six passes at 12^4 left the SMs idle half the time);
// a block's partial sums sit at its own index, so the reductions keep a fixed order. The
// coefficients come ready from the pair stencil's last block.
// BAL: one block per SM (launch_sm_fill), block b taking the contiguous elements
// [b n / G, (b + 1) n / G) of its rhs, so every SM holds the same share of the FP64 work (the
// hardware's placement of many short blocks left the busiest SM 1.4 times the mean SM time at
// 12^4); otherwise many short grid-stride blocks.
// XACC: the second pass of the two-pass mode (x += coef_{j+1} vhat_{j+1}), a compile-time choice:
// as a runtime branch the compiler predicated its FP64 instructions, and predicated-off FP64
// instructions still hold the FP64 pipe (ncu: FP64 pipe 83 % busy in the FP32 update with no FP64
// operation executed).
// nchunk > 0 (FP64 one-block-per-SM update after the dynamically scheduled pair stencil): every
// block sums the stencil's nchunk chunk partials of alpha_j itself, in chunk order (so all blocks
// get the same value), and forms the update coefficients; block 0 stores alpha_j and them. This
// replaces a one-block finishing kernel (7.7 us under ncu at 12^4) by about a microsecond at the
// start of every block.
// defer (BAL only): the deferred step. The block that takes the last ticket at the start (every
// block has read j by then) advances j and sets the pending flag; the sums of this update are
// finished by the blocks of the next pair stencil (or by k_lz_settle) instead of a one-block kernel
// after this one (7-10 us per step at 12^4, most of it the latency of a short serial FP64 chain).
template <class R, bool BAL = false, bool XACC = false>
__global__ void __launch_bounds__(BAL ? kBalBlock : kVecBlock) k_lz_update(Geom g, LzDev lz, typename V2<R>::T* vh,
                                                         typename V2<R>::T* wh, const typename V2<R>::T* av,
                                                         const typename V2<R>::T* aw, int nchunk, int defer) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  __shared__ int jsh;
  if (threadIdx.x == 0) {
    jsh = lz.j[rhs];
    if (BAL && defer) {
      __threadfence();  // this block's read of j completes before its ticket
      if (atomicAdd(lz.count + rhs, 1u) == gridDim.x - 1) {
        lz.count[rhs] = 0u;
        lz.j[rhs] = jsh + 1;
        lz.pending[rhs] = 1;
      }
    }
  }
  __syncthreads();
  const int j = jsh;
  const size_t n = (size_t)12 * g.vol;
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  R u[8];  // the four complex coefficients of LzDev::ucoef
  if (BAL && nchunk > 0) {
    __shared__ double uc[8];
    // the earlier steps' scalars are requested before the sum (their latency overlaps it)
    AlphaIn ain{};
    if (threadIdx.x == 0) ain = lz_alpha_inputs(lz, o, j);
    double pv[2];
    sum_partials_by_warp<2, kBalBlock / 64>(lz.part + (size_t)rhs * lz.nblk * 4, nchunk, 4, pv);
    if (threadIdx.x == 0) {
      const double p4[4] = {pv[0], pv[1], 0.0, 0.0};
      double2 c[4];
      const zd alpha = lz_alpha_coeffs(ain, p4, c);
      for (int i = 0; i < 4; ++i) {
        uc[2 * i] = c[i].x;
        uc[2 * i + 1] = c[i].y;
      }
      if (blockIdx.x == 0) lz_alpha_store(lz, rhs, o, j, alpha, c);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) u[i] = (R)uc[i];
  } else {
    scalars_in<R, 8>((const double*)(lz.ucoef + (size_t)rhs * 4), u);
  }
  const cplx<R> a1 = mk<R>(u[0], u[1]), a2 = mk<R>(u[2], u[3]);
  const cplx<R> b1 = mk<R>(u[4], u[5]), b2 = mk<R>(u[6], u[7]);
  const T* vj = vh + vcol(lz, rhs, j, n);
  const T* vjm = vh + vcol(lz, rhs, j > 1 ? j - 1 : 1, n);
  T* vnew = vh + vcol(lz, rhs, j + 1, n);
  double2* xa = XACC ? lz.xacc + (size_t)rhs * n : nullptr;  // second pass: x += coef_{j+1} vhat_{j+1}
  const zd xc = XACC ? ldc<double>(lz.xcoef, o + j + 1) : mk(0.0, 0.0);
  const T* wj = wh + ((size_t)(j & 1) * lz.nrhs + rhs) * n;
  T* wnew = wh + ((size_t)((j + 1) & 1) * lz.nrhs + rhs) * n;  // holds what_{j-1} until overwritten
  const T* avr = av + (size_t)rhs * n;
  const T* awr = aw + (size_t)rhs * n;
  const bool prev = j > 1;
  Red<R> acc[4];
  const size_t hi = BAL ? n * (blockIdx.x + 1) / gridDim.x : n;
  const size_t first = BAL ? n * blockIdx.x / gridDim.x + threadIdx.x : (size_t)blockIdx.x * blockDim.x * 2 + threadIdx.x;
  const size_t step = BAL ? (size_t)blockDim.x * 2 : (size_t)gridDim.x * blockDim.x * 2;
  for (size_t e0 = first; e0 < hi; e0 += step) {
    const size_t e1 = e0 + blockDim.x;
    const bool has1 = e1 < hi;
    const cplx<R> z = mk<R>(0, 0);
    const cplx<R> A0 = ldc<R>(avr, e0), W0 = ldc<R>(awr, e0), v0 = ldc<R>(vj, e0), w0 = ldc<R>(wj, e0);
    const cplx<R> A1 = has1 ? ldc<R>(avr, e1) : z, W1 = has1 ? ldc<R>(awr, e1) : z;
    const cplx<R> v1 = has1 ? ldc<R>(vj, e1) : z, w1 = has1 ? ldc<R>(wj, e1) : z;
    cplx<R> pv0 = z, pw0 = z, pv1 = z, pw1 = z;
    if (prev) {
      pv0 = ldc<R>(vjm, e0);
      pw0 = ldc<R>(wnew, e0);
      if (has1) {
        pv1 = ldc<R>(vjm, e1);
        pw1 = ldc<R>(wnew, e1);
      }
    }
    cplx<R> x0 = cmsub(A0, a1, v0), y0 = cmsub(W0, b1, w0);
    cplx<R> x1 = cmsub(A1, a1, v1), y1 = cmsub(W1, b1, w1);
    if (prev) {
      x0 = cmsub(x0, a2, pv0);
      y0 = cmsub(y0, b2, pw0);
      x1 = cmsub(x1, a2, pv1);
      y1 = cmsub(y1, b2, pw1);
    }
    stc<R>(vnew, e0, x0);
    stc<R>(wnew, e0, y0);
    if constexpr (XACC) {  // the stored (rounded) vector, in the order of the one-pass combine
      const cplx<R> s0 = ldc<R>(vnew, e0);
      stc<double>(xa, e0, ldc<double>(xa, e0) + xc * mk((double)s0.re, (double)s0.im));
    }
    acc[0].dot2(y0.re, x0.re, y0.im, x0.im);  // (y^H x).re
    acc[1].dot2(y0.re, x0.im, -y0.im, x0.re);  // (y^H x).im
    acc[2].dot2(x0.re, x0.re, x0.im, x0.im);
    acc[3].dot2(y0.re, y0.re, y0.im, y0.im);
    if (has1) {
      stc<R>(vnew, e1, x1);
      stc<R>(wnew, e1, y1);
      if constexpr (XACC) {
        const cplx<R> s1 = ldc<R>(vnew, e1);
        stc<double>(xa, e1, ldc<double>(xa, e1) + xc * mk((double)s1.re, (double)s1.im));
      }
      acc[0].dot2(y1.re, x1.re, y1.im, x1.im);
      acc[1].dot2(y1.re, x1.im, -y1.im, x1.re);
      acc[2].dot2(x1.re, x1.re, x1.im, x1.im);
      acc[3].dot2(y1.re, y1.re, y1.im, y1.im);
    }
  }
  double tot[4];
  block_reduce4<R>(acc, tot);
  double* part = lz.part + (size_t)rhs * lz.nblk * 4;
  if (BAL) {  // block partials only (above the chunk partials); k_lz_beta_finish sums them
    if (lin_tid() == 0)
#pragma unroll
      for (int i = 0; i < 4; ++i) part[(size_t)(lz.nblk - kMaxFillSMs + blockIdx.x) * 4 + i] = tot[i];
    return;
  }
  if (publish_partials<4>(tot, part, lz.count + rhs)) {
    double sums[4];
    reduce_partials<4>(part, gridDim.x, sums);
    if (lin_tid() == 0) lz_beta_finish(lz, rhs, o, j, sums);
  }
}

// The end of a balanced update or pair step in a kernel of its own (one block per rhs): the sum of
// the partials and the scalars of the step. In the kernel that produced the partials, the last
// block to finish did this after an atomic ticket and a memory fence per block. Every FP64 warp
// instruction occupies GB300's FP64 pipe for many cycles (two FP64 lanes per SM and clock), so a
// short serial FP64 chain is long: with eight warps summing all values through a block tree, the
// update's finish took 10.2 us under ncu at 12^4. Here each warp sums one value over a share of
// the partials (lane-strided, then a butterfly), and thread 0 adds the shares in a fixed order.
constexpr int kFinishBlock = 256;  // 8 warps: (value, share) pairs of sum_partials_by_warp

__global__ void __launch_bounds__(kFinishBlock) k_lz_beta_finish(LzDev lz, int nparts) {
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  double sums[4];
  sum_partials_by_warp<4, 2>(lz.part + ((size_t)rhs * lz.nblk + lz.nblk - kMaxFillSMs) * 4, nparts, 4, sums);
  if (threadIdx.x == 0) lz_beta_finish(lz, rhs, (size_t)rhs * (lz.kmax + 2), j, sums);
}

// The finish of a deferred update whose successor is not a pair stencil (the chunk's last step).
__global__ void __launch_bounds__(kFinishBlock) k_lz_settle(LzDev lz, int nparts) {
  // let the pair stencil that follows launch now (it reads the scales only after waiting for this)
  asm volatile("griddepcontrol.launch_dependents;");
  const int rhs = blockIdx.y;
  __shared__ int go, jsh;
  if (threadIdx.x == 0) {
    go = ld_acquire(lz.pending + rhs) && !lz.status[rhs];
    jsh = lz.j[rhs];
  }
  __syncthreads();
  if (!go) return;
  const int j = jsh;
  double sums[4];
  sum_partials_by_warp<4, 2>(lz.part + ((size_t)rhs * lz.nblk + lz.nblk - kMaxFillSMs) * 4, nparts, 4, sums);
  if (threadIdx.x == 0) {
    const BetaVals b = lz_beta_vals(sums);
    lz_beta_store(lz, rhs, (size_t)rhs * (lz.kmax + 2), j - 1, b);
    if (!b.ok) lz.j[rhs] = j - 1;
    lz.pending[rhs] = 0;
  }
}

__global__ void __launch_bounds__(kFinishBlock) k_lz_alpha_finish(LzDev lz, int nparts) {
  const int rhs = blockIdx.y;
  if (lz.status[rhs]) return;
  const int j = lz.j[rhs];
  const size_t o = (size_t)rhs * (lz.kmax + 2);
  double pv[2];
  sum_partials_by_warp<2, 4>(lz.part + (size_t)rhs * lz.nblk * 4, nparts, 4, pv);
  if (threadIdx.x == 0) {
    const double p4[4] = {pv[0], pv[1], 0.0, 0.0};
    lz_alpha_finish(lz, rhs, o, j, lz.sw[o + j], p4);
  }
}

// k_lz_pair_dyn on one block per SM, with as many warps as the tasks need (at most kDynMaxWarps).
// True where the FP64 update runs one block per SM (and then, after pair variant 7, sums alpha's
// chunk partials itself).
static bool fp64_update_balanced() {
  const int nsm = sm_count();
  return nsm > 0 && nsm <= kMaxFillSMs;
}

// In the deferred FP64 step the settle kernel (the previous update's finish) runs first and the
// stencil is launched early behind it (see k_lz_pair_dyn); `first` is recorded between them.
template <class R, int LF>
static cudaError_t pair_dyn_launch(const Geom& g, const Links& U, const HopCoef<R>& cp, const HopCoef<R>& cm,
                                   const LzDev& lz, const LzVecs& vec, cudaStream_t st, cudaEvent_t first,
                                   cudaEvent_t mid) {
  const int nsm = std::max(1, sm_count());
  const int ntask = 2 * ((g.vol + 31) >> 5);
  const int warps = std::max(1, std::min(kDynMaxWarps, (ntask + nsm - 1) / nsm));
  using T = typename V2<R>::T;
  const bool deferred = sizeof(R) == 8 && fp64_update_balanced();
  cudaError_t e;
  if (deferred && (e = launch_plain(k_lz_settle, dim3(1, lz.nrhs), dim3(kFinishBlock), st, lz, nsm))) return e;
  if (first && (e = record_timing(first, st))) return e;
  e = launch_sm_fill(k_lz_pair_dyn<R, LF>, lz.nrhs, dim3(32 * warps), st, deferred, g, U, cp, cm, lz,
                     (const T*)vec.vh, (const T*)vec.wh, (T*)vec.av, (T*)vec.aw);
  if (e != cudaSuccess) return e;
  if (mid && (e = record_timing(mid, st))) return e;
  if (sizeof(R) == 8 && fp64_update_balanced()) return cudaSuccess;  // the update's blocks finish alpha
  return launch_plain(k_lz_alpha_finish, dim3(1, lz.nrhs), dim3(kFinishBlock), st, lz, ntask / 2);
}

template <int PS, bool ONE_ROLE = false>
static cudaError_t pair_unsplit(const Geom& g, const Links& U, int lf, bool f64, HopCoef<double> dp, HopCoef<double> dm,
                                HopCoef<float> fp, HopCoef<float> fm, const LzDev& lz, const LzVecs& vec,
                                cudaStream_t st) {
  const unsigned nb = (unsigned)((g.vol + PS - 1) / PS);
  dim3 grid(ONE_ROLE ? 2 * nb : nb, lz.nrhs), block(PS, ONE_ROLE ? 1 : 2);
  if (f64)
    return launch_plain(k_lz_pair<double, LINK_F64, PS, ONE_ROLE>, grid, block, st, g, U, dp, dm, lz,
                        (const double2*)vec.vh, (const double2*)vec.wh, (double2*)vec.av, (double2*)vec.aw);
  if (lf == LINK_F16R12)
    return launch_plain(k_lz_pair<float, LINK_F16R12, PS, ONE_ROLE>, grid, block, st, g, U, fp, fm, lz,
                        (const float2*)vec.vh, (const float2*)vec.wh, (float2*)vec.av, (float2*)vec.aw);
  return launch_plain(k_lz_pair<float, LINK_F32, PS, ONE_ROLE>, grid, block, st, g, U, fp, fm, lz,
                      (const float2*)vec.vh, (const float2*)vec.wh, (float2*)vec.av, (float2*)vec.aw);
}

template <int MINB, int SITES>
static cudaError_t pair_split_launch(const Geom& g, const Links& U, int lf, bool f64, const HopCoef<double>& dp,
                                     const HopCoef<double>& dm, const HopCoef<float>& fp, const HopCoef<float>& fm,
                                     const LzDev& lz, const LzVecs& vec, cudaStream_t st) {
  dim3 grid((g.vol + SITES - 1) / SITES, lz.nrhs), block(SITES, 8);
  if (f64)
    return launch_plain(k_lz_pair_split<double, LINK_F64, MINB, SITES>, grid, block, st, g, U, dp, dm, lz,
                        (const double2*)vec.vh, (const double2*)vec.wh, (double2*)vec.av, (double2*)vec.aw);
  if (lf == LINK_F16R12)
    return launch_plain(k_lz_pair_split<float, LINK_F16R12, MINB, SITES>, grid, block, st, g, U, fp, fm, lz,
                        (const float2*)vec.vh, (const float2*)vec.wh, (float2*)vec.av, (float2*)vec.aw);
  return launch_plain(k_lz_pair_split<float, LINK_F32, MINB, SITES>, grid, block, st, g, U, fp, fm, lz,
                      (const float2*)vec.vh, (const float2*)vec.wh, (float2*)vec.av, (float2*)vec.aw);
}

int resolve_pair_variant(const Geom& g, int lf, bool f64) {
  const int v = tuned_pair_variant(g.vol, f64 ? 0 : lf);
  return v >= 0 ? v : (use_split(g) ? 1 : 0);
}

// FP64 steps with pair shape 7 and the one-block-per-SM update run deferred (see k_lz_update).
static bool deferred_step(bool f64, int variant) { return f64 && variant == 7 && fp64_update_balanced(); }

cudaError_t launch_lanczos_pair(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu,
                                const LzDev& lz, const LzVecs& vec, cudaStream_t st, int variant, cudaEvent_t mid,
                                cudaEvent_t first) {
  if (variant < 0) variant = resolve_pair_variant(g, lf, f64);
  const HopCoef<double> dp = hop_coef<double>(m_w, mu), dm = hop_coef<double>(m_w, -mu);
  const HopCoef<float> fp = hop_coef<float>(m_w, mu), fm = hop_coef<float>(m_w, -mu);
  const double2 *dv = (const double2*)vec.vh, *dw = (const double2*)vec.wh;
  const float2 *fv = (const float2*)vec.vh, *fw = (const float2*)vec.wh;
  cudaError_t e;
  if (variant != 7 && first && (e = record_timing(first, st))) return e;
  if (variant == 1) {
    e = pair_split_launch<1, kSplitSites>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 4) {  // held to 128 registers: two blocks per SM
    e = pair_split_launch<2, kSplitSites>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 5) {  // 16 sites per block held to 168 registers: three blocks per SM
    e = pair_split_launch<3, 16>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 2) {
    e = pair_unsplit<48>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 3) {
    e = pair_unsplit<32>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 6) {
    e = pair_unsplit<32, true>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 8 && !f64 && lz.nrhs > 1) {  // FP32 batches: links once per group of 4 sources
    const unsigned ntile = (unsigned)((g.vol + kGroupSites - 1) / kGroupSites), ngroups = (unsigned)((lz.nrhs + 3) / 4);
    const dim3 grid(ntile * ngroups), block(kGroupSites, 2);
    e = lf == LINK_F16R12
            ? launch_plain(k_lz_pair_group<LINK_F16R12, 4>, grid, block, st, g, U, fp, fm, lz,
                           (const float2*)vec.vh, (const float2*)vec.wh, (float2*)vec.av, (float2*)vec.aw)
            : launch_plain(k_lz_pair_group<LINK_F32, 4>, grid, block, st, g, U, fp, fm, lz,
                           (const float2*)vec.vh, (const float2*)vec.wh, (float2*)vec.av, (float2*)vec.aw);
  } else if (variant == 8) {  // other cases: the 32-site one-thread-per-site shape
    e = pair_unsplit<32>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  } else if (variant == 7) {
    e = f64 ? pair_dyn_launch<double, LINK_F64>(g, U, dp, dm, lz, vec, st, first, mid)
            : lf == LINK_F16R12 ? pair_dyn_launch<float, LINK_F16R12>(g, U, fp, fm, lz, vec, st, first, mid)
                                : pair_dyn_launch<float, LINK_F32>(g, U, fp, fm, lz, vec, st, first, mid);
    first = mid = nullptr;  // recorded around the stencil kernel
  } else {
    e = pair_unsplit<kPairSites>(g, U, lf, f64, dp, dm, fp, fm, lz, vec, st);
  }
  if (e == cudaSuccess && mid) e = record_timing(mid, st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_update(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, cudaStream_t st,
                                  int variant, cudaEvent_t mid) {
  // FP64 (bound by the FP64 pipe): one block per SM with an equal share of the elements; FP32
  // (bound by HBM): enough elements per thread to amortise the block reduction, at least four
  // blocks per SM over the batch
  const int elt = f64 ? 2 : std::max(2, (vec_elts(g, lz.nrhs, false) + 1) & ~1);
  dim3 grid(vec_blocks(g, elt), lz.nrhs);
  cudaError_t e;
  const int nsm = f64 ? sm_count() : 0;
  const bool xacc = lz.xacc != nullptr;
  if (f64 && fp64_update_balanced()) {
    // after pair variant 7 the blocks sum alpha's chunk partials themselves, and the step is deferred
    const int nchunk = variant == 7 ? (g.vol + 31) >> 5 : 0;
    const int defer = deferred_step(f64, variant) ? 1 : 0;
    e = xacc ? launch_sm_fill(k_lz_update<double, true, true>, lz.nrhs, dim3(kBalBlock), st, false, g, lz,
                              (double2*)vec.vh, (double2*)vec.wh, (const double2*)vec.av, (const double2*)vec.aw,
                              nchunk, defer)
             : launch_sm_fill(k_lz_update<double, true, false>, lz.nrhs, dim3(kBalBlock), st, false, g, lz,
                              (double2*)vec.vh, (double2*)vec.wh, (const double2*)vec.av, (const double2*)vec.aw,
                              nchunk, defer);
    if (e == cudaSuccess && mid) e = record_timing(mid, st);
    mid = nullptr;
    if (e == cudaSuccess && !defer)
      e = launch_plain(k_lz_beta_finish, dim3(1, lz.nrhs), dim3(kFinishBlock), st, lz, nsm);
  } else if (f64) {
    e = xacc ? launch_plain(k_lz_update<double, false, true>, grid, dim3(kVecBlock), st, g, lz, (double2*)vec.vh,
                            (double2*)vec.wh, (const double2*)vec.av, (const double2*)vec.aw, 0, 0)
             : launch_plain(k_lz_update<double, false, false>, grid, dim3(kVecBlock), st, g, lz, (double2*)vec.vh,
                            (double2*)vec.wh, (const double2*)vec.av, (const double2*)vec.aw, 0, 0);
  } else {
    e = xacc ? launch_plain(k_lz_update<float, false, true>, grid, dim3(kVecBlock), st, g, lz, (float2*)vec.vh,
                            (float2*)vec.wh, (const float2*)vec.av, (const float2*)vec.aw, 0, 0)
             : launch_plain(k_lz_update<float, false, false>, grid, dim3(kVecBlock), st, g, lz, (float2*)vec.vh,
                            (float2*)vec.wh, (const float2*)vec.av, (const float2*)vec.aw, 0, 0);
  }
  if (e == cudaSuccess && mid) e = record_timing(mid, st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_step(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu, const LzDev& lz,
                                const LzVecs& vec, cudaStream_t st, int variant) {
  cudaError_t e = launch_lanczos_pair(g, U, lf, f64, m_w, mu, lz, vec, st, variant);
  if (e != cudaSuccess) return e;
  return launch_lanczos_update(g, f64, lz, vec, st, variant);
}

cudaError_t launch_lanczos_settle(const Geom& g, bool f64, const LzDev& lz, cudaStream_t st, int variant) {
  if (!deferred_step(f64, variant)) return cudaSuccess;
  return launch_plain(k_lz_settle, dim3(1, lz.nrhs), dim3(kFinishBlock), st, lz, sm_count());
}

int lanczos_settle_launches(bool f64, int variant) { return deferred_step(f64, variant) ? 1 : 0; }

int lanczos_step_launches(const Geom& g, int lf, bool f64, int variant) {
  (void)g;
  (void)lf;
  const bool bal = f64 && fp64_update_balanced();
  if (deferred_step(f64, variant)) return 3;  // settle, stencil, update
  return (variant == 7 && !bal ? 2 : 1) + (bal ? 2 : 1);
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
