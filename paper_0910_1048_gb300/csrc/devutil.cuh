// Device helpers shared by the kernel translation units.
#pragma once

#include "wilson.cuh"

namespace ovl {

template <class R> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };

template <class R>
__device__ __forceinline__ cplx<R> ldc(const typename V2<R>::T* p, size_t i) {
  typename V2<R>::T v = p[i];
  return mk<R>(v.x, v.y);
}
template <class R>
__device__ __forceinline__ void stc(typename V2<R>::T* p, size_t i, cplx<R> a) {
  typename V2<R>::T v;
  v.x = a.re;
  v.y = a.im;
  p[i] = v;
}

__device__ __forceinline__ int lin_tid() { return threadIdx.x + threadIdx.y * blockDim.x; }
__device__ __forceinline__ int lin_nthreads() { return blockDim.x * blockDim.y; }

// Sum NV doubles over the block; result valid in thread 0. Block size multiple of 32.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sm[NV][32];
  const int t = lin_tid();
  const int lane = t & 31, warp = t >> 5, nw = lin_nthreads() >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[i][warp] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = lane < nw ? sm[i][lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    }
  }
  __syncthreads();
}

// c - a b with fused multiply-adds (complex).
template <class R>
__device__ __forceinline__ cplx<R> cmsub(cplx<R> c, cplx<R> a, cplx<R> b) {
  return mk<R>(fma(-a.re, b.re, fma(a.im, b.im, c.re)), fma(-a.re, b.im, fma(-a.im, b.re, c.im)));
}

// ------------------------------------------------------------------ reduction accumulators
// FP64 kernels accumulate in double. FP32 kernels accumulate in float-float (an unevaluated sum
// hi + lo of two FP32 words, about 48 significant bits, Dekker/Knuth two-sum): this GPU's FP64
// pipe runs at 1/64 of the FP32 rate, so double sums would bound the FP32 kernels. Block
// results are converted to double; the cross-block sums stay FP64.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);  // exact error of s (two-sum)
  e += a.lo + b.lo;
  const float hi = s + e;
  return FF{hi, e - (hi - s)};
}

// N FP64 scalars in the kernel's precision R, converted once per block: on this GPU a
// double -> float conversion issues on the FP64 pipe (1/64 of the FP32 rate), so FP32 threads
// that each convert their own coefficients spend a large share of an element-wise kernel on it
// (ncu, 16 sources at 16^4: the FP32 Lanczos update had its FP64 pipe 87% active). Every thread of
// the block must call this (it synchronises the block); src is read by threads 0..N-1 only.
template <class R, int N>
__device__ __forceinline__ void scalars_in(const double* src, R (&out)[N]) {
  if constexpr (sizeof(R) == 8) {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = src[i];
  } else {
    __shared__ R sh[N];
    const int t = lin_tid();
    if (t < N) sh[t] = (R)src[t];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = sh[i];
  }
}

template <class R> struct Red;
template <> struct Red<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(const Red& o) { v += o.v; }
  __device__ __forceinline__ Red shfl_down(int off) const {
    Red r;
    r.v = __shfl_down_sync(0xffffffffu, v, off);
    return r;
  }
  __device__ __forceinline__ Red shfl_xor(int m) const {
    Red r;
    r.v = __shfl_xor_sync(0xffffffffu, v, m);
    return r;
  }
  // v += a b + c d with two fused operations
  __device__ __forceinline__ void dot2(double a, double b, double c, double d) { v = fma(a, b, fma(c, d, v)); }
  __device__ __forceinline__ double get() const { return v; }
};
template <> struct Red<float> {
  FF v{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { v = ff_add(v, FF{x, 0.f}); }
  __device__ __forceinline__ void add(const Red& o) { v = ff_add(v, o.v); }
  __device__ __forceinline__ Red shfl_down(int off) const {
    Red r;
    r.v.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    r.v.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    return r;
  }
  __device__ __forceinline__ Red shfl_xor(int m) const {
    Red r;
    r.v.hi = __shfl_xor_sync(0xffffffffu, v.hi, m);
    r.v.lo = __shfl_xor_sync(0xffffffffu, v.lo, m);
    return r;
  }
  // v += a b + c d (the product pair rounded in FP32, the sum kept in float-float)
  __device__ __forceinline__ void dot2(float a, float b, float c, float d) { add(fmaf(a, b, c * d)); }
  __device__ __forceinline__ double get() const { return (double)v.hi + (double)v.lo; }
};

// Sum NV accumulators over the block; out valid in thread 0. Block size multiple of 32.
template <class R, int NV>
__device__ __forceinline__ void block_reduce(Red<R> (&a)[NV], double (&out)[NV]) {
  __shared__ Red<R> sm[NV][32];
  const int t = lin_tid();
  const int lane = t & 31, warp = t >> 5, nw = lin_nthreads() >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a[i].add(a[i].shfl_down(off));
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[i][warp] = a[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      a[i] = lane < nw ? sm[i][lane] : Red<R>();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) a[i].add(a[i].shfl_down(off));
      out[i] = a[i].get();
    }
  }
  __syncthreads();
}

// Sum 4 accumulators over the block with fewer shuffles: in the first two butterfly levels each
// lane keeps half of its values and sends the other half (4 -> 2 -> 1 value per lane), then one
// value per lane finishes the warp; out valid in thread 0. Block size a multiple of 32, <= 1024.
template <class R>
__device__ __forceinline__ void block_reduce4(Red<R> (&a)[4], double (&out)[4]) {
  __shared__ Red<R> sm[4][32];
  const int t = lin_tid();
  const int lane = t & 31, warp = t >> 5, nw = lin_nthreads() >> 5;
  // level 1 (offset 16): lanes < 16 keep values 0, 1; lanes >= 16 keep 2, 3
  const bool hi16 = lane & 16;
  Red<R> k0 = hi16 ? a[2] : a[0], k1 = hi16 ? a[3] : a[1];
  Red<R> s0 = hi16 ? a[0] : a[2], s1 = hi16 ? a[1] : a[3];
  k0.add(s0.shfl_xor(16));
  k1.add(s1.shfl_xor(16));
  // level 2 (offset 8): lanes with bit 8 clear keep k0, set keep k1
  const bool hi8 = lane & 8;
  Red<R> k = hi8 ? k1 : k0, sd = hi8 ? k0 : k1;
  k.add(sd.shfl_xor(8));
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) k.add(k.shfl_xor(off));
  // lane 0 holds value 0, lane 8 value 1, lane 16 value 2, lane 24 value 3 of this warp
  if ((lane & 7) == 0) sm[lane >> 3][warp] = k;
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Red<R> v = lane < nw ? sm[i][lane] : Red<R>();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v.add(v.shfl_down(off));
      out[i] = v.get();
    }
  }
  __syncthreads();
}

// Write this block's NV partials; returns true in every thread of the last block to arrive.
// The counter is reset to 0 by the last block so the next launch starts clean.
template <int NV>
__device__ __forceinline__ bool publish_partials(double (&v)[NV], double* part, unsigned* count) {
  __shared__ bool last;
  if (lin_tid() == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[(size_t)blockIdx.x * NV + i] = v[i];
    __threadfence();
    unsigned t = atomicAdd(count, 1u);
    last = (t == gridDim.x - 1);
    if (last) *count = 0u;
  }
  __syncthreads();
  return last;
}

// Sum over b < count of part[b * stride + v] for the NV values v, result in thread 0: each warp
// sums one value over a share of the partials (lane-strided, then a butterfly) and thread 0 adds
// the shares in a fixed order. blockDim.x = 32 * NV * SPLIT. Few FP64 instructions in a short
// dependent chain, which is what costs time on GB300's narrow FP64 pipe.
template <int NV, int SPLIT>
__device__ __forceinline__ void sum_partials_by_warp(const double* part, int count, int stride, double (&out)[NV]) {
  static_assert(NV * SPLIT <= 32, "at most 32 warps");
  __shared__ double sh[NV * SPLIT];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, v = w % NV, q = w / NV;
  double s = 0.0;
#pragma unroll 4
  for (int b = q * 32 + lane; b < count; b += 32 * SPLIT) s += __ldcg(part + (size_t)b * stride + v);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) sh[w] = s;
  __syncthreads();
  if (t == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double a = sh[i];
#pragma unroll
      for (int k = 1; k < SPLIT; ++k) a += sh[k * NV + i];
      out[i] = a;
    }
}

// Fixed-order sum of nblk partials (NV each) by the last block; result in thread 0. With at least
// NV warps, each warp sums one value over a share of the partials (lane-strided, then a butterfly)
// and thread 0 adds the shares in order: on GB300 every FP64 warp instruction holds the FP64 pipe
// for many cycles, and a tree over all warps and values costs several times more instructions.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* part, int nblk, double (&v)[NV]) {
  __threadfence();
  const int nt = lin_nthreads(), t = lin_tid(), nw = nt >> 5;
  if (nw >= NV) {
    __shared__ double sh[32];
    const int split = nw / NV, lane = t & 31, w = t >> 5, val = w % NV, q = w / NV;
    double s = 0.0;
    if (q < split) {
#pragma unroll 4
      for (int b = q * 32 + lane; b < nblk; b += 32 * split) s += __ldcg(part + (size_t)b * NV + val);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0 && q < split) sh[w] = s;
    __syncthreads();
    if (t == 0)
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        double a = sh[i];
        for (int k = 1; k < split; ++k) a += sh[k * NV + i];
        v[i] = a;
      }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  // four partials per thread per pass, loaded before they are added (one memory round trip per
  // pass instead of one per partial)
  for (int b0 = t; b0 < nblk; b0 += 4 * nt) {
    double x[4][NV];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * nt;
#pragma unroll
      for (int i = 0; i < NV; ++i) x[u][i] = b < nblk ? __ldcg(part + (size_t)b * NV + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] += x[u][i];
  }
  block_sum<NV>(v);
}

// ------------------------------------------------------------------ spinor loaders
template <class R, bool NATIVE>
struct Loader {
  const typename V2<R>::T* p;
  int vol;
  bool g5;
  __device__ __forceinline__ void operator()(int s, Spin<R>& o) const {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      size_t i = NATIVE ? (size_t)c * vol + s : (size_t)s * 12 + c;
      o.c[c / 3][c % 3] = ldc<R>(p, i);
    }
    if (g5) gamma5_inplace(o);
  }
};

template <class R, bool NATIVE>
__device__ __forceinline__ void store_spin(typename V2<R>::T* p, int vol, int s, const Spin<R>& o) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    size_t i = NATIVE ? (size_t)c * vol + s : (size_t)s * 12 + c;
    stc<R>(p, i, o.c[c / 3][c % 3]);
  }
}


// ------------------------------------------------------------------ split-site pair stencil
// For small lattices (too few sites to fill 152 SMs with one thread per site) every site is
// shared by 8 threads: threadIdx.y = which * 4 + dir, `which` selecting input 0 (coefficients
// c0) or input 1 (c1), `dir` one direction's forward and backward hops. After the hops each
// thread finalises one spin of its site (spin = dir, the three colours): the other three
// directions leave their contributions to that spin in shared memory, and the finalising thread
// adds them to its own and to the diagonal term, then hands D_W(+-mu) psi at (spin, colours
// 0..2) to `emit(which, site, spin, x[3])`. The epilogue (scaling, stores, reductions) is thus
// spread over all eight warps of the block instead of the two that held the first direction.
// SITES sites per block (blockDim = (SITES, 8)).
constexpr int kSplitSites = 32;

template <class R, int SITES = kSplitSites>
struct SplitSmem {
  cplx<R> part[2][3][12][SITES];  // [which][slot of the contributing direction][component][site]
};

template <class R, int LF, int SITES = kSplitSites, class Emit>
__device__ __forceinline__ void pair_split(const Geom& g, const Links& U, const HopCoef<R>& c0, const HopCoef<R>& c1,
                                           const typename V2<R>::T* in0, const typename V2<R>::T* in1,
                                           SplitSmem<R, SITES>& sm, Emit emit) {
  const int tx = threadIdx.x, which = threadIdx.y >> 2, dir = threadIdx.y & 3;
  const int s = blockIdx.x * SITES + tx;
  const typename V2<R>::T* in = which ? in1 : in0;
  const HopCoef<R>& c = which ? c1 : c0;
  Loader<R, true> ld{in, g.vol, false};
  Spin<R> acc;
#pragma unroll
  for (int q = 0; q < 12; ++q) acc.c[q / 3][q % 3] = mk<R>(0, 0);
  if (s < g.vol) {
    Nbr n;
    neighbours(g, s, n);
    if (dir == 0) {
      hop_dir<0, LF>(g, U, s, n, c.ks, c.ks, ld, acc);
    } else if (dir == 1) {
      hop_dir<1, LF>(g, U, s, n, c.ks, c.ks, ld, acc);
    } else if (dir == 2) {
      hop_dir<2, LF>(g, U, s, n, c.ks, c.ks, ld, acc);
    } else {
      R ktf = (n.t == g.lt - 1) ? (R)g.t_bc * c.ktf : c.ktf;
      R ktb = (n.t == 0) ? (R)g.t_bc * c.ktb : c.ktb;
      hop_dir<3, LF>(g, U, s, n, ktf, ktb, ld, acc);
    }
    // contributions to the spins finalised by the other three threads; slot = this direction's
    // index among the three
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
      if (sp != dir)
#pragma unroll
        for (int a = 0; a < 3; ++a) sm.part[which][dir < sp ? dir : dir - 1][sp * 3 + a][tx] = acc.c[sp][a];
  }
  __syncthreads();
  if (s < g.vol) {
    cplx<R> x[3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
      if (sp == dir)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int q = sp * 3 + a;
          x[a] = ldc<R>(in, (size_t)q * g.vol + s) + acc.c[sp][a] + sm.part[which][0][q][tx] +
                 sm.part[which][1][q][tx] + sm.part[which][2][q][tx];
        }
    emit(which, s, dir, x);
  }
}

}  // namespace ovl
