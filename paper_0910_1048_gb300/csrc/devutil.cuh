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

// Fixed-order sum of nblk partials (NV each) by the last block; result in thread 0.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* part, int nblk, double (&v)[NV]) {
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int b = lin_tid(); b < nblk; b += lin_nthreads())
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __ldcg(part + (size_t)b * NV + i);
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
// c0) or input 1 (c1), `dir` one direction's forward and backward hops. Directions 1..3 leave
// their partial spinors in shared memory; the dir-0 thread of each (site, which) adds them to
// its own hops and the diagonal term and hands the full D_W(+-mu) psi to `emit`.
constexpr int kSplitSites = 32;

template <class R>
struct SplitSmem {
  cplx<R> part[2][3][12][kSplitSites];
};

template <class R, int LF, class Emit>
__device__ __forceinline__ void pair_split(const Geom& g, const Links& U, const HopCoef<R>& c0, const HopCoef<R>& c1,
                                           const typename V2<R>::T* in0, const typename V2<R>::T* in1,
                                           SplitSmem<R>& sm, Emit emit) {
  const int tx = threadIdx.x, which = threadIdx.y >> 2, dir = threadIdx.y & 3;
  const int s = blockIdx.x * kSplitSites + tx;
  const typename V2<R>::T* in = which ? in1 : in0;
  const HopCoef<R>& c = which ? c1 : c0;
  Loader<R, true> ld{in, g.vol, false};
  Spin<R> acc;
  if (s < g.vol) {
    Nbr n;
    neighbours(g, s, n);
    if (dir == 0) {
      ld(s, acc);  // diagonal term
      hop_dir<0, LF>(g, U, s, n, c.ks, c.ks, ld, acc);
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) acc.c[q / 3][q % 3] = mk<R>(0, 0);
      if (dir == 1) {
        hop_dir<1, LF>(g, U, s, n, c.ks, c.ks, ld, acc);
      } else if (dir == 2) {
        hop_dir<2, LF>(g, U, s, n, c.ks, c.ks, ld, acc);
      } else {
        R ktf = (n.t == g.lt - 1) ? (R)g.t_bc * c.ktf : c.ktf;
        R ktb = (n.t == 0) ? (R)g.t_bc * c.ktb : c.ktb;
        hop_dir<3, LF>(g, U, s, n, ktf, ktb, ld, acc);
      }
#pragma unroll
      for (int q = 0; q < 12; ++q) sm.part[which][dir - 1][q][tx] = acc.c[q / 3][q % 3];
    }
  }
  __syncthreads();
  if (dir == 0 && s < g.vol) {
#pragma unroll
    for (int q = 0; q < 12; ++q)
      acc.c[q / 3][q % 3] = acc.c[q / 3][q % 3] + sm.part[which][0][q][tx] + sm.part[which][1][q][tx] +
                            sm.part[which][2][q][tx];
    emit(which, s, acc);
  }
}

}  // namespace ovl
