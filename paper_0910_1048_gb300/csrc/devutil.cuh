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


}  // namespace ovl
