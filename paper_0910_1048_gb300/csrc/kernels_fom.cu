// Kernels of restarted FOM-LR on A^2 (Algorithm 1 with Section 5's rational sign).
//
// The Arnoldi basis of a cycle is V[j][rhs][12][V] (j = 0..k; the rhs of a Krylov index contiguous,
// so a stencil over all right-hand sides reads one block). Step j: w = A(A v_j) into V[j+1] (two
// stencil launches), then classical Gram-Schmidt twice against v_0..v_j:
//   gs pass 0:  c1 = V^H w                                  (column dots)
//   gs pass 1:  w -= V c1;  c2 = V^H w                      (update and dots in one read of V)
//   gs pass 2:  w -= V c2;  h_{j+1,j} = |w|;  H[0..j][j] = c1 + c2
//   scale:      v_{j+1} = w / h_{j+1,j}
// Every reduction is deterministic: per-block partials, then one block per value sums them in
// block order (no last-block tail over many columns) and writes the FP64 results.
#include "devutil.cuh"
#include "kernels_fom.h"

namespace ovl {

// One Gram-Schmidt pass over columns 0..j for every rhs (blockIdx.y): block partials only.
// PASS 0: dots of w; PASS 1: w -= V c1, dots of the new w; PASS 2: w -= V c2, |w|^2. E elements per
// thread. j = -1 (PASS 2): |v_0|^2.
template <class R, int PASS>
__global__ void __launch_bounds__(kFomBlock) k_fom_gs(FomDev f, int j, int E) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (f.status[rhs]) return;
  const size_t n = f.n;
  const int nc = j + 1;  // columns v_0..v_j
  __shared__ cplx<R> cs[kFomMaxK + 1];
  const T* V = (const T*)f.V;
  T* w = (T*)f.V + ((size_t)(j + 1) * f.nrhs + rhs) * n;
  const size_t cstride = (size_t)f.nrhs * n;  // between columns
  const T* v0 = V + (size_t)rhs * n;
  if (PASS > 0 && nc > 0) {
    const double2* c = (PASS == 1 ? f.c1 : f.c2) + (size_t)rhs * (f.kcap + 1);
    for (int i = threadIdx.x; i < nc; i += blockDim.x) cs[i] = mk<R>((R)c[i].x, (R)c[i].y);
    __syncthreads();
  }
  // this thread's elements: E runs of the block, each coalesced
  const size_t base = (size_t)blockIdx.x * blockDim.x * E + threadIdx.x;
  cplx<R> wl[kFomMaxE];
#pragma unroll
  for (int q = 0; q < kFomMaxE; ++q) {
    const size_t e = base + (size_t)q * blockDim.x;
    wl[q] = (q < E && e < n) ? ldc<R>(w, e) : mk<R>(0, 0);
  }
  if (PASS > 0 && nc > 0) {
    for (int i = 0; i < nc; ++i) {
      const cplx<R> ci = cs[i];
#pragma unroll
      for (int q = 0; q < kFomMaxE; ++q) {
        const size_t e = base + (size_t)q * blockDim.x;
        if (q < E && e < n) wl[q] = cmsub(wl[q], ci, ldc<R>(v0 + (size_t)i * cstride, e));
      }
    }
#pragma unroll
    for (int q = 0; q < kFomMaxE; ++q) {
      const size_t e = base + (size_t)q * blockDim.x;
      if (q < E && e < n) stc<R>(w, e, wl[q]);
    }
  }
  double* part = f.part + ((size_t)rhs * f.nblk + blockIdx.x) * f.pstride;
  if (PASS < 2) {
    for (int i = 0; i < nc; ++i) {
      Red<R> acc[2];
#pragma unroll
      for (int q = 0; q < kFomMaxE; ++q) {
        const size_t e = base + (size_t)q * blockDim.x;
        if (q < E && e < n) {
          const cplx<R> v = ldc<R>(v0 + (size_t)i * cstride, e);
          acc[0].dot2(v.re, wl[q].re, v.im, wl[q].im);   // (v^H w).re
          acc[1].dot2(v.re, wl[q].im, -v.im, wl[q].re);  // (v^H w).im
        }
      }
      double tot[2];
      block_reduce<R, 2>(acc, tot);
      if (threadIdx.x == 0) {
        part[2 * i] = tot[0];
        part[2 * i + 1] = tot[1];
      }
    }
  } else {
    Red<R> acc[1];
#pragma unroll
    for (int q = 0; q < kFomMaxE; ++q) acc[0].dot2(wl[q].re, wl[q].re, wl[q].im, wl[q].im);
    double tot[1];
    block_reduce<R, 1>(acc, tot);
    if (threadIdx.x == 0) part[0] = tot[0];
  }
}

// The sums of the block partials of pass PASS, one block per value (blockIdx.x) and rhs, each in
// block order, and what they define: c1 (PASS 0), c2 (PASS 1), or (PASS 2) column j of H with
// h_{j+1,j} = |w| and the scale of v_{j+1} (j = -1: beta = |v_0| and its scale).
template <int PASS>
__global__ void __launch_bounds__(128) k_fom_reduce(FomDev f, int j, int nb) {
  const int rhs = blockIdx.y, v = blockIdx.x;
  if (f.status[rhs]) return;
  const double* part = f.part + (size_t)rhs * f.nblk * f.pstride;
  double acc[1] = {0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc[0] += __ldcg(part + (size_t)b * f.pstride + v);
  block_sum<1>(acc);
  if (threadIdx.x != 0) return;
  const size_t cb = (size_t)rhs * (f.kcap + 1);
  if (PASS == 0) {
    double* c = reinterpret_cast<double*>(f.c1 + cb);
    c[v] = acc[0];
  } else if (PASS == 1) {
    double* c = reinterpret_cast<double*>(f.c2 + cb);
    c[v] = acc[0];
  } else {
    const double h = sqrt(acc[0]);
    if (j < 0) {
      f.beta[rhs] = h;
      f.scale[rhs] = h > 0.0 ? 1.0 / h : 0.0;
      f.kdone[rhs] = 0;
      return;
    }
    double2* Hc = f.H + ((size_t)rhs * f.kcap + j) * (f.kcap + 1);
    for (int i = 0; i <= j; ++i)
      Hc[i] = make_double2(f.c1[cb + i].x + f.c2[cb + i].x, f.c1[cb + i].y + f.c2[cb + i].y);
    Hc[j + 1] = make_double2(h, 0.0);
    f.kdone[rhs] = j + 1;
    if (!(h > 0.0) || !(h < 1e300))
      f.status[rhs] = 1;  // the Krylov space is invariant (or non-finite): the cycle ends here
    else
      f.scale[rhs] = 1.0 / h;
  }
}

// v_{j+1} = w * scale[rhs]  (also used for v_0 = r / |r| with j = -1)
template <class R>
__global__ void __launch_bounds__(256) k_fom_scale(FomDev f, int j) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (f.status[rhs]) return;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  R s[1];
  scalars_in<R, 1>(f.scale + rhs, s);
  if (e >= f.n) return;
  T* w = (T*)f.V + ((size_t)(j + 1) * f.nrhs + rhs) * f.n;
  stc<R>(w, e, s[0] * ldc<R>(w, e));
}

static int fom_elts(size_t n) {
  // enough elements per thread to amortise the per-column block reductions, at least about two
  // blocks per SM for one rhs; independent of the batch, so that a rhs's reductions run in the same
  // order alone and in a batch
  return (int)std::max<size_t>(1, std::min<size_t>(kFomMaxE, n / ((size_t)kFomBlock * 304)));
}

int fom_partial_slots(size_t n) { return (int)((n + kFomBlock - 1) / kFomBlock); }

cudaError_t launch_fom_gs(const FomDev& f, bool f64, int j, int pass, cudaStream_t st) {
  const int E = fom_elts(f.n);
  const unsigned nb = (unsigned)((f.n + (size_t)kFomBlock * E - 1) / ((size_t)kFomBlock * E));
  dim3 grid(nb, f.nrhs);
  if (f64) {
    if (pass == 0) k_fom_gs<double, 0><<<grid, kFomBlock, 0, st>>>(f, j, E);
    else if (pass == 1) k_fom_gs<double, 1><<<grid, kFomBlock, 0, st>>>(f, j, E);
    else k_fom_gs<double, 2><<<grid, kFomBlock, 0, st>>>(f, j, E);
  } else {
    if (pass == 0) k_fom_gs<float, 0><<<grid, kFomBlock, 0, st>>>(f, j, E);
    else if (pass == 1) k_fom_gs<float, 1><<<grid, kFomBlock, 0, st>>>(f, j, E);
    else k_fom_gs<float, 2><<<grid, kFomBlock, 0, st>>>(f, j, E);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned nv = pass < 2 ? (unsigned)(2 * (j + 1)) : 1u;
  if (nv == 0) return cudaSuccess;
  dim3 rgrid(nv, f.nrhs);
  if (pass == 0) k_fom_reduce<0><<<rgrid, 128, 0, st>>>(f, j, (int)nb);
  else if (pass == 1) k_fom_reduce<1><<<rgrid, 128, 0, st>>>(f, j, (int)nb);
  else k_fom_reduce<2><<<rgrid, 128, 0, st>>>(f, j, (int)nb);
  return cudaGetLastError();
}

cudaError_t launch_fom_scale(const FomDev& f, bool f64, int j, cudaStream_t st) {
  dim3 grid((unsigned)((f.n + 255) / 256), f.nrhs);
  if (f64) k_fom_scale<double><<<grid, 256, 0, st>>>(f, j);
  else k_fom_scale<float><<<grid, 256, 0, st>>>(f, j);
  return cudaGetLastError();
}

// ---- start, restart, combine

// From canonical b: x_P = R sign(Lambda) c (c = L^H b from k_defl_dots), r = b - R c into V[0]
// (native, the basis precision), X = 0.
template <class R>
__global__ void __launch_bounds__(kBlock) k_fom_start(Geom g, FomDev f, const double2* b, int m, const double2* Rv,
                                                      const double* lam_sign, const double2* dots, double2* xp,
                                                      double2* X) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.vol) return;
  const size_t n = f.n;
  T* v0 = (T*)f.V + (size_t)rhs * n;
  const double2* dr = dots + (size_t)rhs * 2 * m;
  for (int c = 0; c < 12; ++c) {
    zd r = ldc<double>(b, (size_t)rhs * n + (size_t)s * 12 + c), x = mk(0.0, 0.0);
    for (int i = 0; i < m; ++i) {
      const zd ci = ldc<double>(dr, i);
      const zd ri = ldc<double>(Rv, (size_t)i * n + (size_t)c * g.vol + s);
      r = r - ci * ri;
      x = x + lam_sign[i] * (ci * ri);
    }
    const size_t e = (size_t)c * g.vol + s;
    if (xp) stc<double>(xp, (size_t)rhs * n + e, x);
    stc<double>(X, (size_t)rhs * n + e, mk(0.0, 0.0));
    stc<R>(v0, e, mk<R>((R)r.re, (R)r.im));
  }
}

cudaError_t launch_fom_start(const Geom& g, bool f64, const FomDev& f, const double2* b, int m, const double2* R,
                             const double2* L, const double* lam_sign, double2* dots, double* dpart, unsigned* dcount,
                             double2* xp, double2* X, cudaStream_t st) {
  dim3 grid((g.vol + kBlock - 1) / kBlock, f.nrhs);
  if (m > 0) {
    cudaError_t e = launch_defl_dots(g, f.nrhs, m, b, R, L, dpart, dcount, dots, st);
    if (e != cudaSuccess) return e;
  }
  if (f64) k_fom_start<double><<<grid, kBlock, 0, st>>>(g, f, b, m, R, lam_sign, dots, xp, X);
  else k_fom_start<float><<<grid, kBlock, 0, st>>>(g, f, b, m, R, lam_sign, dots, xp, X);
  return cudaGetLastError();
}

// Restart: V[0] = (I - P) V[k] with P = R L^H. Dots d_i = l_i^H v (per-block partials, last block
// sums in order), then the update in a second launch.
template <class R>
__global__ void __launch_bounds__(kBlock) k_fom_proj_dots(Geom g, FomDev f, int k, int m, const double2* Lv,
                                                          double* part, unsigned* count, double2* d) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (f.status[rhs] == 2) return;
  const size_t n = f.n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const T* vk = (const T*)f.V + ((size_t)k * f.nrhs + rhs) * n;
  double* pr = part + (size_t)rhs * m * gridDim.x * 2;
  for (int i = 0; i < m; ++i) {
    double acc[2] = {0, 0};
    if (e < n) {
      const cplx<R> v = ldc<R>(vk, e);
      const zd l = ldc<double>(Lv, (size_t)i * n + e);
      const zd p = cdot(l, mk((double)v.re, (double)v.im));
      acc[0] = p.re;
      acc[1] = p.im;
    }
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
      pr[((size_t)i * gridDim.x + blockIdx.x) * 2] = acc[0];
      pr[((size_t)i * gridDim.x + blockIdx.x) * 2 + 1] = acc[1];
    }
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(count + rhs, 1u);
    last = (t == gridDim.x - 1);
    if (last) count[rhs] = 0u;
  }
  __syncthreads();
  if (!last) return;
  for (int i = 0; i < m; ++i) {
    double acc[2];
    reduce_partials<2>(pr + (size_t)i * gridDim.x * 2, gridDim.x, acc);
    if (threadIdx.x == 0) d[(size_t)rhs * m + i] = make_double2(acc[0], acc[1]);
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_fom_proj_apply(FomDev f, int k, int m, const double2* Rv, const double2* d) {
  using T = typename V2<R>::T;
  const int rhs = blockIdx.y;
  if (f.status[rhs] == 2) return;
  const size_t n = f.n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const T* vk = (const T*)f.V + ((size_t)k * f.nrhs + rhs) * n;
  T* v0 = (T*)f.V + (size_t)rhs * n;
  const cplx<R> v = ldc<R>(vk, e);
  zd r = mk((double)v.re, (double)v.im);
  for (int i = 0; i < m; ++i) r = r - ldc<double>(d, (size_t)rhs * m + i) * ldc<double>(Rv, (size_t)i * n + e);
  stc<R>(v0, e, mk<R>((R)r.re, (R)r.im));
}

cudaError_t launch_fom_restart(const Geom& g, bool f64, const FomDev& f, int k, int m, const double2* R,
                               const double2* L, double* part, unsigned* count, double2* d, cudaStream_t st) {
  dim3 grid((unsigned)((f.n + kBlock - 1) / kBlock), f.nrhs), grid2((unsigned)((f.n + 255) / 256), f.nrhs);
  if (m > 0) {
    if (f64) k_fom_proj_dots<double><<<grid, kBlock, 0, st>>>(g, f, k, m, L, part, count, d);
    else k_fom_proj_dots<float><<<grid, kBlock, 0, st>>>(g, f, k, m, L, part, count, d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (f64) k_fom_proj_apply<double><<<grid2, 256, 0, st>>>(f, k, m, R, d);
  else k_fom_proj_apply<float><<<grid2, 256, 0, st>>>(f, k, m, R, d);
  return cudaGetLastError();
}

// X += sum_{i < kr} coef_i v_i (FP64 accumulation), kr[rhs] columns of this cycle's basis.
template <class R>
__global__ void __launch_bounds__(256) k_fom_combine(FomDev f, const int* kr, const double2* coef, double2* X) {
  using T = typename V2<R>::T;
  __shared__ double2 cs[kFomMaxK + 1];
  const int rhs = blockIdx.y;
  const int k = kr[rhs];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = coef[(size_t)rhs * (f.kcap + 1) + i];
  __syncthreads();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.n || k == 0) return;
  zd acc = ldc<double>(X, (size_t)rhs * f.n + e);
  for (int i = 0; i < k; ++i) {
    const cplx<R> v = ldc<R>((const T*)f.V + ((size_t)i * f.nrhs + rhs) * f.n, e);
    acc = acc + mk(cs[i].x, cs[i].y) * mk((double)v.re, (double)v.im);
  }
  stc<double>(X, (size_t)rhs * f.n + e, acc);
}

cudaError_t launch_fom_combine(const FomDev& f, bool f64, const int* kr, const double2* coef, double2* X,
                               cudaStream_t st) {
  dim3 grid((unsigned)((f.n + 255) / 256), f.nrhs);
  if (f64) k_fom_combine<double><<<grid, 256, 0, st>>>(f, kr, coef, X);
  else k_fom_combine<float><<<grid, 256, 0, st>>>(f, kr, coef, X);
  return cudaGetLastError();
}

}  // namespace ovl
