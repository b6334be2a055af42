// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <shared_mutex>
#include <string>
#include <vector>

#include "../../include/ovl.h"

#if defined(__CUDACC__)
#define OVL_HD __host__ __device__ __forceinline__
#else
#define OVL_HD inline
#endif

namespace ovl {

// ------------------------------------------------------------------ error reporting
void set_error(const char* fmt, ...);
void clear_error();

#define OVL_CHECK_CUDA(expr)                                                          \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      ::ovl::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
      return _e == cudaErrorMemoryAllocation ? OVL_ENOMEM : OVL_ECUDA;                \
    }                                                                                 \
  } while (0)

#define OVL_REQUIRE(cond, ...)          \
  do {                                  \
    if (!(cond)) {                      \
      ::ovl::set_error(__VA_ARGS__);    \
      return OVL_EINVAL;                \
    }                                   \
  } while (0)

#define OVL_TRY(expr)                   \
  do {                                  \
    ovl_status _s = (expr);             \
    if (_s != OVL_OK) return _s;        \
  } while (0)

// Makes device `dev` current for the guard's lifetime and gives the caller back its own current
// device when the guard goes out of scope (every C-ABI call leaves the caller's device as it was).
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    if ((err = cudaGetDevice(&prev)) != cudaSuccess) {
      prev = -1;
      return;
    }
    if (prev != dev) err = cudaSetDevice(dev);
    else prev = -1;  // nothing to restore
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Enter device `dev` for the rest of the enclosing scope; returns ECUDA from the caller on failure.
#define OVL_DEVICE_SCOPE(dev)                 \
  ::ovl::DeviceGuard _ovl_dev_guard(dev);     \
  OVL_CHECK_CUDA(_ovl_dev_guard.err)

// ------------------------------------------------------------------ complex arithmetic
template <class R>
struct cplx {
  R re, im;
};

template <class R> OVL_HD cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <class R> OVL_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> OVL_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> OVL_HD cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <class R> OVL_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> OVL_HD cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <class R> OVL_HD cplx<R> conj(cplx<R> a) { return {a.re, -a.im}; }
template <class R> OVL_HD cplx<R> times_i(cplx<R> a) { return {-a.im, a.re}; }    // i a
template <class R> OVL_HD cplx<R> times_mi(cplx<R> a) { return {a.im, -a.re}; }   // -i a
template <class R> OVL_HD R norm2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// conj(a) * b
template <class R> OVL_HD cplx<R> cdot(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

using zd = cplx<double>;

// ------------------------------------------------------------------ lattice geometry
struct Geom {
  int lx, ly, lz, lt;
  int vol;       // sites
  int sy, sz, st;  // strides of y, z, t in the canonical site index
  int t_bc;      // +1 periodic, -1 antiperiodic in time
};

// Device-resident links in the formats the caller asked for. Layout [dir][comp][V]
// (component-major, site fastest) so that a warp's 32 consecutive sites read one
// contiguous segment per component.
struct Links {
  const double2* f64 = nullptr;   // [4][9][V]
  const float2* f32 = nullptr;    // [4][9][V]
  const uint32_t* f16 = nullptr;  // [4][6][V] half2 bits, rows 0 and 1
};

enum LinkFmt { LINK_F64 = 0, LINK_F32 = 1, LINK_F16R12 = 2 };

}  // namespace ovl

// ------------------------------------------------------------------ handles
struct ovl_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
};

struct ovl_deflation {
  int m = 0;
  double m_w = 0, mu = 0;
  double2* R = nullptr;    // [m][12][V] native
  double2* L = nullptr;    // [m][12][V] native
  std::vector<double> lam; // 2m (re, im)
};

namespace ovl {
struct DirectWS;
struct MultiWS;
void free_direct_ws(DirectWS*);
void free_multi_ws(MultiWS*);
}  // namespace ovl

struct ovl_lattice {
  ovl_ctx* ctx = nullptr;
  ovl_lattice* parent = nullptr;  // a server view: links and deflation set are the parent's
  std::shared_mutex guard;        // solves hold it shared, ovl_set_links / ovl_set_deflation exclusive
  std::atomic<int> servers{0};    // request servers this lattice is registered with
  bool owns_links = true;    // false for a server view sharing another lattice's links
  bool server_mode = false;  // workspaces allocated stream-ordered and released after each solve
  ovl::DirectWS* dws = nullptr;
  ovl::MultiWS* mws = nullptr;
  ovl::Geom g{};
  uint32_t formats = 0;
  double2* u64 = nullptr;
  float2* u32 = nullptr;
  uint32_t* u16 = nullptr;
  ovl_deflation defl;
  // last direct solve's tridiagonal matrices (host copies), per rhs
  std::vector<std::vector<double>> last_alpha, last_beta, last_delta;
  ovl::Links links() const {
    ovl::Links l;
    l.f64 = u64;
    l.f32 = u32;
    l.f16 = u16;
    return l;
  }
  // the lattice whose links and deflation set a solve on this one uses (a view reads its parent's,
  // so later ovl_set_links / ovl_set_deflation on the field are seen by every view)
  const ovl_lattice* src() const { return parent ? parent : this; }
  ovl_lattice* src() { return parent ? parent : this; }
};
