// Allocation-free variant of the direct two-sided Lanczos sign solve.
//
// Some callers cannot allocate device memory: processes whose device memory is owned by
// another allocator (a framework's caching pool, or a server that reserves its whole budget
// at start-up), and latency-critical loops that must not call cudaMalloc/cudaFree (which can
// synchronize the device and can fail with out-of-memory in the middle of a run). For them,
// ovl_apply_sign_noalloc runs the same kernels as ovl_apply_sign's direct method with every
// scratch buffer (Krylov basis, work vectors, recurrence scalars, reduction partials) placed
// in one file-scope __device__ array of fixed size. It creates no streams, events or graphs
// and allocates no pinned memory; it works on the caller's stream and synchronizes it.
//
// Host code cannot use the array's name as a device address (it names a host-side stand-in),
// so the address is taken with cudaGetSymbolAddress with the lattice's device current: on the
// first call for that device, which should come before any stream capture, and again on every
// later call made outside a capture (an address cached before a device reset is never reused).
// The caller's current device is restored on return, and a stream of another device is refused.
// Every call shares the array: a call clears the counters that must start at zero, and calls
// that overlap on the GPU (two streams, two threads) race on the array.
#include <chrono>
#include <complex>
#include <mutex>

#include "kernels.h"
#include "stoprule.h"

namespace ovl {

ovl_status small_sign(int k, const std::complex<double>* al, const std::complex<double>* be,
                      const std::complex<double>* de, std::complex<double>* y, int method, double* hint_c,
                      int* hint_s, int* ritz_count);

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kMaxDevices = 128;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
char* g_addr[kMaxDevices] = {nullptr};

// Device address of the static array on device `dev` (current). Looked up again on every call
// made outside a stream capture, so that an address cached before a device reset is never
// reused; inside a capture the address cached by an earlier call is used.
ovl_status static_scratch(int dev, cudaStream_t st, char** out) {
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("apply_sign_noalloc: device ordinal %d out of range", dev);
    return OVL_EINVAL;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // unknown: keep the cached address if there is one
  }
  if (!g_addr[dev] || cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);  // the device is current here
    if (e != cudaSuccess || !p) {
      set_error("apply_sign_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return OVL_ECUDA;
    }
    g_addr[dev] = (char*)p;
  }
  *out = g_addr[dev];
  return OVL_OK;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Rhs {
  int k = 0;
  std::vector<std::complex<double>> y, yprev;
  double est = 1e300, hint_c = 0;
  int hint_s = 0, evals = 0, ritz = 0;
  StopTrack trk;
  ovl_status status = OVL_PENDING;
  bool done = false;
};

}  // namespace

}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_apply_sign_noalloc(ovl_lattice* lat, const ovl_sign_params* p, int32_t nrhs,
                                             const void* b, void* x, ovl_sign_info* info, void* stream) {
  clear_error();
  auto t0 = std::chrono::steady_clock::now();
  OVL_REQUIRE(lat && p && b && x, "apply_sign_noalloc: NULL argument");
  OVL_REQUIRE(p->method == OVL_DIRECT_2SL, "apply_sign_noalloc: only the direct two-sided Lanczos method");
  OVL_REQUIRE(!p->host_io, "apply_sign_noalloc: b and x must be device buffers");
  OVL_REQUIRE(!p->two_pass, "apply_sign_noalloc: the two-pass mode is not available here");
  OVL_REQUIRE(nrhs >= 1 && nrhs <= 64, "apply_sign_noalloc: nrhs must be in [1, 64]");
  OVL_REQUIRE(p->precision >= OVL_PREC_F64 && p->precision <= OVL_PREC_F32_F16LINKS, "apply_sign_noalloc: precision");
  OVL_REQUIRE(2.0 * p->m_W + 8.0 != 0.0, "apply_sign_noalloc: m_W = -4 has no kappa");
  const bool f64 = p->precision == OVL_PREC_F64;
  const int lf = p->precision == OVL_PREC_F32_F16LINKS ? LINK_F16R12 : (f64 ? LINK_F64 : LINK_F32);
  OVL_REQUIRE(lat->src()->u64 && (f64 || (lf == LINK_F32 ? lat->src()->u32 != nullptr : lat->src()->u16 != nullptr)),
              "apply_sign_noalloc: links not set in the format this precision needs");
  int m = 0;
  if (p->use_deflation) {
    OVL_REQUIRE(lat->src()->defl.m > 0 && lat->src()->defl.m_w == p->m_W && lat->src()->defl.mu == p->mu,
                "apply_sign_noalloc: no deflation set for this (m_W, mu)");
    m = lat->src()->defl.m;
  }
  const int kmax = p->fixed_k > 0 ? p->fixed_k : p->k_max;
  OVL_REQUIRE(kmax >= 1, "apply_sign_noalloc: k_max must be >= 1");
  std::shared_lock<std::shared_mutex> shared(lat->src()->guard);  // links / deflation set stay as they are
  OVL_DEVICE_SCOPE(lat->ctx->device);  // the caller's current device is restored on return
  cudaStream_t st = (cudaStream_t)stream;
  if (st) {  // the scratch address below is this device's: the stream must belong to it too
    int sdev = -1;
    OVL_CHECK_CUDA(cudaStreamGetDevice(st, &sdev));
    OVL_REQUIRE(sdev == lat->ctx->device, "apply_sign_noalloc: the stream belongs to device %d, the lattice to %d",
                sdev, lat->ctx->device);
  }
  char* base = nullptr;
  OVL_TRY(static_scratch(lat->ctx->device, st, &base));
  const Geom& g = lat->g;
  const size_t n = (size_t)12 * g.vol, elt = f64 ? 16 : 8;
  const int nblk = partial_slots(g), ks = kmax + 2;
  // layout inside the static array (same buffers as the allocating path)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al256(bytes);
    return o;
  };
  size_t o_vh = take((size_t)nrhs * (kmax + 1) * n * elt), o_wh = take((size_t)2 * nrhs * n * elt);
  size_t o_av = take((size_t)nrhs * n * elt), o_aw = take((size_t)nrhs * n * elt);
  size_t o_xp = take((size_t)nrhs * n * 16), o_j = take((size_t)nrhs * 4), o_st = take((size_t)nrhs * 4);
  size_t o_sv = take((size_t)nrhs * ks * 8), o_sw = take((size_t)nrhs * ks * 16);
  size_t o_al = take((size_t)nrhs * ks * 16), o_be = take((size_t)nrhs * ks * 16);
  size_t o_de = take((size_t)nrhs * ks * 8), o_vn = take((size_t)nrhs * ks * 8), o_b0 = take((size_t)nrhs * 8);
  size_t o_pa = take((size_t)nrhs * std::max(m, 1) * nblk * 4 * 8), o_cn = take((size_t)nrhs * 12);
  size_t o_uc = take((size_t)nrhs * 4 * 16);
  size_t o_do = take((size_t)nrhs * 2 * std::max(m, 1) * 16), o_ls = take((size_t)std::max(m, 1) * 8);
  size_t o_co = take((size_t)nrhs * kmax * 16), o_kr = take((size_t)nrhs * 4);
  // buffers of the stopping estimate (the same kernel and rule as ovl_apply_sign)
  size_t o_n1 = take((size_t)nrhs * kmax * 16), o_n2 = take((size_t)nrhs * kmax * 16);
  size_t o_nk = take((size_t)nrhs * 4), o_np = take((size_t)nrhs * 2 * vec_blocks(g) * 8);
  size_t o_nc = take((size_t)nrhs * 4), o_no = take((size_t)nrhs * 2 * 8);
  if (off > kStaticScratchBytes) {
    set_error("apply_sign_noalloc: needs %zu bytes of scratch, the static array holds %zu (64 MiB); "
              "use ovl_apply_sign or a smaller k_max / lattice / nrhs", off, kStaticScratchBytes);
    return OVL_EINVAL;
  }
  LzDev lz;
  lz.kmax = kmax;
  lz.nrhs = nrhs;
  lz.nblk = nblk;
  lz.vcols = kmax + 1;  // the whole basis
  lz.j = (int*)(base + o_j);
  lz.status = (int*)(base + o_st);
  lz.sv = (double*)(base + o_sv);
  lz.sw = (double2*)(base + o_sw);
  lz.alpha = (double2*)(base + o_al);
  lz.beta = (double2*)(base + o_be);
  lz.delta = (double*)(base + o_de);
  lz.vnorm = (double*)(base + o_vn);
  lz.beta0 = (double*)(base + o_b0);
  lz.part = (double*)(base + o_pa);
  lz.count = (unsigned*)(base + o_cn);
  lz.claim = lz.count + nrhs;
  lz.pending = (int*)(lz.claim + nrhs);
  lz.ucoef = (double2*)(base + o_uc);
  LzVecs vec;
  vec.vh = base + o_vh;
  vec.wh = base + o_wh;
  vec.av = base + o_av;
  vec.aw = base + o_aw;
  vec.xp = m > 0 ? (double2*)(base + o_xp) : nullptr;
  double2* dots = (double2*)(base + o_do);
  double* lam_sign = (double*)(base + o_ls);
  double2* coef = (double2*)(base + o_co);
  int* kr = (int*)(base + o_kr);
  double2 *nd1 = (double2*)(base + o_n1), *nd2 = (double2*)(base + o_n2);
  int* nkr = (int*)(base + o_nk);
  double* npart = (double*)(base + o_np);
  unsigned* ncount = (unsigned*)(base + o_nc);
  double* nout = (double*)(base + o_no);
  // the array keeps the previous call's contents: the block counters must start at zero
  OVL_CHECK_CUDA(cudaMemsetAsync(lz.count, 0, (size_t)nrhs * 12, st));
  OVL_CHECK_CUDA(cudaMemsetAsync(ncount, 0, (size_t)nrhs * 4, st));
  std::vector<double> ls(std::max(m, 1));
  for (int i = 0; i < m; ++i) ls[i] = lat->src()->defl.lam[2 * i] >= 0 ? 1.0 : -1.0;
  if (m > 0) OVL_CHECK_CUDA(cudaMemcpyAsync(lam_sign, ls.data(), m * 8, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(launch_lanczos_start(g, f64, lz, vec, (const double2*)b, m, lat->src()->defl.R, lat->src()->defl.L, lam_sign,
                                      dots, st));
  const Links U = lat->src()->links();
  const int chunk = std::max(1, std::min(p->check_every > 0 ? p->check_every : 20, kmax));
  const bool fixed = p->fixed_k > 0;
  // host copies of the scalars (pageable: the copies complete before the host reads them)
  std::vector<double2> h_al((size_t)nrhs * ks), h_be((size_t)nrhs * ks);
  std::vector<double> h_de((size_t)nrhs * ks), h_vn((size_t)nrhs * ks), h_sv((size_t)nrhs * ks), h_b0(nrhs);
  std::vector<int> h_j(nrhs), h_st(nrhs);
  auto snapshot = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h_al.data(), lz.alpha, h_al.size() * 16, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_be.data(), lz.beta, h_be.size() * 16, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_de.data(), lz.delta, h_de.size() * 8, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_vn.data(), lz.vnorm, h_vn.size() * 8, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_sv.data(), lz.sv, h_sv.size() * 8, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_b0.data(), lz.beta0, nrhs * 8, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_j.data(), lz.j, nrhs * 4, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(h_st.data(), lz.status, nrhs * 4, cudaMemcpyDeviceToHost, st))) return e;
    return cudaStreamSynchronize(st);
  };
  std::vector<Rhs> rs(nrhs);
  double t_small = 0;
  auto evaluate = [&](int r) -> ovl_status {
    Rhs& s = rs[r];
    int j = h_j[r], stt = h_st[r];
    int k = stt == 3 ? 0 : (stt == 1 ? j : j - 1);
    if (k < 1) {
      s.k = 0;
      s.y.clear();
      s.est = 0;
      return OVL_OK;
    }
    std::vector<std::complex<double>> al(k), be(k), de(k), y(k);
    for (int i = 0; i < k; ++i) {
      al[i] = {h_al[r * ks + i + 1].x, h_al[r * ks + i + 1].y};
      if (i + 1 < k) {
        be[i] = {h_be[r * ks + i + 1].x, h_be[r * ks + i + 1].y};
        de[i] = h_de[r * ks + i + 1];
      }
    }
    auto ts = std::chrono::steady_clock::now();
    ++s.evals;
    ovl_status e = small_sign(k, al.data(), be.data(), de.data(), y.data(), 0, &s.hint_c, &s.hint_s, &s.ritz);
    t_small += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    if (e != OVL_OK) return e;
    s.est = 1e300;
    s.yprev.swap(s.y);
    s.y.swap(y);
    s.k = k;
    return OVL_OK;
  };
  // relative change ||V (y_k - [y_k'; 0])|| / ||V y_k|| of the evaluated rhs, on the GPU
  auto changes = [&](const std::vector<int>& which) -> ovl_status {
    std::vector<double2> d1((size_t)nrhs * kmax, make_double2(0, 0)), d2 = d1;
    std::vector<int> kk(nrhs, 0);
    bool any = false;
    for (int r : which) {
      Rhs& s = rs[r];
      if (s.k < 1 || s.yprev.empty()) continue;
      kk[r] = s.k;
      any = true;
      for (int i = 0; i < s.k; ++i) {
        std::complex<double> pv = i < (int)s.yprev.size() ? s.yprev[i] : 0.0;
        std::complex<double> a = (s.y[i] - pv) * h_sv[r * ks + i + 1], c = s.y[i] * h_sv[r * ks + i + 1];
        d1[(size_t)r * kmax + i] = make_double2(a.real(), a.imag());
        d2[(size_t)r * kmax + i] = make_double2(c.real(), c.imag());
      }
    }
    if (!any) return OVL_OK;
    OVL_CHECK_CUDA(cudaMemcpyAsync(nd1, d1.data(), d1.size() * 16, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(cudaMemcpyAsync(nd2, d2.data(), d2.size() * 16, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(cudaMemcpyAsync(nkr, kk.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(launch_lanczos_vnorms(g, f64, lz, vec, nkr, nd1, nd2, kmax, npart, ncount, nout, st));
    std::vector<double> out((size_t)nrhs * 2);
    OVL_CHECK_CUDA(cudaMemcpyAsync(out.data(), nout, out.size() * 8, cudaMemcpyDeviceToHost, st));
    OVL_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int r : which)
      if (kk[r] > 0) rs[r].est = out[2 * r + 1] > 0 ? std::sqrt(out[2 * r] / out[2 * r + 1]) : 1e300;
    return OVL_OK;
  };
  int queued = 0, launches = 1 + (m > 0 ? 1 : 0) + 1;
  const int pvar = resolve_pair_variant(g, lf, f64);  // one shape for every step of this call
  while (queued < kmax) {
    int ns = std::min(chunk, kmax - queued);
    for (int i = 0; i < ns; ++i)
      OVL_CHECK_CUDA(launch_lanczos_step(g, U, lf, f64, p->m_W, p->mu, lz, vec, st, pvar));
    OVL_CHECK_CUDA(launch_lanczos_settle(g, f64, lz, st, pvar));  // before the scalars are read
    queued += ns;
    launches += lanczos_step_launches(g, lf, f64, pvar) * ns + lanczos_settle_launches(f64, pvar);
    if (fixed) continue;
    OVL_CHECK_CUDA(snapshot());
    const bool final_snapshot = queued >= kmax;
    std::vector<int> todo;  // same per-rhs schedule as the allocating driver
    for (int r = 0; r < nrhs; ++r)
      if (!rs[r].done && stop_due(rs[r].trk, queued, final_snapshot, h_st[r] != 0)) todo.push_back(r);
    if (todo.empty()) continue;
    std::vector<ovl_status> es(nrhs, OVL_OK);
    std::vector<int> evaluated;
    for (int r : todo) {
      es[r] = evaluate(r);
      if (es[r] == OVL_OK) evaluated.push_back(r);
    }
    OVL_TRY(changes(evaluated));
    for (int r : todo) {
      Rhs& s = rs[r];
      if (es[r] != OVL_OK && !final_snapshot && h_st[r] == 0) {  // as in the allocating driver
        s.trk.next = stop_next_eval(queued, chunk, -1.0);
        continue;
      }
      bool converged = false;
      if (es[r] == OVL_OK && h_st[r] == 0) {
        stop_record(s.trk, s.k, s.est < 1e299 ? s.est : -1.0);
        s.est = s.trk.err;
        converged = stop_converged(s.trk, p->tol);
        stop_schedule(s.trk, queued, chunk, p->tol);
      }
      if (es[r] != OVL_OK) {
        s.status = es[r], s.done = true;
      } else if (h_st[r] == 3) {
        s.status = OVL_OK, s.done = true;
      } else if (h_st[r] == 1) {
        s.status = OVL_EBREAKDOWN, s.done = true;
      } else if (converged) {
        s.status = OVL_OK, s.done = true;
      } else if (final_snapshot) {
        s.status = OVL_ENOCONV, s.done = true;
      }
      if (s.done && h_st[r] == 0) OVL_CHECK_CUDA(cudaMemsetAsync(lz.status + r, 2, sizeof(int), st));
    }
    bool all = true;
    for (int r = 0; r < nrhs; ++r) all = all && rs[r].done;
    if (all) break;
  }
  if (fixed) {
    OVL_CHECK_CUDA(snapshot());
    for (int r = 0; r < nrhs; ++r) {
      ovl_status e = evaluate(r);
      rs[r].status = e != OVL_OK ? e : (h_st[r] == 1 && rs[r].k < kmax ? OVL_EBREAKDOWN : OVL_OK);
      rs[r].est = 0;
    }
  }
  // x = x_P + beta V_k y
  std::vector<double2> hc((size_t)nrhs * kmax, make_double2(0, 0));
  std::vector<int> hk(nrhs);
  ovl_status result = OVL_OK;
  for (int r = 0; r < nrhs; ++r) {
    hk[r] = rs[r].k;
    for (int i = 0; i < rs[r].k; ++i) {
      std::complex<double> c = h_b0[r] * rs[r].y[i] * h_sv[r * ks + i + 1];
      hc[(size_t)r * kmax + i] = make_double2(c.real(), c.imag());
    }
    if (rs[r].status != OVL_OK && result == OVL_OK) result = rs[r].status;
  }
  OVL_CHECK_CUDA(cudaMemcpyAsync(coef, hc.data(), hc.size() * 16, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(cudaMemcpyAsync(kr, hk.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(launch_lanczos_combine(g, f64, lz, vec, kr, coef, kmax, (double2*)x, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  double t_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info)
    for (int r = 0; r < nrhs; ++r) {
      std::memset(&info[r], 0, sizeof(ovl_sign_info));
      info[r].status = rs[r].status;
      info[r].iterations = rs[r].k;
      info[r].matvecs = 2 * rs[r].k;
      info[r].est_error = rs[r].est;
      info[r].t_total_ms = t_total;
      info[r].t_small_ms = t_small;
      info[r].kernel_launches = launches;
      info[r].evaluations = rs[r].evals;
      info[r].ritz_evaluations = rs[r].ritz;
    }
  if (result != OVL_OK) set_error("apply_sign_noalloc: at least one right-hand side ended with status %d", result);
  return result;
}
