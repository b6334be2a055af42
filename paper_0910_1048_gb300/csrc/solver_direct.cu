// Host driver of direct two-sided Lanczos-LR(m, k), Algorithm 4:
//   x_P = R f(Lambda) L^H b;  r = b - R L^H b;  r~ = b - L R^H b;  v_1 = r/beta, w_1 ~ r~;
//   k steps of two-sided Lanczos (Eqs. 2sided1/2);  x = x_P + beta V_k f(H_k) e_1.
// The paper fixes k a priori; this driver also stops early: the scalars of every chunk of
// `check_every` steps are copied to the host, and at each right-hand side's own evaluation
// points (stoprule.h) y_j = sign(H_j) e_1 is evaluated and the relative change
//   ||V_j (y_j - [y_j'; 0])|| / ||V_j y_j||
// since the previous evaluation j' (both norms on the GPU, side stream) feeds the rate-corrected
// error estimate that decides the stop and the next evaluation point.
// All per-step scalars stay on the device (no host round trip inside a chunk), so a chunk
// of steps is one CUDA graph, replayed; the next chunk is queued before the host checks
// the previous one, overlapping sign(H_j) e_1 with device work.
#include <chrono>
#include <complex>
#include <cstdlib>
#include <thread>

#include "kernels.h"
#include "stoprule.h"

namespace ovl {

ovl_status small_sign(int k, const std::complex<double>* al, const std::complex<double>* be,
                      const std::complex<double>* de, std::complex<double>* y, int method, double* hint_c,
                      int* hint_s, int* ritz_count);
void set_sign_concurrency(int n);

struct DirectWS {
  int nrhs = 0, kmax = 0, f64 = -1, m = 0, vol = 0, prio = 0, two_pass = 0;
  LzDev lz;
  LzVecs vec;
  void* dev_block = nullptr;  // one allocation for everything
  size_t dev_bytes = 0;
  double2* dots = nullptr;
  double* lam_sign = nullptr;
  double2* coef = nullptr;
  int* kr = nullptr;          // [nrhs] Krylov dimension per rhs for the combine
  double2* bdev = nullptr;    // staging for host b / x
  double2* xdev = nullptr;
  double2* xacc = nullptr;    // two-pass: [nrhs][12][V] FP64 accumulator of the second pass
  double2* xcoef = nullptr;   // two-pass: [nrhs][kmax+2] coefficient of basis column j
  // pinned host mirrors of the device scalars, double-buffered: the copies behind one
  // chunk's event never overwrite the snapshot the host is reading
  struct Mirror {
    double2* alpha = nullptr;
    double2* beta = nullptr;
    double* delta = nullptr;
    double* vnorm = nullptr;
    double* sv = nullptr;
    double* beta0 = nullptr;
    int* j = nullptr;
    int* status = nullptr;
  } h[2];
  void* h_block = nullptr;
  bool pageable = false;  // server views: host mirrors in pageable memory (no pinned alloc/free)
  // two graphs of `gchunk - 1` steps (alternating chunks); graph q records timing events around
  // its middle step's pair stencil (tev[q][0..1]) and update (tev[q][2..3]); tev[q][4] / [5] mark the
  // end of the stencil / update kernel itself, before a finishing kernel, and tev[q][6] the start of
  // the stencil kernel after the settle kernel of a deferred step
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaEvent_t tev[2][7] = {};
  int gchunk = 0;
  double g_mw = 0, g_mu = 0;
  int g_lf = -1;
  int g_var = -1;  // the pair-stencil shape the graphs launch (a pinned shape may change between solves)
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  // stopping estimate ||V (y_j - y_j')|| / ||V y_j||, computed on a side stream with its own
  // scratch so that it overlaps the chunk in flight on `stream`
  cudaStream_t nstream = nullptr;
  double2* nd1 = nullptr;     // [nrhs][kmax] coefficients of the change
  double2* nd2 = nullptr;     // [nrhs][kmax] coefficients of the Krylov part
  int* nkr = nullptr;         // [nrhs]
  double* npart = nullptr;    // [nrhs][2][vec blocks]
  unsigned* ncount = nullptr; // [nrhs]
  double* nout = nullptr;     // [nrhs][2]
};

void free_direct_ws(DirectWS* w) {
  if (!w) return;
  for (int q = 0; q < 2; ++q) {
    if (w->graph[q]) cudaGraphExecDestroy(w->graph[q]);
    for (auto e : w->tev[q])
      if (e) cudaEventDestroy(e);
  }
  if (w->dev_block) cudaFreeAsync(w->dev_block, w->stream);  // stream-ordered: no device-wide sync
  if (w->h_block) {
    if (w->pageable)
      std::free(w->h_block);
    else
      cudaFreeHost(w->h_block);
  }
  if (w->stream) cudaStreamDestroy(w->stream);
  if (w->nstream) cudaStreamDestroy(w->nstream);
  if (w->ev) cudaEventDestroy(w->ev);
  delete w;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static ovl_status ensure_ws(ovl_lattice* lat, int nrhs, int kmax, bool f64, int m, int prio, bool two_pass) {
  DirectWS* w = lat->dws;
  const int vol = lat->g.vol;
  if (w && w->nrhs == nrhs && w->kmax == kmax && w->f64 == (int)f64 && w->m >= m && w->vol == vol && w->prio == prio &&
      w->two_pass == (int)two_pass)
    return OVL_OK;
  free_direct_ws(w);
  lat->dws = nullptr;
  w = new DirectWS();
  w->nrhs = nrhs;
  w->kmax = kmax;
  w->f64 = f64;
  w->m = m;
  w->vol = vol;
  w->prio = prio;
  w->two_pass = two_pass;
  const size_t n = (size_t)12 * vol;
  const int vcols = two_pass ? 3 : kmax + 1;  // the two-pass mode keeps a window of three columns
  const size_t elt = f64 ? 16 : 8;
  const int nblk = partial_slots(lat->g);  // the most blocks of any reduction kernel
  const int ks = kmax + 2;
  // carve one device block
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  size_t o_vh = take((size_t)nrhs * vcols * n * elt);
  size_t o_wh = take((size_t)2 * nrhs * n * elt);
  size_t o_av = take((size_t)nrhs * n * elt);
  size_t o_aw = take((size_t)nrhs * n * elt);
  size_t o_xp = take((size_t)nrhs * n * 16);
  size_t o_j = take((size_t)nrhs * 4);
  size_t o_st = take((size_t)nrhs * 4);
  size_t o_sv = take((size_t)nrhs * ks * 8);
  size_t o_sw = take((size_t)nrhs * ks * 16);
  size_t o_al = take((size_t)nrhs * ks * 16);
  size_t o_be = take((size_t)nrhs * ks * 16);
  size_t o_de = take((size_t)nrhs * ks * 8);
  size_t o_vn = take((size_t)nrhs * ks * 8);
  size_t o_b0 = take((size_t)nrhs * 8);
  size_t o_pa = take((size_t)nrhs * std::max(m, 1) * nblk * 4 * 8);
  size_t o_cn = take((size_t)nrhs * 12);  // last-block counters, task counters, pending flags
  size_t o_uc = take((size_t)nrhs * 4 * 16);
  size_t o_do = take((size_t)nrhs * 2 * std::max(m, 1) * 16);
  size_t o_ls = take((size_t)std::max(m, 1) * 8);
  size_t o_co = take((size_t)nrhs * kmax * 16);
  size_t o_kr = take((size_t)nrhs * 4);
  size_t o_bd = take((size_t)nrhs * n * 16);
  size_t o_xd = take((size_t)nrhs * n * 16);
  size_t o_n1 = take((size_t)nrhs * kmax * 16), o_n2 = take((size_t)nrhs * kmax * 16);
  size_t o_nk = take((size_t)nrhs * 4), o_np = take((size_t)nrhs * 2 * vec_blocks(lat->g) * 8);
  size_t o_nc = take((size_t)nrhs * 4), o_no = take((size_t)nrhs * 2 * 8);
  size_t o_xa = take(two_pass ? (size_t)nrhs * n * 16 : 0), o_xc = take(two_pass ? (size_t)nrhs * ks * 16 : 0);
  // stream priority: 0 the default; p > 0 asks for p levels more urgent (numerically lower,
  // clamped to the device's range), so that concurrent solves can favour the longest one
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int sp = std::max(greatest, least - std::max(0, prio));
  if (cudaStreamCreateWithPriority(&w->stream, cudaStreamNonBlocking, sp) != cudaSuccess ||
      cudaStreamCreateWithPriority(&w->nstream, cudaStreamNonBlocking, sp) != cudaSuccess) {
    delete w;
    set_error("apply_sign: cannot create a stream");
    return OVL_ECUDA;
  }
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, off, w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) {
    cudaStreamDestroy(w->stream);
    cudaStreamDestroy(w->nstream);
    delete w;
    set_error("apply_sign: cannot allocate %zu bytes of device workspace: %s", off, cudaGetErrorString(e));
    return OVL_ENOMEM;
  }
  w->dev_block = base;
  w->dev_bytes = off;
  w->vec.vh = base + o_vh;
  w->vec.wh = base + o_wh;
  w->vec.av = base + o_av;
  w->vec.aw = base + o_aw;
  w->vec.xp = (double2*)(base + o_xp);
  LzDev& lz = w->lz;
  lz.kmax = kmax;
  lz.nrhs = nrhs;
  lz.nblk = nblk;
  lz.vcols = vcols;
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
  w->dots = (double2*)(base + o_do);
  w->lam_sign = (double*)(base + o_ls);
  w->coef = (double2*)(base + o_co);
  w->kr = (int*)(base + o_kr);
  w->bdev = (double2*)(base + o_bd);
  w->xdev = (double2*)(base + o_xd);
  w->nd1 = (double2*)(base + o_n1);
  w->nd2 = (double2*)(base + o_n2);
  w->nkr = (int*)(base + o_nk);
  w->npart = (double*)(base + o_np);
  w->ncount = (unsigned*)(base + o_nc);
  w->nout = (double*)(base + o_no);
  if (two_pass) {
    w->xacc = (double2*)(base + o_xa);
    w->xcoef = (double2*)(base + o_xc);
  }
  if (cudaMemsetAsync(lz.count, 0, (size_t)nrhs * 12, w->stream) != cudaSuccess ||
      cudaMemsetAsync(w->ncount, 0, (size_t)nrhs * 4, w->stream) != cudaSuccess) {
    free_direct_ws(w);
    set_error("apply_sign: cudaMemset failed");
    return OVL_ECUDA;
  }
  // pinned mirrors: alpha, beta (16 B), delta, vnorm, sv (8 B), beta0, j, status
  size_t hb = (size_t)nrhs * ks * (16 + 16 + 8 + 8 + 8) + nrhs * (8 + 4 + 4) + 64;
  char* hp = nullptr;
  w->pageable = lat->server_mode;
  if (w->pageable)
    hp = (char*)std::malloc(2 * hb);
  else if (cudaMallocHost(&hp, 2 * hb) != cudaSuccess)
    hp = nullptr;
  if (!hp) {
    free_direct_ws(w);
    set_error("apply_sign: cannot allocate host memory for the scalar mirrors");
    return OVL_ENOMEM;
  }
  w->h_block = hp;
  for (int q = 0; q < 2; ++q) {
    DirectWS::Mirror& h = w->h[q];
    h.alpha = (double2*)(hp + q * hb);
    h.beta = h.alpha + (size_t)nrhs * ks;
    h.delta = (double*)(h.beta + (size_t)nrhs * ks);
    h.vnorm = h.delta + (size_t)nrhs * ks;
    h.sv = h.vnorm + (size_t)nrhs * ks;
    h.beta0 = h.sv + (size_t)nrhs * ks;
    h.j = (int*)(h.beta0 + nrhs);
    h.status = h.j + nrhs;
  }
  bool ev_ok = true;
  for (int q = 0; q < 2; ++q)
    for (int i = 0; i < 7; ++i) ev_ok = ev_ok && cudaEventCreate(&w->tev[q][i]) == cudaSuccess;
  if (!ev_ok || cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming) != cudaSuccess) {
    free_direct_ws(w);
    set_error("apply_sign: cannot create stream/event");
    return OVL_ECUDA;
  }
  lat->dws = w;
  return OVL_OK;
}

// queue copies of the scalar arrays to the pinned mirrors
static cudaError_t queue_scalar_copies(DirectWS* w, int q, cudaStream_t st) {
  const size_t ks = (size_t)w->kmax + 2, nr = (size_t)w->nrhs;
  const LzDev& lz = w->lz;
  DirectWS::Mirror& h = w->h[q];
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h.alpha, lz.alpha, nr * ks * 16, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(h.beta, lz.beta, nr * ks * 16, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(h.delta, lz.delta, nr * ks * 8, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(h.vnorm, lz.vnorm, nr * ks * 8, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(h.sv, lz.sv, nr * ks * 8, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(h.beta0, lz.beta0, nr * 8, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(h.j, lz.j, nr * 4, cudaMemcpyDeviceToHost, st))) return e;
  return cudaMemcpyAsync(h.status, lz.status, nr * 4, cudaMemcpyDeviceToHost, st);
}

struct RhsState {
  int k = 0;                       // Krylov dimension of y
  std::vector<std::complex<double>> y, yprev;
  double est = 1e300;
  int status = OVL_PENDING;        // OK / ENOCONV / EBREAKDOWN / EILLPOSED once final
  bool done = false;
  double hint_c = 0;               // (c, s) of the rational small sign, reused between checks
  int hint_s = 0;
  StopTrack trk;                   // rate-corrected stopping estimate (stoprule.h)
  int evals = 0, ritz = 0;         // evaluations of sign(H_j) e_1, of which with new Ritz values
};

// Snapshot of rhs r from the pinned mirrors: H_k, y = sign(H_k) e_1, error estimate.
static ovl_status evaluate_rhs(DirectWS* w, int q, int r, RhsState& rs, double* t_small) {
  const size_t ks = (size_t)w->kmax + 2;
  const DirectWS::Mirror& h = w->h[q];
  int j = h.j[r];
  int st = h.status[r];
  int k = (st == 1) ? j : j - 1;  // after a breakdown alpha_j exists but no beta_j
  if (st == 3) k = 0;              // empty Krylov part: x = x_P
  if (k < 1) {
    rs.k = 0;
    rs.y.clear();
    rs.est = 0;
    return OVL_OK;
  }
  std::vector<std::complex<double>> al(k), be(k), de(k);
  for (int i = 0; i < k; ++i) {
    double2 a = h.alpha[r * ks + i + 1];
    al[i] = {a.x, a.y};
    if (i + 1 < k) {
      double2 b = h.beta[r * ks + i + 1];
      be[i] = {b.x, b.y};
      de[i] = h.delta[r * ks + i + 1];
    }
  }
  std::vector<std::complex<double>> y(k);
  auto t0 = std::chrono::steady_clock::now();
  ++rs.evals;
  ovl_status s = small_sign(k, al.data(), be.data(), de.data(), y.data(), 0, &rs.hint_c, &rs.hint_s, &rs.ritz);
  *t_small += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (s != OVL_OK) return s;
  rs.est = 1e300;  // set by estimate_changes()
  rs.yprev.swap(rs.y);
  rs.y.swap(y);
  rs.k = k;
  return OVL_OK;
}

// est_r = ||V_k (y_k - [y_k'; 0])|| / ||V_k y_k|| for the rhs in `which` (the relative change of
// the Krylov part of x since the previous evaluation), computed on the side stream.
static ovl_status estimate_changes(DirectWS* w, const Geom& g, bool f64, const LzVecs& vec, int q,
                                   std::vector<RhsState>& rs, const std::vector<int>& which) {
  const int nrhs = w->nrhs, kmax = w->kmax;
  const size_t ks = (size_t)kmax + 2;
  const DirectWS::Mirror& h = w->h[q];
  if (w->two_pass) {
    // no stored basis: the change is measured with the column norms |v_i| as if the columns were
    // orthogonal, sum |dy_i|^2 |v_i|^2 / sum |y_i|^2 |v_i|^2
    for (int r : which) {
      RhsState& s = rs[r];
      if (s.k < 1 || s.yprev.empty()) continue;
      double num = 0, den = 0;
      for (int i = 0; i < s.k; ++i) {
        const std::complex<double> pv = i < (int)s.yprev.size() ? s.yprev[i] : 0.0;
        const double vn2 = h.vnorm[r * ks + i + 1] * h.vnorm[r * ks + i + 1];
        num += std::norm(s.y[i] - pv) * vn2;
        den += std::norm(s.y[i]) * vn2;
      }
      s.est = den > 0 ? std::sqrt(num / den) : 1e300;
    }
    return OVL_OK;
  }
  std::vector<double2> d1((size_t)nrhs * kmax, make_double2(0, 0)), d2 = d1;
  std::vector<int> kr(nrhs, 0);
  bool any = false;
  for (int r : which) {
    RhsState& s = rs[r];
    if (s.k < 1 || s.yprev.empty()) continue;
    kr[r] = s.k;
    any = true;
    for (int i = 0; i < s.k; ++i) {
      std::complex<double> p = i < (int)s.yprev.size() ? s.yprev[i] : 0.0;
      std::complex<double> a = (s.y[i] - p) * h.sv[r * ks + i + 1], b = s.y[i] * h.sv[r * ks + i + 1];
      d1[(size_t)r * kmax + i] = make_double2(a.real(), a.imag());
      d2[(size_t)r * kmax + i] = make_double2(b.real(), b.imag());
    }
  }
  if (!any) return OVL_OK;
  cudaStream_t ns = w->nstream;
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->nd1, d1.data(), d1.size() * 16, cudaMemcpyHostToDevice, ns));
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->nd2, d2.data(), d2.size() * 16, cudaMemcpyHostToDevice, ns));
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->nkr, kr.data(), nrhs * 4, cudaMemcpyHostToDevice, ns));
  OVL_CHECK_CUDA(launch_lanczos_vnorms(g, f64, w->lz, vec, w->nkr, w->nd1, w->nd2, kmax, w->npart, w->ncount, w->nout,
                                       ns));
  std::vector<double> out((size_t)nrhs * 2);
  OVL_CHECK_CUDA(cudaMemcpyAsync(out.data(), w->nout, out.size() * 8, cudaMemcpyDeviceToHost, ns));
  OVL_CHECK_CUDA(cudaStreamSynchronize(ns));
  for (int r : which)
    if (kr[r] > 0) rs[r].est = out[2 * r + 1] > 0 ? std::sqrt(out[2 * r] / out[2 * r + 1]) : 1e300;
  return OVL_OK;
}

ovl_status solve_direct(ovl_lattice* lat, const ovl_sign_params* p, int nrhs, const double2* b, double2* x,
                        ovl_sign_info* info, cudaStream_t user_stream) {
  auto t_start = std::chrono::steady_clock::now();
  const bool f64 = p->precision == OVL_PREC_F64;
  const int lf = p->precision == OVL_PREC_F32_F16LINKS ? LINK_F16R12 : (f64 ? LINK_F64 : LINK_F32);
  OVL_REQUIRE(p->k_max >= 1 && p->k_max <= 100000, "apply_sign: k_max must be in [1, 100000]");
  OVL_REQUIRE(lat->src()->u64, "apply_sign: links not set");
  OVL_REQUIRE(f64 || (lf == LINK_F32 ? lat->src()->u32 != nullptr : lat->src()->u16 != nullptr),
              "apply_sign: links not set in the format this precision needs (ovl_set_links formats)");
  int m = 0;
  if (p->use_deflation) {
    OVL_REQUIRE(lat->src()->defl.m > 0, "apply_sign: use_deflation but no deflation set");
    OVL_REQUIRE(lat->src()->defl.m_w == p->m_W && lat->src()->defl.mu == p->mu,
                "apply_sign: deflation set was computed for (m_W, mu) = (%g, %g)", lat->src()->defl.m_w, lat->src()->defl.mu);
    m = lat->src()->defl.m;
  }
  const int kmax = p->fixed_k > 0 ? p->fixed_k : p->k_max;
  const bool two_pass = p->two_pass != 0;
  OVL_TRY(ensure_ws(lat, nrhs, kmax, f64, m, p->priority, two_pass));
  DirectWS* w = lat->dws;
  cudaStream_t st = w->stream;
  const Geom& g = lat->g;
  const size_t n = (size_t)12 * g.vol;
  // order after the caller's stream
  OVL_CHECK_CUDA(cudaEventRecord(w->ev, user_stream));
  OVL_CHECK_CUDA(cudaStreamWaitEvent(st, w->ev, 0));
  const double2* bd = b;
  if (p->host_io) {
    OVL_CHECK_CUDA(cudaMemcpyAsync(w->bdev, b, (size_t)nrhs * n * 16, cudaMemcpyHostToDevice, st));
    bd = w->bdev;
  }
  // start: deflation split and first vectors
  if (m > 0) {
    std::vector<double> ls(m);
    for (int i = 0; i < m; ++i) ls[i] = lat->src()->defl.lam[2 * i] >= 0 ? 1.0 : -1.0;
    OVL_CHECK_CUDA(cudaMemcpyAsync(w->lam_sign, ls.data(), m * 8, cudaMemcpyHostToDevice, st));
  }
  LzVecs vec = w->vec;
  if (m == 0) vec.xp = nullptr;
  OVL_CHECK_CUDA(launch_lanczos_start(g, f64, w->lz, vec, bd, m, lat->src()->defl.R, lat->src()->defl.L, w->lam_sign, w->dots, st));
  const Links U = lat->src()->links();
  // autotuner: on first use of (volume, precision) time every pair-stencil variant on this
  // solve's step-1 data (the real step-1 launch below recomputes everything they write)
  struct TuneArg {
    const Geom* g;
    const Links* U;
    int lf;
    bool f64;
    const ovl_sign_params* p;
    const LzDev* lz;
    const LzVecs* vec;
    cudaStream_t st;
  } targ{&g, &U, lf, f64, p, &w->lz, &vec, st};
  auto measure = [](void* v) -> int {
    TuneArg& t = *(TuneArg*)v;
    float best[kPairVariants];
    for (float& b : best) b = 1e30f;
    cudaEvent_t a, b2;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b2) != cudaSuccess) {
      cudaEventDestroy(a);
      return -1;
    }
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep)
      for (int var = 0; var < kPairVariants && ok; ++var) {
        ok = cudaEventRecord(a, t.st) == cudaSuccess &&
             launch_lanczos_pair(*t.g, *t.U, t.lf, t.f64, t.p->m_W, t.p->mu, *t.lz, *t.vec, t.st, var) ==
                 cudaSuccess &&
             cudaEventRecord(b2, t.st) == cudaSuccess && cudaEventSynchronize(b2) == cudaSuccess;
        float ms_ = 0;
        if (ok && rep > 0 && cudaEventElapsedTime(&ms_, a, b2) == cudaSuccess) best[var] = std::min(best[var], ms_);
      }
    cudaEventDestroy(a);
    cudaEventDestroy(b2);
    cudaGetLastError();
    int pick = 0;
    for (int var = 1; var < kPairVariants; ++var)
      if (best[var] < best[pick]) pick = var;
    return ok ? pick : -1;
  };
  tune_pair_variant(g.vol, f64 ? 0 : lf, measure, &targ);
  const int pvar = resolve_pair_variant(g, lf, f64);  // one shape for every step of this solve
  const int chunk = std::max(1, std::min(p->check_every > 0 ? p->check_every : 20, kmax));
  // one step, with timing events around its two launches when `tev` is given
  auto step = [&](cudaEvent_t* tev) -> cudaError_t {
    cudaError_t e;
    if (tev && (e = record_timing(tev[0], st))) return e;
    if ((e = launch_lanczos_pair(g, U, lf, f64, p->m_W, p->mu, w->lz, vec, st, pvar, tev ? tev[4] : nullptr,
                                 tev ? tev[6] : nullptr)))
      return e;
    if (tev && (e = record_timing(tev[1], st))) return e;
    if (tev && (e = record_timing(tev[2], st))) return e;
    if ((e = launch_lanczos_update(g, f64, w->lz, vec, st, pvar, tev ? tev[5] : nullptr))) return e;
    if (tev && (e = record_timing(tev[3], st))) return e;
    return cudaSuccess;
  };
  // a chunk = one step launched directly on the stream, then a CUDA graph of the chunk's other
  // steps (re-captured when they change). The chunks alternate between two graphs, each recording
  // timing events (tev[q]) around the two kernels of its middle step, so the sampled launches are
  // steady-state ones inside a busy stream; a chunk without a graph records them around its first
  // step instead.
  bool use_graph = p->use_graphs != 0 && chunk > 1;
  if (use_graph && !(w->graph[0] && w->graph[1] && w->gchunk == chunk && w->g_mw == p->m_W && w->g_mu == p->mu &&
                     w->g_lf == lf && w->g_var == pvar)) {
    const int mid = std::max(1, chunk / 2);
    for (int q = 0; q < 2; ++q) {
      if (w->graph[q]) cudaGraphExecDestroy(w->graph[q]);
      w->graph[q] = nullptr;
      cudaGraph_t gr;
      OVL_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      for (int i = 1; i < chunk && e == cudaSuccess; ++i) e = step(i == mid ? w->tev[q] : nullptr);
      cudaError_t e2 = cudaStreamEndCapture(st, &gr);
      if (e != cudaSuccess) {
        set_error("apply_sign: capture failed: %s", cudaGetErrorString(e));
        return OVL_ECUDA;
      }
      OVL_CHECK_CUDA(e2);
      e = cudaGraphInstantiate(&w->graph[q], gr, 0);
      cudaGraphDestroy(gr);
      OVL_CHECK_CUDA(e);
    }
    w->gchunk = chunk;
    w->g_mw = p->m_W;
    w->g_mu = p->mu;
    w->g_lf = lf;
    w->g_var = pvar;
  }
  int launches = 1 + (m > 0 ? 1 : 0) + 1;  // start (+ deflation dots) and the combine
  // the chunk's steps, then the finish of a deferred last step (before the scalars are read)
  auto run_steps = [&](int nsteps, int q) -> cudaError_t {
    launches += lanczos_step_launches(g, lf, f64, pvar) * nsteps + lanczos_settle_launches(f64, pvar);
    const bool graph = use_graph && nsteps == chunk;
    cudaError_t e = step(graph ? nullptr : w->tev[q]);
    if (e != cudaSuccess) return e;
    if (graph) {
      if ((e = cudaGraphLaunch(w->graph[q], st))) return e;
    } else {
      for (int i = 1; i < nsteps; ++i)
        if ((e = step(nullptr)) != cudaSuccess) return e;
    }
    return launch_lanczos_settle(g, f64, w->lz, st, pvar);
  };
  double t_pair = 0, t_upd = 0, t_fin = 0;
  int nsamp = 0;
  auto sample = [&](int q) {  // durations of the sampled step of the chunk behind slot q
    float a = 0, b = 0, f0 = 0, fa = 0, fb = 0;
    if (cudaEventElapsedTime(&a, w->tev[q][6], w->tev[q][4]) == cudaSuccess &&
        cudaEventElapsedTime(&b, w->tev[q][2], w->tev[q][5]) == cudaSuccess &&
        cudaEventElapsedTime(&f0, w->tev[q][0], w->tev[q][6]) == cudaSuccess &&
        cudaEventElapsedTime(&fa, w->tev[q][4], w->tev[q][1]) == cudaSuccess &&
        cudaEventElapsedTime(&fb, w->tev[q][5], w->tev[q][3]) == cudaSuccess) {
      t_pair += a;
      t_upd += b;
      t_fin += f0 + fa + fb;
      ++nsamp;
    }
    cudaGetLastError();  // a failed timing query must not surface as a launch error later
  };
  std::vector<RhsState> rs(nrhs);
  double t_small = 0;
  int queued = 0;  // steps queued on the device
  cudaEvent_t evc[2];
  OVL_CHECK_CUDA(cudaEventCreateWithFlags(&evc[0], cudaEventDisableTiming));
  OVL_CHECK_CUDA(cudaEventCreateWithFlags(&evc[1], cudaEventDisableTiming));
  int evq[2] = {0, 0};  // steps covered by the snapshot in each mirror slot
  int next_slot = 0;
  std::vector<int> pending;  // slots whose copies are in flight, oldest first
  const bool fixed = p->fixed_k > 0;
  auto launch_chunk = [&]() -> cudaError_t {
    int ns = std::min(chunk, kmax - queued);
    int q = next_slot;
    next_slot ^= 1;
    cudaError_t e = run_steps(ns, q);
    if (e) return e;
    queued += ns;
    if ((e = queue_scalar_copies(w, q, st))) return e;
    evq[q] = queued;
    if ((e = cudaEventRecord(evc[q], st))) return e;
    pending.push_back(q);
    return cudaSuccess;
  };
  ovl_status result = OVL_OK;
  cudaError_t ce = cudaSuccess;
  int qlast = 0;
  bool any_running = true;  // a chunk launched while some rhs ran did real work
  if (fixed) {
    while (queued < kmax && ce == cudaSuccess) {
      int ns = std::min(chunk, kmax - queued);
      ce = run_steps(ns, queued == 0 ? 0 : 1);
      queued += ns;
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) sample(0);
    if (ce == cudaSuccess) ce = queue_scalar_copies(w, 0, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    for (int r = 0; r < nrhs && ce == cudaSuccess; ++r) {
      ovl_status s = evaluate_rhs(w, 0, r, rs[r], &t_small);
      rs[r].status = s != OVL_OK ? s : (w->h[0].status[r] == 1 && rs[r].k < kmax ? OVL_EBREAKDOWN : OVL_OK);
      rs[r].est = 0;
      rs[r].done = true;
    }
  } else {
    ce = launch_chunk();
    while (ce == cudaSuccess) {
      // keep one more chunk queued while the host evaluates the oldest snapshot
      if (queued < kmax && pending.size() < 2) {
        ce = launch_chunk();
        if (ce) break;
      }
      int q = pending.front();
      pending.erase(pending.begin());
      ce = cudaEventSynchronize(evc[q]);
      if (ce) break;
      if (any_running) sample(q);
      qlast = q;
      const bool final_snapshot = evq[q] >= kmax;
      const int jq = evq[q];
      std::vector<int> todo;  // rhs due for an evaluation of sign(H_j) e_1 at this snapshot
      for (int r = 0; r < nrhs; ++r)
        if (!rs[r].done && stop_due(rs[r].trk, jq, final_snapshot, w->h[q].status[r] != 0)) todo.push_back(r);
      if (todo.empty()) {
        any_running = false;
        for (int r = 0; r < nrhs; ++r) any_running = any_running || w->h[q].status[r] == 0;
        continue;
      }
      bool all_done = true;
      std::vector<ovl_status> es_r(nrhs, OVL_OK);
      std::vector<int> evaluated;
      if (todo.size() <= 1) {
        for (int r : todo) es_r[r] = evaluate_rhs(w, q, r, rs[r], &t_small);
      } else {  // several right-hand sides: their sign(H_k) e_1 are independent, run them side by side
        std::vector<double> ts(nrhs, 0.0);
        std::vector<std::thread> th;
        const int conc = (int)todo.size();
        for (int r : todo)
          th.emplace_back([&, r] {
            set_sign_concurrency(conc);
            es_r[r] = evaluate_rhs(w, q, r, rs[r], &ts[r]);
          });
        for (auto& t : th) t.join();
        double tmax = 0;
        for (double t : ts) tmax = std::max(tmax, t);
        t_small += tmax;
      }
      for (int r : todo)
        if (es_r[r] == OVL_OK) evaluated.push_back(r);
      {
        ovl_status est_st = estimate_changes(w, g, f64, vec, q, rs, evaluated);
        if (est_st != OVL_OK) return est_st;
      }
      for (int r : todo) {
        RhsState& s = rs[r];
        ovl_status es = es_r[r];
        if (es != OVL_OK && !final_snapshot && w->h[q].status[r] == 0) {
          // this H_j defeated every small-sign route (a Ritz value near the imaginary axis, which
          // later steps may move away): keep the last good y and evaluate again later
          s.trk.next = stop_next_eval(jq, chunk, -1.0);
          continue;
        }
        bool converged = false;
        if (es == OVL_OK && w->h[q].status[r] == 0) {
          stop_record(s.trk, s.k, s.est < 1e299 ? s.est : -1.0);
          s.est = s.trk.err;
          converged = stop_converged(s.trk, p->tol);
          stop_schedule(s.trk, jq, chunk, p->tol);
        }
        if (es != OVL_OK) {
          s.status = es;
          s.done = true;
        } else if (w->h[q].status[r] == 3) {
          s.status = OVL_OK;
          s.done = true;
        } else if (w->h[q].status[r] == 1) {
          s.status = OVL_EBREAKDOWN;
          s.done = true;
        } else if (converged) {
          s.status = OVL_OK;
          s.done = true;
        } else if (final_snapshot) {
          s.status = OVL_ENOCONV;
          s.done = true;
        }
        if (s.done && w->h[q].status[r] == 0) {
          // retire this right-hand side: later steps skip it (any nonzero status)
          ce = cudaMemsetAsync(w->lz.status + r, 2, sizeof(int), st);
          if (ce) break;
        }
      }
      for (int r = 0; r < nrhs; ++r) all_done = all_done && rs[r].done;
      any_running = false;
      for (int r = 0; r < nrhs; ++r) any_running = any_running || w->h[q].status[r] == 0;
      if (all_done || ce) break;
    }
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaEventDestroy(evc[0]);
  cudaEventDestroy(evc[1]);
  if (ce != cudaSuccess) {
    set_error("apply_sign: CUDA error in the Lanczos loop: %s", cudaGetErrorString(ce));
    return OVL_ECUDA;
  }
  const DirectWS::Mirror& hm = w->h[qlast];
  // combine: x = x_P + beta V_k y with coef_j = beta0 y_j sv_j
  std::vector<double2> coef((size_t)nrhs * kmax, make_double2(0, 0));
  const size_t ks = (size_t)kmax + 2;
  lat->last_alpha.assign(nrhs, {});
  lat->last_beta.assign(nrhs, {});
  lat->last_delta.assign(nrhs, {});
  for (int r = 0; r < nrhs; ++r) {
    RhsState& s = rs[r];
    double b0 = hm.beta0[r];
    for (int i = 0; i < s.k; ++i) {
      std::complex<double> c = b0 * s.y[i] * hm.sv[r * ks + i + 1];
      coef[(size_t)r * kmax + i] = make_double2(c.real(), c.imag());
    }
    for (int i = 0; i < s.k; ++i) {
      double2 a = hm.alpha[r * ks + i + 1];
      lat->last_alpha[r].push_back(a.x);
      lat->last_alpha[r].push_back(a.y);
      if (i + 1 < s.k) {
        double2 bb = hm.beta[r * ks + i + 1];
        lat->last_beta[r].push_back(bb.x);
        lat->last_beta[r].push_back(bb.y);
        lat->last_delta[r].push_back(hm.delta[r * ks + i + 1]);
        lat->last_delta[r].push_back(0.0);
      }
    }
    if (s.status != OVL_OK && result == OVL_OK) result = s.status;
  }
  // coefficients and per-rhs k travel in one pinned upload
  std::vector<int> kr(nrhs);
  for (int r = 0; r < nrhs; ++r) kr[r] = rs[r].k;
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->coef, coef.data(), coef.size() * 16, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->kr, kr.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
  double2* xd = p->host_io ? w->xdev : x;
  if (!two_pass) {
    OVL_CHECK_CUDA(launch_lanczos_combine(g, f64, w->lz, vec, w->kr, w->coef, kmax, xd, st));
  } else {
    // second pass (the two-pass strategy of Section 2.3): the same start and steps regenerate
    // vhat_1..vhat_k bit for bit (fixed-order reductions), and each column is added to x with its
    // coefficient as it appears; a right-hand side retires once its k columns are in
    std::vector<double2> xc((size_t)nrhs * ks, make_double2(0, 0));
    int kmax2 = 0;
    for (int r = 0; r < nrhs; ++r) {
      for (int i = 0; i < rs[r].k; ++i) xc[(size_t)r * ks + i + 1] = coef[(size_t)r * kmax + i];
      kmax2 = std::max(kmax2, rs[r].k);
    }
    OVL_CHECK_CUDA(cudaMemcpyAsync(w->xcoef, xc.data(), xc.size() * 16, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(cudaMemsetAsync(w->xacc, 0, (size_t)nrhs * n * 16, st));
    LzDev lz2 = w->lz;
    lz2.xacc = w->xacc;
    lz2.xcoef = w->xcoef;
    OVL_CHECK_CUDA(launch_lanczos_start(g, f64, lz2, vec, bd, m, lat->src()->defl.R, lat->src()->defl.L, w->lam_sign,
                                        w->dots, st));
    launches += 1 + (m > 0 ? 1 : 0);
    auto retire = [&](int jdone) -> cudaError_t {  // rhs whose last column is jdone
      for (int r = 0; r < nrhs; ++r)
        if (rs[r].k == jdone) {
          cudaError_t e = cudaMemsetAsync(w->lz.status + r, 2, sizeof(int), st);
          if (e != cudaSuccess) return e;
        }
      return cudaSuccess;
    };
    OVL_CHECK_CUDA(retire(1));
    for (int j = 1; j < kmax2; ++j) {  // step j adds column j + 1
      OVL_CHECK_CUDA(launch_lanczos_pair(g, U, lf, f64, p->m_W, p->mu, lz2, vec, st, pvar));
      OVL_CHECK_CUDA(launch_lanczos_update(g, f64, lz2, vec, st, pvar));
      launches += lanczos_step_launches(g, lf, f64, pvar);
      OVL_CHECK_CUDA(retire(j + 1));
    }
    OVL_CHECK_CUDA(launch_lanczos_settle(g, f64, lz2, st, pvar));
    launches += lanczos_settle_launches(f64, pvar);
    OVL_CHECK_CUDA(launch_ms_finish(g, nrhs, w->xacc, vec.xp, xd, st));
  }
  if (p->host_io) OVL_CHECK_CUDA(cudaMemcpyAsync(x, w->xdev, (size_t)nrhs * n * 16, cudaMemcpyDeviceToHost, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  double t_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (info) {
    for (int r = 0; r < nrhs; ++r) {
      info[r].status = rs[r].status;
      info[r].iterations = rs[r].k;
      info[r].matvecs = 2 * rs[r].k;
      info[r].poles = 0;
      info[r].est_error = rs[r].est;
      info[r].t_total_ms = t_total;
      info[r].t_small_ms = t_small;
      info[r].residual = 0;
      info[r].t_kernel_ms = nsamp ? t_pair / nsamp : 0;
      info[r].t_update_ms = nsamp ? t_upd / nsamp : 0;
      info[r].t_finish_ms = nsamp ? t_fin / nsamp : 0;
      info[r].kernel_samples = nsamp;
      info[r].kernel_launches = launches;
      info[r].evaluations = rs[r].evals;
      info[r].ritz_evaluations = rs[r].ritz;
    }
  }
  if (lat->server_mode) {  // the server accounts device memory per request
    free_direct_ws(lat->dws);
    lat->dws = nullptr;
  }
  if (result != OVL_OK) set_error("apply_sign: at least one right-hand side ended with status %d", result);
  return result;
}

size_t direct_footprint(int vol, int nrhs, int kmax, bool f64, bool two_pass) {
  const size_t n = (size_t)12 * vol, elt = f64 ? 16 : 8;
  if (two_pass) kmax = 2;  // three basis columns in a rotating window, plus the FP64 accumulator of x
  const size_t xacc = two_pass ? n * 16 : 0;
  const size_t slots = (n + kVecBlock - 1) / kVecBlock + kMaxFillSMs;  // partial_slots
  return (size_t)nrhs * ((size_t)(kmax + 1) * n * elt + 4 * n * elt + 3 * n * 16 + xacc + 16 * slots * 32) +
         ((size_t)1 << 20);
}

}  // namespace ovl
