// Host driver of BiCG-LR(m) with a rational sign approximation (Algorithm 3, Section 5):
//   x_P = R f(Lambda) L^H b;  r = (I - P) b;  shadow r~ = b - L R^H b;
//   multishift BiCG for (A^2 - sigma_i) x^(i) = r, i = 1..s (all systems share one Krylov
//   space of M = A^2; footnote of Section 6: FOM/BiCG on Eq. pfe_s works with A^2);
//   x = x_P + A sum_i omega_i x^(i)   (g(A) r with g(t) = t sum_i omega_i / (t^2 - sigma_i)).
// Stopping rule (Section 6): every shifted residual below tol relative to |r|; shifts are
// retired individually. Coefficients: Neuberger (Eq. pfe_s; s and c from Eq. no_of_poles with
// the circle through spec_lo, spec_hi), Zolotarev on [spec_lo, spec_hi], or caller-given.
#include <algorithm>
#include <chrono>

#include "kernels.h"

namespace ovl {

void neuberger(int s, double c, double* omega, double* sigma);
void neuberger_for_spectrum(double lo, double hi, double eps, int* s_out, double* c_out, double* d_out);
double neuberger_bound(int s, double d);
double zolotarev(int n, double lo, double hi, double* omega, double* sigma);

struct MultiWS {
  int nrhs = 0, s = 0, f64 = -1, vol = 0, m = 0, prio = 0;
  bool refine = false;
  // refinement (reliable updates): the correction systems (A^2 - sigma_i) e = r^(i) of up to
  // `grp` (rhs, shift) pairs are solved as one batch; per system: FP64 residual, two stencil
  // temporaries and a canonical copy (native layout), its FP32 BiCG state (gms / gv), its seed
  // shift and tolerance; plus the single-pole coefficients {1}, {0} and the shifts sigma_i
  int grp = 0;
  double2 *res = nullptr, *t1 = nullptr, *t2 = nullptr, *ecan = nullptr;
  double *rpart = nullptr, *rout = nullptr, *one_zero = nullptr, *sg_all = nullptr, *gsig = nullptr, *gtol = nullptr;
  unsigned* rcount = nullptr;
  MsDev gms;
  MsVecs gv;
  double* h_gout = nullptr;  // pinned [grp] squared residual norms
  int* h_gst = nullptr;      // pinned [2][grp] statuses of the correction solves (two chunks in flight)
  cudaGraphExec_t rgraph = nullptr;  // one chunk of correction iterations for rg_gn systems
  int rg_gn = -1, rg_chunk = 0, rg_lf = -1;
  double rg_mw = 0, rg_mu = 0;
  MsDev ms;
  MsVecs v;
  char* dev = nullptr;
  double2* dots = nullptr;
  double* lam_sign = nullptr;
  double* omega = nullptr;
  double* dsig = nullptr;
  double2* ax = nullptr;
  double2* bdev = nullptr;
  double2* xdev = nullptr;
  int* h_status = nullptr;  // pinned [2][nrhs] status + [2][nrhs] k
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // alternating chunks, each with its events
  cudaEvent_t tev[2][4] = {};
  int gchunk = 0, g_lf = -1;
  int g_var = -1, rg_var = -1;  // the pair-stencil shape the graphs were captured with
  double g_mw = 0, g_mu = 0, g_s1 = 0, g_tol = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

void free_multi_ws(MultiWS* w) {
  if (!w) return;
  if (w->rgraph) cudaGraphExecDestroy(w->rgraph);
  for (int q = 0; q < 2; ++q) {
    if (w->graph[q]) cudaGraphExecDestroy(w->graph[q]);
    for (auto e : w->tev[q])
      if (e) cudaEventDestroy(e);
  }
  if (w->dev) cudaFreeAsync(w->dev, w->stream);
  if (w->h_status) cudaFreeHost(w->h_status);
  if (w->h_gout) cudaFreeHost(w->h_gout);
  if (w->h_gst) cudaFreeHost(w->h_gst);
  if (w->stream) cudaStreamDestroy(w->stream);
  for (auto e : w->ev)
    if (e) cudaEventDestroy(e);
  delete w;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static ovl_status ensure_mws(ovl_lattice* lat, int nrhs, int s, bool f64, int m, bool refine, int prio) {
  MultiWS* w = lat->mws;
  const int vol = lat->g.vol;
  if (w && w->nrhs == nrhs && w->s == s && w->f64 == (int)f64 && w->vol == vol && w->m >= m && w->refine == refine &&
      w->prio == prio)
    return OVL_OK;
  free_multi_ws(w);
  lat->mws = nullptr;
  w = new MultiWS();
  w->nrhs = nrhs;
  w->s = s;
  w->f64 = f64;
  w->vol = vol;
  w->m = m;
  w->refine = refine;
  w->prio = prio;
  const size_t n = (size_t)12 * vol, elt = f64 ? 16 : 8;
  const int nblk = partial_slots(lat->g);
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += al256(b);
    return o;
  };
  size_t o_vec[8];
  for (int i = 0; i < 8; ++i) o_vec[i] = take((size_t)nrhs * n * elt);
  size_t o_ps = take((size_t)nrhs * s * n * elt);
  size_t o_X = take((size_t)nrhs * n * 16);
  size_t o_xp = take((size_t)nrhs * n * 16);
  size_t o_ax = take((size_t)nrhs * n * 16);
  size_t o_bd = take((size_t)nrhs * n * 16);
  size_t o_xd = take((size_t)nrhs * n * 16);
  size_t o_k = take((size_t)nrhs * 4);
  size_t o_st = take((size_t)nrhs * 4);
  size_t o_seed = take((size_t)nrhs * 8 * 16);
  size_t o_z = take((size_t)nrhs * s * 3 * 16);
  size_t o_a = take((size_t)nrhs * s * 16);
  size_t o_b = take((size_t)nrhs * s * 16);
  size_t o_act = take((size_t)nrhs * s * 4);
  size_t o_om = take((size_t)s * 8);
  size_t o_ds = take((size_t)s * 8);
  size_t o_pa = take((size_t)nrhs * std::max(m, 1) * nblk * 4 * 8);
  size_t o_cn = take((size_t)nrhs * 4);
  size_t o_do = take((size_t)nrhs * 2 * std::max(m, 1) * 16);
  size_t o_ls = take((size_t)std::max(m, 1) * 8);
  const size_t rn = refine ? n : 0;
  // correction batch: at most kRefineGroup systems and about kRefineBytes of buffers
  // (per system 9 FP32 vectors + 5 FP64 vectors)
  const size_t per_sys = n * (9 * 8 + 5 * 16);
  size_t ref_bytes = kRefineBytes;
  if (refine) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) ref_bytes = std::min(ref_bytes, free_b / 4);
  }
  // one batch for all (rhs, shift) systems when they fit: converged systems cost nothing, so the
  // batch runs as long as its hardest system, once
  const int grp = refine ? (int)std::max<size_t>(1, std::min<size_t>({(size_t)nrhs * s, (size_t)kRefineGroup,
                                                                       ref_bytes / per_sys}))
                         : 0;
  const size_t gq = (size_t)grp;
  size_t o_xs = take((size_t)nrhs * s * rn * 16), o_r64 = take((size_t)nrhs * rn * 16);
  size_t o_res = take(gq * rn * 16), o_t1 = take(gq * rn * 16), o_t2 = take(gq * rn * 16), o_ec = take(gq * rn * 16);
  size_t o_rp = take(std::max<size_t>(1, gq) * vec_blocks(lat->g) * 8), o_ro = take(std::max<size_t>(1, gq) * 8),
         o_oz = take(16), o_rc = take(std::max<size_t>(1, gq) * 4);
  size_t o_gvec[9];
  for (int i = 0; i < 9; ++i) o_gvec[i] = take(gq * rn * 8);
  size_t o_gX = take(gq * rn * 16), o_gk = take(gq * 4), o_gst = take(gq * 4), o_gseed = take(gq * 8 * 16),
         o_gz = take(gq * 3 * 16), o_ga = take(gq * 16), o_gb = take(gq * 16), o_gact = take(gq * 4),
         o_gpa = take(gq * nblk * 4 * 8), o_gcn = take(gq * 4), o_sga = take((size_t)s * 8), o_gsig = take(gq * 8),
         o_gtol = take(gq * 8);
  int least = 0, greatest = 0;  // stream priority as in the direct driver
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (cudaStreamCreateWithPriority(&w->stream, cudaStreamNonBlocking, std::max(greatest, least - std::max(0, prio))) !=
      cudaSuccess) {
    delete w;
    set_error("apply_sign: cannot create a stream");
    return OVL_ECUDA;
  }
  cudaError_t e = cudaMallocAsync((void**)&w->dev, off, w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) {
    cudaStreamDestroy(w->stream);
    delete w;
    set_error("apply_sign: cannot allocate %zu bytes of device workspace: %s", off, cudaGetErrorString(e));
    return OVL_ENOMEM;
  }
  char* b = w->dev;
  void** vp[8] = {&w->v.r, &w->v.rt, &w->v.p, &w->v.pt, &w->v.t, &w->v.tt, &w->v.q, &w->v.qt};
  for (int i = 0; i < 8; ++i) *vp[i] = b + o_vec[i];
  w->v.ps = b + o_ps;
  w->v.X = (double2*)(b + o_X);
  w->v.xp = (double2*)(b + o_xp);
  w->ax = (double2*)(b + o_ax);
  w->bdev = (double2*)(b + o_bd);
  w->xdev = (double2*)(b + o_xd);
  MsDev& ms = w->ms;
  ms.nrhs = nrhs;
  ms.s = s;
  ms.nblk = nblk;
  ms.k = (int*)(b + o_k);
  ms.status = (int*)(b + o_st);
  ms.seed = (double2*)(b + o_seed);
  ms.zeta = (double2*)(b + o_z);
  ms.ash = (double2*)(b + o_a);
  ms.bsh = (double2*)(b + o_b);
  ms.active = (int*)(b + o_act);
  w->omega = (double*)(b + o_om);
  w->dsig = (double*)(b + o_ds);
  ms.omega = w->omega;
  ms.dsig = w->dsig;
  ms.part = (double*)(b + o_pa);
  ms.count = (unsigned*)(b + o_cn);
  w->dots = (double2*)(b + o_do);
  w->lam_sign = (double*)(b + o_ls);
  w->grp = grp;
  if (refine) {
    w->v.xs = (double2*)(b + o_xs);
    w->v.r64 = (double2*)(b + o_r64);
    w->res = (double2*)(b + o_res);
    w->t1 = (double2*)(b + o_t1);
    w->t2 = (double2*)(b + o_t2);
    w->ecan = (double2*)(b + o_ec);
    void** gp[9] = {&w->gv.r, &w->gv.rt, &w->gv.p, &w->gv.pt, &w->gv.t, &w->gv.tt, &w->gv.q, &w->gv.qt, &w->gv.ps};
    for (int i = 0; i < 9; ++i) *gp[i] = b + o_gvec[i];
    w->gv.X = (double2*)(b + o_gX);
    MsDev& gm = w->gms;
    gm.nrhs = grp;
    gm.s = 1;
    gm.nblk = nblk;
    gm.k = (int*)(b + o_gk);
    gm.status = (int*)(b + o_gst);
    gm.seed = (double2*)(b + o_gseed);
    gm.zeta = (double2*)(b + o_gz);
    gm.ash = (double2*)(b + o_ga);
    gm.bsh = (double2*)(b + o_gb);
    gm.active = (int*)(b + o_gact);
    gm.part = (double*)(b + o_gpa);
    gm.count = (unsigned*)(b + o_gcn);
    w->sg_all = (double*)(b + o_sga);
    w->gsig = (double*)(b + o_gsig);
    w->gtol = (double*)(b + o_gtol);
    gm.sig1v = w->gsig;
    gm.tolv = w->gtol;
  }
  w->rpart = (double*)(b + o_rp);
  w->rout = (double*)(b + o_ro);
  w->one_zero = (double*)(b + o_oz);
  w->rcount = (unsigned*)(b + o_rc);
  const double oz[2] = {1.0, 0.0};
  bool ev_ok = true;
  for (int q = 0; q < 2; ++q)
    for (int i = 0; i < 4; ++i) ev_ok = ev_ok && cudaEventCreate(&w->tev[q][i]) == cudaSuccess;
  w->gms.omega = w->one_zero;
  w->gms.dsig = w->one_zero + 1;
  if (!ev_ok || cudaMemsetAsync(ms.count, 0, (size_t)nrhs * 4, w->stream) != cudaSuccess ||
      cudaMemsetAsync(w->rcount, 0, std::max<size_t>(1, gq) * 4, w->stream) != cudaSuccess ||
      (grp > 0 && cudaMemsetAsync(w->gms.count, 0, gq * 4, w->stream) != cudaSuccess) ||
      (grp > 0 && cudaMallocHost(&w->h_gout, gq * 8) != cudaSuccess) ||
      (grp > 0 && cudaMallocHost(&w->h_gst, 2 * gq * 4) != cudaSuccess) ||
      cudaMemcpy(w->one_zero, oz, 16, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMallocHost(&w->h_status, (size_t)4 * nrhs * sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    free_multi_ws(w);
    set_error("apply_sign: cannot set up the multishift workspace");
    return OVL_ECUDA;
  }
  lat->mws = w;
  return OVL_OK;
}

// Rational coefficients for the call; returns the approximation's own error bound. Shared with the
// restarted FOM driver.
ovl_status rational_coefficients(const ovl_sign_params* p, std::vector<double>& om, std::vector<double>& sg,
                                 double* bound) {
  if (p->rational_kind == OVL_RAT_CUSTOM) {
    OVL_REQUIRE(p->s >= 1 && p->s <= kMaxShifts && p->omega && p->sigma, "apply_sign: custom rational needs s, omega, sigma");
    om.assign(p->omega, p->omega + p->s);
    sg.assign(p->sigma, p->sigma + p->s);
    for (double x : sg) OVL_REQUIRE(x <= 0, "apply_sign: shifts must satisfy sigma_i <= 0");
    *bound = 0;
    return OVL_OK;
  }
  OVL_REQUIRE(p->spec_lo > 0 && p->spec_hi > p->spec_lo,
              "apply_sign: the rational variant needs spectrum bounds 0 < spec_lo < spec_hi");
  if (p->rational_kind == OVL_RAT_NEUBERGER) {
    int s;
    double c, d;
    neuberger_for_spectrum(p->spec_lo, p->spec_hi, std::max(p->tol, 1e-15), &s, &c, &d);
    if (p->s > 0) s = p->s;
    OVL_REQUIRE(s <= kMaxShifts, "apply_sign: %d poles needed (max %d)", s, kMaxShifts);
    om.resize(s);
    sg.resize(s);
    neuberger(s, c, om.data(), sg.data());
    *bound = neuberger_bound(s, d);
    return OVL_OK;
  }
  if (p->rational_kind == OVL_RAT_ZOLOTAREV) {
    OVL_REQUIRE(p->s >= 1 && p->s <= kMaxShifts, "apply_sign: Zolotarev needs 1 <= s <= %d", kMaxShifts);
    om.resize(p->s);
    sg.resize(p->s);
    *bound = zolotarev(p->s, p->spec_lo, p->spec_hi, om.data(), sg.data());
    return OVL_OK;
  }
  set_error("apply_sign: unknown rational_kind %d", p->rational_kind);
  return OVL_EINVAL;
}

ovl_status solve_multishift(ovl_lattice* lat, const ovl_sign_params* p, int nrhs, const double2* b, double2* x,
                            ovl_sign_info* info, cudaStream_t user_stream) {
  auto t0 = std::chrono::steady_clock::now();
  const bool f64 = p->precision == OVL_PREC_F64;
  const int lf = p->precision == OVL_PREC_F32_F16LINKS ? LINK_F16R12 : (f64 ? LINK_F64 : LINK_F32);
  OVL_REQUIRE(lat->src()->u64, "apply_sign: links not set");
  OVL_REQUIRE(f64 || (lf == LINK_F32 ? lat->src()->u32 != nullptr : lat->src()->u16 != nullptr),
              "apply_sign: links not set in the format this precision needs (ovl_set_links formats)");
  OVL_REQUIRE(p->k_max >= 1 && p->k_max <= 1000000, "apply_sign: k_max must be in [1, 1e6]");
  std::vector<double> om, sg;
  double bound = 0;
  OVL_TRY(rational_coefficients(p, om, sg, &bound));
  const int s = (int)om.size();
  int m = 0;
  if (p->use_deflation) {
    OVL_REQUIRE(lat->src()->defl.m > 0, "apply_sign: use_deflation but no deflation set");
    OVL_REQUIRE(lat->src()->defl.m_w == p->m_W && lat->src()->defl.mu == p->mu,
                "apply_sign: deflation set was computed for (m_W, mu) = (%g, %g)", lat->src()->defl.m_w, lat->src()->defl.mu);
    m = lat->src()->defl.m;
  }
  // FP32 iterations reach about 1e-6; below that each shifted system is refined with FP64
  // residuals (reliable updates): x^(i) kept in FP64, r^(i) = r - (A^2 - sigma_i) x^(i) from the
  // FP64 stencil, corrections from FP32 single-shift BiCG solves on the same kernels
  const bool refine = !f64 && p->tol < kFp32Floor;
  OVL_TRY(ensure_mws(lat, nrhs, s, f64, m, refine, p->priority));
  MultiWS* w = lat->mws;
  cudaStream_t st = w->stream;
  const Geom& g = lat->g;
  const size_t n = (size_t)12 * g.vol;
  // seed shift: the one closest to 0 (the hardest system); others relative to it
  double s1 = *std::max_element(sg.begin(), sg.end());
  std::vector<double> ds(s);
  for (int i = 0; i < s; ++i) ds[i] = sg[i] - s1;
  MsDev ms = w->ms;
  ms.sigma1 = s1;
  ms.tol = refine ? kFp32Floor : p->tol;
  OVL_CHECK_CUDA(cudaEventRecord(w->ev[0], user_stream));
  OVL_CHECK_CUDA(cudaStreamWaitEvent(st, w->ev[0], 0));
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->omega, om.data(), s * 8, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(cudaMemcpyAsync(w->dsig, ds.data(), s * 8, cudaMemcpyHostToDevice, st));
  const double2* bd = b;
  if (p->host_io) {
    OVL_CHECK_CUDA(cudaMemcpyAsync(w->bdev, b, (size_t)nrhs * n * 16, cudaMemcpyHostToDevice, st));
    bd = w->bdev;
  }
  std::vector<double> ls(std::max(m, 1));
  for (int i = 0; i < m; ++i) ls[i] = lat->src()->defl.lam[2 * i] >= 0 ? 1.0 : -1.0;
  if (m > 0) OVL_CHECK_CUDA(cudaMemcpyAsync(w->lam_sign, ls.data(), m * 8, cudaMemcpyHostToDevice, st));
  MsVecs v = w->v;
  if (m == 0) v.xp = nullptr;
  if (!refine) v.xs = v.r64 = nullptr;
  OVL_CHECK_CUDA(launch_ms_start(g, f64, ms, v, bd, m, lat->src()->defl.R, lat->src()->defl.L, w->lam_sign, w->dots, st));
  const Links U = lat->src()->links();
  const int chunk = std::max(1, std::min(p->check_every > 0 ? p->check_every : 20, p->k_max));
  const bool use_graph = p->use_graphs != 0 && chunk > 1;
  // the chunks alternate between two graphs; graph q records timing events (tev[q]) around its
  // middle iteration, so the sampled launches are steady-state ones inside a busy stream
  const int gvar = ms_pair_split(g, f64 ? 0 : lf) ? 1 : 0;  // the stencil shape the graphs launch
  if (use_graph && !(w->graph[0] && w->graph[1] && w->gchunk == chunk && w->g_lf == lf && w->g_mw == p->m_W &&
                     w->g_mu == p->mu && w->g_s1 == s1 && w->g_tol == ms.tol && w->g_var == gvar)) {
    const int mid = std::max(1, chunk / 2);
    for (int q = 0; q < 2; ++q) {
      if (w->graph[q]) cudaGraphExecDestroy(w->graph[q]);
      w->graph[q] = nullptr;
      cudaGraph_t gr;
      OVL_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      for (int i = 1; i < chunk && e == cudaSuccess; ++i)
        e = launch_ms_step(g, U, lf, f64, p->m_W, p->mu, ms, v, st, i == mid ? w->tev[q] : nullptr);
      cudaError_t e2 = cudaStreamEndCapture(st, &gr);
      OVL_CHECK_CUDA(e);
      OVL_CHECK_CUDA(e2);
      e = cudaGraphInstantiate(&w->graph[q], gr, 0);
      cudaGraphDestroy(gr);
      OVL_CHECK_CUDA(e);
    }
    w->gchunk = chunk;
    w->g_lf = lf;
    w->g_var = gvar;
    w->g_mw = p->m_W;
    w->g_mu = p->mu;
    w->g_s1 = s1;
    w->g_tol = ms.tol;
  }
  int launches = 1 + (m > 0 ? 1 : 0) + 2;  // start (+ deflation dots), final stencil and finish
  // a chunk = one iteration launched directly, then a graph of the rest (events: see above)
  auto run_chunk = [&](int ns, int q) -> cudaError_t {
    launches += 4 * ns;
    const bool graph = use_graph && ns == chunk;
    cudaError_t e = launch_ms_step(g, U, lf, f64, p->m_W, p->mu, ms, v, st, graph ? nullptr : w->tev[q]);
    if (e != cudaSuccess || ns == 1) return e;
    if (graph) return cudaGraphLaunch(w->graph[q], st);
    for (int i = 1; i < ns; ++i)
      if ((e = launch_ms_step(g, U, lf, f64, p->m_W, p->mu, ms, v, st)) != cudaSuccess) return e;
    return cudaSuccess;
  };
  double t_pair = 0, t_upd = 0;
  int nsamp = 0;
  auto sample = [&](int q) {
    float a = 0, b = 0;
    if (cudaEventElapsedTime(&a, w->tev[q][0], w->tev[q][1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, w->tev[q][2], w->tev[q][3]) == cudaSuccess) {
      t_pair += a;
      t_upd += b;
      ++nsamp;
    }
    cudaGetLastError();  // a failed timing query must not surface as a launch error later
  };
  // chunks with status snapshots; one chunk stays queued while the host looks at the last
  int queued = 0, slot = 0;
  std::vector<int> pend;
  cudaError_t ce = cudaSuccess;
  auto launch = [&]() -> cudaError_t {
    int ns = std::min(chunk, p->k_max - queued);
    cudaError_t e = run_chunk(ns, slot);
    if (e) return e;
    queued += ns;
    int* hs = w->h_status + (size_t)slot * 2 * nrhs;
    if ((e = cudaMemcpyAsync(hs, ms.status, nrhs * 4, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(hs + nrhs, ms.k, nrhs * 4, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaEventRecord(w->ev[slot], st))) return e;
    pend.push_back(slot);
    slot ^= 1;
    return cudaSuccess;
  };
  ce = launch();
  bool done = false, any_running = true;
  while (ce == cudaSuccess && !done) {
    if (queued < p->k_max && pend.size() < 2) {
      ce = launch();
      if (ce) break;
    }
    int q = pend.front();
    pend.erase(pend.begin());
    ce = cudaEventSynchronize(w->ev[q]);
    if (ce) break;
    if (any_running) sample(q);
    const int* hs = w->h_status + (size_t)q * 2 * nrhs;
    done = true;
    for (int r = 0; r < nrhs; ++r)
      if (hs[r] == 0) done = false;
    any_running = !done;
    if (pend.empty() && queued >= p->k_max) done = true;
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    set_error("apply_sign: CUDA error in the multishift loop: %s", cudaGetErrorString(ce));
    return OVL_ECUDA;
  }
  // final state, per-shift residual estimates
  std::vector<int> hst(nrhs), hk(nrhs), act((size_t)nrhs * s);
  std::vector<double2> seed((size_t)nrhs * 8), zeta((size_t)nrhs * s * 3);
  OVL_CHECK_CUDA(cudaMemcpy(hst.data(), ms.status, nrhs * 4, cudaMemcpyDeviceToHost));
  OVL_CHECK_CUDA(cudaMemcpy(hk.data(), ms.k, nrhs * 4, cudaMemcpyDeviceToHost));
  OVL_CHECK_CUDA(cudaMemcpy(act.data(), ms.active, act.size() * 4, cudaMemcpyDeviceToHost));
  OVL_CHECK_CUDA(cudaMemcpy(seed.data(), ms.seed, seed.size() * 16, cudaMemcpyDeviceToHost));
  OVL_CHECK_CUDA(cudaMemcpy(zeta.data(), ms.zeta, zeta.size() * 16, cudaMemcpyDeviceToHost));
  // ---- reliable updates of every shifted system (reduced precision below kFp32Floor)
  int ref_sweeps = 0, ref_iters = 0;
  double ref_worst = 0;
  if (refine) {
    // The (rhs, shift) systems j = rhs*s + i are refined in batches of up to grp: per sweep, the
    // FP64 residuals r^(i) = r - (A^2 - sigma_i) x^(i) of the batch (two FP64 stencils over the
    // batch), then for the systems above tol one batched FP32 BiCG solve of
    // (A^2 - sigma_i) e = r^(i) (each system its own shift and relative target), x^(i) += e.
    // Systems already converged get a zero right-hand side, which the solve skips.
    const int total = nrhs * s, grp = w->grp;
    // the correction solves run with FP32 links when the field has them: with FP16 12-real links
    // the operator itself is off by ~1e-3, which would cap what one correction sweep can gain
    const int lf_ref = lat->src()->u32 ? LINK_F32 : lf;
    OVL_CHECK_CUDA(launch_ff_to_f64((size_t)total * n, v.xs, st));
    launches += 1;
    MsDev gm = w->gms;
    MsVecs gvv = w->gv;
    gvv.xs = gvv.r64 = gvv.xp = nullptr;
    OVL_CHECK_CUDA(cudaMemcpyAsync(w->sg_all, sg.data(), s * 8, cudaMemcpyHostToDevice, st));
    std::vector<double> gsig(grp), gtol(grp);
    for (int j0 = 0; j0 < total; j0 += grp) {
      const int gn = std::min(grp, total - j0);
      gm.nrhs = gn;
      double2* xg = v.xs + (size_t)j0 * n;
      std::vector<double> resn(gn, 0.0), r0(gn);
      for (int j = 0; j < gn; ++j) r0[j] = seed[(size_t)((j0 + j) / s) * 8 + 4].x;
      for (int sweep = 0;; ++sweep) {
        OVL_CHECK_CUDA(launch_dslash(g, U, LINK_F64, true, p->m_W, p->mu, false, true, true, true, gn, xg, w->t1, st));
        OVL_CHECK_CUDA(launch_dslash(g, U, LINK_F64, true, p->m_W, p->mu, false, true, true, true, gn, w->t1, w->t2, st));
        OVL_CHECK_CUDA(launch_ms_residual_batch(g, j0, gn, s, v.r64, w->t2, xg, w->sg_all, w->res, w->rpart,
                                                w->rcount, w->rout, st));
        launches += 3;
        OVL_CHECK_CUDA(cudaMemcpyAsync(w->h_gout, w->rout, gn * 8, cudaMemcpyDeviceToHost, st));
        OVL_CHECK_CUDA(cudaStreamSynchronize(st));
        int need = 0;
        for (int j = 0; j < gn; ++j) {
          resn[j] = std::sqrt(w->h_gout[j]);
          if (resn[j] > p->tol * r0[j]) ++need;
        }
        if (need == 0 || sweep >= kMaxRefineSweeps) break;
        ++ref_sweeps;
        for (int j = 0; j < gn; ++j) {
          const bool above = resn[j] > p->tol * r0[j];
          gsig[j] = sg[(j0 + j) % s];
          // the FP32 iteration only needs to take this system's residual below tol
          gtol[j] = above ? std::max(2.0 * kFp32Floor, std::min(0.5, 0.3 * p->tol * r0[j] / resn[j])) : 0.5;
          if (!above) OVL_CHECK_CUDA(cudaMemsetAsync(w->res + (size_t)j * n, 0, n * 16, st));
        }
        OVL_CHECK_CUDA(cudaMemcpyAsync(w->gsig, gsig.data(), gn * 8, cudaMemcpyHostToDevice, st));
        OVL_CHECK_CUDA(cudaMemcpyAsync(w->gtol, gtol.data(), gn * 8, cudaMemcpyHostToDevice, st));
        OVL_CHECK_CUDA(launch_from_native(g, gn, true, w->res, true, w->ecan, st));
        OVL_CHECK_CUDA(launch_ms_start(g, false, gm, gvv, w->ecan, 0, nullptr, nullptr, nullptr, nullptr, st));
        launches += 2;
        // chunks of correction iterations, a CUDA graph per (batch size, chunk); two chunks in
        // flight so the host's status check overlaps the next chunk (finished systems skip it)
        const bool rg = p->use_graphs != 0 && chunk > 1;
        const int rvar = ms_pair_split(g, lf_ref) ? 1 : 0;  // the corrections run in FP32
        if (rg && !(w->rgraph && w->rg_gn == gn && w->rg_chunk == chunk && w->rg_lf == lf_ref && w->rg_mw == p->m_W &&
                    w->rg_mu == p->mu && w->rg_var == rvar)) {
          if (w->rgraph) cudaGraphExecDestroy(w->rgraph);
          w->rgraph = nullptr;
          cudaGraph_t gr;
          OVL_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
          cudaError_t e = cudaSuccess;
          for (int q = 0; q < chunk && e == cudaSuccess; ++q)
            e = launch_ms_step(g, U, lf_ref, false, p->m_W, p->mu, gm, gvv, st);
          cudaError_t e2 = cudaStreamEndCapture(st, &gr);
          OVL_CHECK_CUDA(e);
          OVL_CHECK_CUDA(e2);
          e = cudaGraphInstantiate(&w->rgraph, gr, 0);
          cudaGraphDestroy(gr);
          OVL_CHECK_CUDA(e);
          w->rg_gn = gn;
          w->rg_chunk = chunk;
          w->rg_lf = lf_ref;
          w->rg_var = rvar;
          w->rg_mw = p->m_W;
          w->rg_mu = p->mu;
        }
        int it = 0, slot = 0;
        std::vector<int> inflight;
        auto queue_chunk = [&]() -> cudaError_t {
          const int ns = std::min(chunk, p->k_max - it);
          cudaError_t e = cudaSuccess;
          if (rg && ns == chunk) {
            e = cudaGraphLaunch(w->rgraph, st);
          } else {
            for (int q = 0; q < ns && e == cudaSuccess; ++q)
              e = launch_ms_step(g, U, lf_ref, false, p->m_W, p->mu, gm, gvv, st);
          }
          if (e) return e;
          it += ns;
          launches += 4 * ns;
          if ((e = cudaMemcpyAsync(w->h_gst + (size_t)slot * grp, gm.status, gn * 4, cudaMemcpyDeviceToHost, st)))
            return e;
          if ((e = cudaEventRecord(w->ev[slot], st))) return e;
          inflight.push_back(slot);
          slot ^= 1;
          return cudaSuccess;
        };
        OVL_CHECK_CUDA(queue_chunk());
        while (!inflight.empty()) {
          if (it < p->k_max && inflight.size() < 2) OVL_CHECK_CUDA(queue_chunk());
          const int q = inflight.front();
          inflight.erase(inflight.begin());
          OVL_CHECK_CUDA(cudaEventSynchronize(w->ev[q]));
          bool running = false;
          for (int j = 0; j < gn; ++j) running = running || w->h_gst[(size_t)q * grp + j] == 0;
          if (!running) break;
        }
        // iterations actually run (a chunk queued after the last system finished skips them all)
        OVL_CHECK_CUDA(cudaMemcpyAsync(w->h_gst, gm.k, gn * 4, cudaMemcpyDeviceToHost, st));
        OVL_CHECK_CUDA(cudaStreamSynchronize(st));
        int kmax_run = 0;
        for (int j = 0; j < gn; ++j) kmax_run = std::max(kmax_run, w->h_gst[j]);
        ref_iters += kmax_run;
        OVL_CHECK_CUDA(launch_axpy_f64_masked(g, gn, gm.status, gvv.X, xg, st));
        launches += 1;
      }
      for (int j = 0; j < gn; ++j) ref_worst = std::max(ref_worst, r0[j] > 0 ? resn[j] / r0[j] : 0.0);
    }
    OVL_CHECK_CUDA(launch_ms_combine_shifts(g, nrhs, s, w->omega, v.xs, v.X, st));
    launches += 1;
  }
  // x = x_P + A X (FP64 stencil, native layout)
  OVL_CHECK_CUDA(launch_dslash(g, U, LINK_F64, true, p->m_W, p->mu, false, true, true, true, nrhs, v.X, w->ax, st));
  double2* xd = p->host_io ? w->xdev : x;
  OVL_CHECK_CUDA(launch_ms_finish(g, nrhs, w->ax, v.xp, xd, st));
  if (p->host_io) OVL_CHECK_CUDA(cudaMemcpyAsync(x, w->xdev, (size_t)nrhs * n * 16, cudaMemcpyDeviceToHost, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  double t_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  ovl_status result = OVL_OK;
  for (int r = 0; r < nrhs; ++r) {
    int stt = hst[r];
    double r0 = seed[(size_t)r * 8 + 4].x, rn = seed[(size_t)r * 8 + 4].y;
    double worst = 0;
    for (int i = 0; i < s; ++i) {
      double2 z = zeta[((size_t)r * s + i) * 3 + 1];
      if (r0 > 0) worst = std::max(worst, std::sqrt(z.x * z.x + z.y * z.y) * rn / r0);
    }
    ovl_status rs = (stt == 2 || stt == 3 || stt == 4) ? OVL_OK : (stt == 1 ? OVL_EBREAKDOWN : OVL_ENOCONV);
    if (stt == 0) {
      bool all = true;
      for (int i = 0; i < s; ++i) all = all && act[(size_t)r * s + i] != 1;
      if (all) rs = OVL_OK;
    }
    if (refine) {  // the refined true residuals decide
      worst = ref_worst;
      rs = ref_worst <= p->tol ? OVL_OK : OVL_ENOCONV;
    }
    if (rs != OVL_OK && result == OVL_OK) result = rs;
    if (info) {
      info[r].status = rs;
      info[r].iterations = hk[r] + ref_iters;
      info[r].matvecs = 4 * (hk[r] + ref_iters) + 1 + 2 * (ref_sweeps + s);
      info[r].poles = s;
      info[r].est_error = (stt == 3 ? 0.0 : worst) + bound;
      info[r].t_total_ms = t_total;
      info[r].t_small_ms = 0;
      info[r].residual = worst;
      info[r].t_kernel_ms = nsamp ? t_pair / nsamp : 0;
      info[r].t_update_ms = nsamp ? t_upd / nsamp : 0;
      info[r].kernel_samples = nsamp;
      info[r].kernel_launches = launches;
      info[r].evaluations = 0;
      info[r].ritz_evaluations = 0;
    }
  }
  if (lat->server_mode) {  // the server accounts device memory per request
    free_multi_ws(lat->mws);
    lat->mws = nullptr;
  }
  if (result != OVL_OK) set_error("apply_sign: at least one right-hand side ended with status %d", result);
  return result;
}

// Device bytes of one multishift solve (the workspace of ensure_mws, the correction batch at its
// largest), for the server's admission.
size_t multishift_footprint(int vol, int nrhs, int s, bool f64, bool refine) {
  const size_t n = (size_t)12 * vol, elt = f64 ? 16 : 8, nr = (size_t)nrhs;
  const size_t slots = (n + kVecBlock - 1) / kVecBlock + kMaxFillSMs;  // partial_slots
  size_t b = nr * n * (8 * elt + (size_t)s * elt + 5 * 16) + nr * 16 * slots * 32;  // (deflation dots: m <= 16)
  if (refine) {
    const size_t gq = std::min<size_t>(nr * s, kRefineGroup);
    b += nr * s * n * 16 + nr * n * 16 + gq * n * (4 * 16 + 9 * 8 + 16) + gq * slots * 32;
  }
  return b + ((size_t)1 << 20);
}

}  // namespace ovl
