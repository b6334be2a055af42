// Host driver of restarted FOM-LR(m, k) for x = sign(H_W(mu)) b (Algorithm 1, Section 4.1, with
// Section 5's rational sign g(t) = t sum_i omega_i / (t^2 - sigma_i)):
//   x_P = R sign(Lambda) L^H b;  r = (I - P) b;  rho_i = 1;  X = 0
//   per cycle: beta = |r|, v_1 = r / beta, k Arnoldi steps on A = H_W^2 (GPU: two stencils and two
//   classical Gram-Schmidt passes per step, one CUDA graph per cycle);
//   y_i = beta rho_i (H_k - sigma_i)^-1 e_1 (host, FP64, Givens QR of the Hessenberg matrix);
//   X += V_k sum_i omega_i y_i;  rho_i = -h_{k+1,k} e_k^T y_i;  r = (I - P) v_{k+1}
//   until |rho_i| |r| <= tol |r_0| for every shift; then x = x_P + H_W X (FP64 stencil).
// One Krylov basis serves all shifts and, because the shifted residuals stay collinear with
// v_{k+1}, a restart is again a rational function with the same poles (no instability). The
// orthonormal (Arnoldi) basis does not degrade where two-sided Lanczos loses biorthogonality.
#include <chrono>
#include <complex>

#include "kernels_fom.h"

namespace ovl {

ovl_status rational_coefficients(const ovl_sign_params* p, std::vector<double>& om, std::vector<double>& sg,
                                 double* bound);

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

using zc = std::complex<double>;

// y = (H - sigma I)^-1 (c e_1) for the kk x kk upper Hessenberg H (column-major, leading dimension
// ld): Givens rotations reduce it to upper triangular form, then back substitution. O(kk^2).
void hessenberg_solve(int kk, const double2* H, int ld, double sigma, zc c, zc* y) {
  std::vector<zc> a((size_t)kk * kk), rhs(kk, 0.0);
  for (int j = 0; j < kk; ++j)
    for (int i = 0; i < kk; ++i) {
      const double2 h = i <= j + 1 ? H[(size_t)j * ld + i] : make_double2(0, 0);
      a[(size_t)j * kk + i] = i <= j + 1 ? zc(h.x, h.y) - (i == j ? sigma : 0.0) : zc(0.0);
    }
  rhs[0] = c;
  for (int j = 0; j + 1 < kk; ++j) {  // rotate rows j, j+1 to zero a(j+1, j)
    const zc x = a[(size_t)j * kk + j], z = a[(size_t)j * kk + j + 1];
    const double r = std::hypot(std::abs(x), std::abs(z));
    if (r == 0.0) continue;
    const zc cs = x / r, sn = z / r;  // [conj(cs) conj(sn); -sn cs] [x; z] = [r; 0]
    for (int q = j; q < kk; ++q) {
      const zc u = a[(size_t)q * kk + j], v = a[(size_t)q * kk + j + 1];
      a[(size_t)q * kk + j] = std::conj(cs) * u + std::conj(sn) * v;
      a[(size_t)q * kk + j + 1] = -sn * u + cs * v;
    }
    const zc u = rhs[j], v = rhs[j + 1];
    rhs[j] = std::conj(cs) * u + std::conj(sn) * v;
    rhs[j + 1] = -sn * u + cs * v;
  }
  for (int i = kk - 1; i >= 0; --i) {
    zc s = rhs[i];
    for (int q = i + 1; q < kk; ++q) s -= a[(size_t)q * kk + i] * y[q];
    y[i] = s / a[(size_t)i * kk + i];
  }
}

}  // namespace

ovl_status solve_fom(ovl_lattice* lat, const ovl_sign_params* p, int nrhs, const double2* b, double2* x,
                     ovl_sign_info* info, cudaStream_t user_stream) {
  auto t_start = std::chrono::steady_clock::now();
  const bool f64 = p->precision == OVL_PREC_F64;
  const int lf = p->precision == OVL_PREC_F32_F16LINKS ? LINK_F16R12 : (f64 ? LINK_F64 : LINK_F32);
  const ovl_lattice* F = lat->src();
  OVL_REQUIRE(F->u64, "apply_sign: links not set");
  OVL_REQUIRE(f64 || (lf == LINK_F32 ? F->u32 != nullptr : F->u16 != nullptr),
              "apply_sign: links not set in the format this precision needs (ovl_set_links formats)");
  const int k = p->restart_k > 0 ? p->restart_k : 40;
  OVL_REQUIRE(k >= 2 && k <= kFomMaxK, "apply_sign: restart_k must be in [2, %d]", kFomMaxK);
  OVL_REQUIRE(p->k_max >= 1, "apply_sign: k_max must be >= 1");
  std::vector<double> om, sg;
  double bound = 0;
  OVL_TRY(rational_coefficients(p, om, sg, &bound));
  const int s = (int)om.size();
  int m = 0;
  if (p->use_deflation) {
    OVL_REQUIRE(F->defl.m > 0, "apply_sign: use_deflation but no deflation set");
    OVL_REQUIRE(F->defl.m_w == p->m_W && F->defl.mu == p->mu,
                "apply_sign: deflation set was computed for (m_W, mu) = (%g, %g)", F->defl.m_w, F->defl.mu);
    m = F->defl.m;
  }
  const Geom& g = lat->g;
  const size_t n = (size_t)12 * g.vol, elt = f64 ? 16 : 8, nr = (size_t)nrhs;
  const int max_cycles = (p->k_max + k - 1) / k;
  // ---- workspace: one stream-ordered block for the call
  cudaStream_t st = nullptr;
  OVL_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  FomDev f;
  f.n = n;
  f.nrhs = nrhs;
  f.kcap = k;
  f.nblk = fom_partial_slots(n);
  f.pstride = 2 * (k + 1);
  const int dblk = (int)((n + kBlock - 1) / kBlock);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al256(bytes);
    return o;
  };
  const size_t o_V = take((size_t)(k + 1) * nr * n * elt), o_t = take(nr * n * elt), o_X = take(nr * n * 16),
               o_xp = take(nr * n * 16), o_ax = take(nr * n * 16), o_H = take(nr * k * (k + 1) * 16),
               o_c1 = take(nr * (k + 1) * 16), o_c2 = take(nr * (k + 1) * 16),
               o_pa = take(nr * f.nblk * f.pstride * 8), o_sc = take(nr * 8), o_be = take(nr * 8),
               o_st = take(nr * 4), o_kd = take(nr * 4), o_co = take(nr * (k + 1) * 16), o_kr = take(nr * 4),
               o_do = take(nr * 2 * std::max(m, 1) * 16), o_ls = take((size_t)std::max(m, 1) * 8),
               o_dp = take(nr * std::max(m, 1) * std::max<size_t>(dblk, (g.vol + kBlock - 1) / kBlock) * 4 * 8),
               o_dc = take(nr * 4), o_pd = take(nr * std::max(m, 1) * 16), o_bd = take(nr * n * 16),
               o_xd = take(nr * n * 16);
  char* base = nullptr;
  cudaEvent_t order;  // the call's work follows the caller's stream
  OVL_CHECK_CUDA(cudaEventCreateWithFlags(&order, cudaEventDisableTiming));
  OVL_CHECK_CUDA(cudaEventRecord(order, user_stream));
  OVL_CHECK_CUDA(cudaStreamWaitEvent(st, order, 0));
  cudaEventDestroy(order);
  if (cudaMallocAsync((void**)&base, off, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(st);
    set_error("apply_sign: cannot allocate %zu bytes of device workspace", off);
    return OVL_ENOMEM;
  }
  struct Cleanup {
    char* base;
    cudaStream_t st;
    ~Cleanup() {
      cudaFreeAsync(base, st);
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  } cleanup{base, st};
  f.V = base + o_V;
  f.H = (double2*)(base + o_H);
  f.c1 = (double2*)(base + o_c1);
  f.c2 = (double2*)(base + o_c2);
  f.part = (double*)(base + o_pa);
  f.scale = (double*)(base + o_sc);
  f.beta = (double*)(base + o_be);
  f.status = (int*)(base + o_st);
  f.kdone = (int*)(base + o_kd);
  void* tmp = base + o_t;
  double2 *X = (double2*)(base + o_X), *xp = (double2*)(base + o_xp), *ax = (double2*)(base + o_ax);
  double2* coef = (double2*)(base + o_co);
  int* kr = (int*)(base + o_kr);
  double2* dots = (double2*)(base + o_do);
  double* lam_sign = (double*)(base + o_ls);
  double* dpart = (double*)(base + o_dp);
  unsigned* dcount = (unsigned*)(base + o_dc);
  double2* pd = (double2*)(base + o_pd);
  OVL_CHECK_CUDA(cudaMemsetAsync(f.status, 0, nr * 4, st));
  OVL_CHECK_CUDA(cudaMemsetAsync(dcount, 0, nr * 4, st));
  const double2* bd = b;
  if (p->host_io) {
    OVL_CHECK_CUDA(cudaMemcpyAsync(base + o_bd, b, nr * n * 16, cudaMemcpyHostToDevice, st));
    bd = (const double2*)(base + o_bd);
  }
  if (m > 0) {
    std::vector<double> ls(m);
    for (int i = 0; i < m; ++i) ls[i] = F->defl.lam[2 * i] >= 0 ? 1.0 : -1.0;
    OVL_CHECK_CUDA(cudaMemcpyAsync(lam_sign, ls.data(), m * 8, cudaMemcpyHostToDevice, st));
  }
  const Links U = F->links();
  int launches = 0;
  // ---- start: x_P, r = (I - P) b into v_0, beta_0 = |r|, v_0 = r / beta_0
  OVL_CHECK_CUDA(launch_fom_start(g, f64, f, bd, m, F->defl.R, F->defl.L, lam_sign, dots, dpart, dcount,
                                  m > 0 ? xp : nullptr, X, st));
  OVL_CHECK_CUDA(launch_fom_gs(f, f64, -1, 2, st));
  OVL_CHECK_CUDA(launch_fom_scale(f, f64, -1, st));
  launches += (m > 0 ? 1 : 0) + 1 + 2 + 1;
  std::vector<double> beta(nr), r0(nr);
  OVL_CHECK_CUDA(cudaMemcpyAsync(beta.data(), f.beta, nr * 8, cudaMemcpyDeviceToHost, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  r0 = beta;
  // the batched reduced-precision stencil picks its link-group size on its first call (it
  // synchronises): make that call before the cycle is captured
  OVL_CHECK_CUDA(launch_dslash(g, U, lf, f64, p->m_W, p->mu, false, true, true, true, nrhs, f.V, tmp, st));
  // ---- one cycle of k Arnoldi steps, captured once and replayed
  auto arnoldi_step = [&](int j, cudaEvent_t* ev) -> cudaError_t {
    cudaError_t e;
    void* vj = (char*)f.V + (size_t)j * nr * n * elt;
    void* vn = (char*)f.V + (size_t)(j + 1) * nr * n * elt;
    if (ev && (e = cudaEventRecord(ev[0], st))) return e;
    if ((e = launch_dslash(g, U, lf, f64, p->m_W, p->mu, false, true, true, true, nrhs, vj, tmp, st))) return e;
    if ((e = launch_dslash(g, U, lf, f64, p->m_W, p->mu, false, true, true, true, nrhs, tmp, vn, st))) return e;
    if (ev && (e = cudaEventRecord(ev[1], st))) return e;
    for (int pass = 0; pass < 3; ++pass)
      if ((e = launch_fom_gs(f, f64, j, pass, st))) return e;
    if ((e = launch_fom_scale(f, f64, j, st))) return e;
    if (ev && (e = cudaEventRecord(ev[2], st))) return e;
    return cudaSuccess;
  };
  const int per_step = 2 + 2 * 3 - 1 + 1;  // two stencils, three passes (+ their reductions), the scale
  cudaEvent_t tev[3];
  for (auto& e : tev) OVL_CHECK_CUDA(cudaEventCreate(&e));
  cudaGraphExec_t gexec = nullptr;
  struct GraphCleanup {
    cudaGraphExec_t* g;
    cudaEvent_t* ev;
    ~GraphCleanup() {
      if (*g) cudaGraphExecDestroy(*g);
      for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
    }
  } gcleanup{&gexec, tev};
  const bool use_graph = p->use_graphs != 0;
  std::vector<zc> rho((size_t)nr * s, zc(1.0)), ybuf(k);
  std::vector<double2> Hh((size_t)nr * k * (k + 1)), ch((size_t)nr * (k + 1));
  std::vector<int> kd(nr), sth(nr), done(nr, 0), cycles(nr, 0);
  std::vector<double> resid(nr, 0.0);
  for (size_t r = 0; r < nr; ++r)
    if (!(r0[r] > 0)) done[r] = 1;  // b lies in the deflated space: x = x_P
  double t_pair = 0, t_gs = 0;
  int nsamp = 0;
  int cyc = 0;
  for (; cyc < max_cycles; ++cyc) {
    bool any = false;
    for (size_t r = 0; r < nr; ++r) any = any || !done[r];
    if (!any) break;
    if (cyc == 0 || !use_graph) {  // the first cycle directly, with events around the middle step
      for (int j = 0; j < k; ++j) OVL_CHECK_CUDA(arnoldi_step(j, j == k / 2 ? tev : nullptr));
      if (use_graph) {
        cudaGraph_t gr;
        OVL_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int j = 0; j < k && e == cudaSuccess; ++j) e = arnoldi_step(j, nullptr);
        cudaError_t e2 = cudaStreamEndCapture(st, &gr);
        OVL_CHECK_CUDA(e);
        OVL_CHECK_CUDA(e2);
        e = cudaGraphInstantiate(&gexec, gr, 0);
        cudaGraphDestroy(gr);
        OVL_CHECK_CUDA(e);
      }
    } else {
      OVL_CHECK_CUDA(cudaGraphLaunch(gexec, st));
    }
    launches += k * per_step;
    OVL_CHECK_CUDA(cudaMemcpyAsync(Hh.data(), f.H, Hh.size() * 16, cudaMemcpyDeviceToHost, st));
    OVL_CHECK_CUDA(cudaMemcpyAsync(kd.data(), f.kdone, nr * 4, cudaMemcpyDeviceToHost, st));
    OVL_CHECK_CUDA(cudaMemcpyAsync(sth.data(), f.status, nr * 4, cudaMemcpyDeviceToHost, st));
    OVL_CHECK_CUDA(cudaStreamSynchronize(st));
    if (cyc == 0) {
      float a = 0, c = 0;
      if (cudaEventElapsedTime(&a, tev[0], tev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&c, tev[1], tev[2]) == cudaSuccess) {
        t_pair += a;
        t_gs += c;
        ++nsamp;
      }
      cudaGetLastError();
    }
    // shifted Hessenberg solves, the combination of this cycle and the new collinearity factors
    std::fill(ch.begin(), ch.end(), make_double2(0, 0));
    std::vector<int> krh(nr, 0);
    for (size_t r = 0; r < nr; ++r) {
      if (done[r]) continue;
      ++cycles[r];
      const int kk = std::max(1, std::min(kd[r], k));
      krh[r] = kk;
      const double2* Hr = Hh.data() + (size_t)r * k * (k + 1);
      const double hlast = sth[r] == 1 ? 0.0 : Hr[(size_t)(kk - 1) * (k + 1) + kk].x;
      std::vector<zc> acc(kk, 0.0);
      for (int i = 0; i < s; ++i) {
        hessenberg_solve(kk, Hr, k + 1, sg[i], beta[r] * rho[r * s + i], ybuf.data());
        for (int q = 0; q < kk; ++q) acc[q] += om[i] * ybuf[q];
        rho[r * s + i] = -hlast * ybuf[kk - 1];
      }
      for (int q = 0; q < kk; ++q) ch[r * (k + 1) + q] = make_double2(acc[q].real(), acc[q].imag());
      if (sth[r] == 1) done[r] = 1;  // invariant subspace: the iterates are exact
    }
    OVL_CHECK_CUDA(cudaMemcpyAsync(coef, ch.data(), ch.size() * 16, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(cudaMemcpyAsync(kr, krh.data(), nr * 4, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(launch_fom_combine(f, f64, kr, coef, X, st));
    // restart: v_0 = (I - P) v_k, beta = |v_0|; a system has converged when |rho_i| beta <= tol |r_0|
    std::vector<int> stn(nr);
    for (size_t r = 0; r < nr; ++r) stn[r] = done[r] ? 2 : 0;
    OVL_CHECK_CUDA(cudaMemcpyAsync(f.status, stn.data(), nr * 4, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(launch_fom_restart(g, f64, f, k, m, F->defl.R, F->defl.L, dpart, dcount, pd, st));
    OVL_CHECK_CUDA(launch_fom_gs(f, f64, -1, 2, st));
    OVL_CHECK_CUDA(cudaMemcpyAsync(beta.data(), f.beta, nr * 8, cudaMemcpyDeviceToHost, st));
    OVL_CHECK_CUDA(cudaStreamSynchronize(st));
    launches += 1 + (m > 0 ? 2 : 1) + 2;
    for (size_t r = 0; r < nr; ++r) {
      if (done[r]) continue;
      double worst = 0;
      for (int i = 0; i < s; ++i) worst = std::max(worst, std::abs(rho[r * s + i]) * beta[r]);
      resid[r] = worst / r0[r];
      if (worst <= p->tol * r0[r]) done[r] = 1;
    }
    for (size_t r = 0; r < nr; ++r) stn[r] = done[r] ? 2 : 0;
    OVL_CHECK_CUDA(cudaMemcpyAsync(f.status, stn.data(), nr * 4, cudaMemcpyHostToDevice, st));
    OVL_CHECK_CUDA(launch_fom_scale(f, f64, -1, st));
    launches += 1;
  }
  // x = x_P + H_W X: one FP64 stencil with the FP64 links, then the canonical layout
  OVL_CHECK_CUDA(launch_dslash(g, U, LINK_F64, true, p->m_W, p->mu, false, true, true, true, nrhs, X, ax, st));
  double2* xd = p->host_io ? (double2*)(base + o_xd) : x;
  OVL_CHECK_CUDA(launch_ms_finish(g, nrhs, ax, m > 0 ? xp : nullptr, xd, st));
  launches += 2;
  if (p->host_io) OVL_CHECK_CUDA(cudaMemcpyAsync(x, xd, nr * n * 16, cudaMemcpyDeviceToHost, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  const double t_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  ovl_status result = OVL_OK;
  for (size_t r = 0; r < nr; ++r) {
    const ovl_status sr = done[r] ? OVL_OK : OVL_ENOCONV;
    if (sr != OVL_OK && result == OVL_OK) result = sr;
    if (info) {
      std::memset(&info[r], 0, sizeof(ovl_sign_info));
      info[r].status = sr;
      info[r].iterations = cycles[r] * k;
      info[r].matvecs = 2 * cycles[r] * k;
      info[r].poles = s;
      info[r].residual = resid[r];
      info[r].est_error = resid[r] + bound;
      info[r].t_total_ms = t_total;
      info[r].t_kernel_ms = nsamp ? t_pair / nsamp : 0;
      info[r].t_update_ms = nsamp ? t_gs / nsamp : 0;
      info[r].kernel_samples = nsamp;
      info[r].kernel_launches = launches;
      info[r].evaluations = cycles[r];
    }
  }
  if (result != OVL_OK) set_error("apply_sign: at least one right-hand side ended with status %d", result);
  return result;
}

}  // namespace ovl
