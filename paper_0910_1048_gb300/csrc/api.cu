// C ABI entry points (include/ovl.h): context, lattice, links, deflation, D_W, sign solves.
#include <cstdarg>
#include <mutex>
#include <cstdlib>
#include <vector>

#include "kernels.h"

namespace ovl {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

ovl_status solve_direct(ovl_lattice* lat, const ovl_sign_params* p, int nrhs, const double2* b, double2* x,
                        ovl_sign_info* info, cudaStream_t st);
ovl_status solve_multishift(ovl_lattice* lat, const ovl_sign_params* p, int nrhs, const double2* b, double2* x,
                            ovl_sign_info* info, cudaStream_t st);
ovl_status solve_fom(ovl_lattice* lat, const ovl_sign_params* p, int nrhs, const double2* b, double2* x,
                     ovl_sign_info* info, cudaStream_t st);

// A lattice with its own workspaces that reads `parent`'s links and deflation set at every solve
// (so it sees later ovl_set_links / ovl_set_deflation on the parent).
ovl_lattice* lattice_view(ovl_lattice* parent) {
  ovl_lattice* v = new ovl_lattice();
  v->ctx = parent->ctx;
  v->g = parent->g;
  v->parent = parent;
  v->owns_links = false;
  v->server_mode = true;
  return v;
}

}  // namespace ovl

using namespace ovl;

extern "C" {

const char* ovl_last_error(void) { return g_err; }

const char* ovl_version(void) { return "ovl 1.0 sm_103a"; }

ovl_status ovl_set_pair_variant(int64_t volume, int32_t precision, int32_t variant) {
  clear_error();
  OVL_REQUIRE(volume >= 1 && volume <= (int64_t(1) << 26), "ovl_set_pair_variant: volume out of range");
  OVL_REQUIRE(precision >= OVL_PREC_F64 && precision <= OVL_PREC_F32_F16LINKS,
              "ovl_set_pair_variant: unknown precision %d", precision);
  OVL_REQUIRE(variant >= -1 && variant < ovl::kPairVariants, "ovl_set_pair_variant: variant %d outside -1..%d",
              variant, ovl::kPairVariants - 1);
  static_assert(OVL_PREC_F64 == ovl::LINK_F64 && OVL_PREC_F32 == ovl::LINK_F32 &&
                    OVL_PREC_F32_F16LINKS == ovl::LINK_F16R12,
                "the tuner's key is the link format of the precision");
  ovl::set_pair_variant((int)volume, precision, variant);
  return OVL_OK;
}

int32_t ovl_get_pair_variant(int64_t volume, int32_t precision) {
  if (volume < 1 || volume > (int64_t(1) << 26) || precision < OVL_PREC_F64 || precision > OVL_PREC_F32_F16LINKS)
    return -1;
  return ovl::tuned_pair_variant((int)volume, precision);
}

ovl_status ovl_ctx_create(int32_t device, ovl_ctx** out) {
  clear_error();
  OVL_REQUIRE(out != nullptr, "ovl_ctx_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  OVL_CHECK_CUDA(cudaGetDeviceCount(&ndev));
  OVL_REQUIRE(device >= 0 && device < ndev, "ovl_ctx_create: device %d not in [0, %d)", device, ndev);
  OVL_DEVICE_SCOPE(device);
  ovl_ctx* c = new ovl_ctx();
  c->device = device;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    set_error("ovl_ctx_create: %s", cudaGetErrorString(e));
    return OVL_ECUDA;
  }
  *out = c;
  return OVL_OK;
}

ovl_status ovl_ctx_destroy(ovl_ctx* ctx) {
  clear_error();
  if (!ctx) return OVL_OK;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return OVL_OK;
}

ovl_status ovl_create_lattice(ovl_ctx* ctx, const int32_t dims[4], int32_t t_bc, ovl_lattice** out) {
  clear_error();
  OVL_REQUIRE(ctx && dims && out, "ovl_create_lattice: NULL argument");
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    OVL_REQUIRE(dims[i] >= 2 && dims[i] % 2 == 0 && dims[i] <= 4096, "ovl_create_lattice: extent %d = %d must be even and >= 2",
                i, dims[i]);
  OVL_REQUIRE(t_bc == 1 || t_bc == -1, "ovl_create_lattice: t_bc must be +1 or -1");
  long long vol = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  OVL_REQUIRE(vol <= (1LL << 26), "ovl_create_lattice: volume %lld exceeds 2^26 sites", vol);
  ovl_lattice* l = new ovl_lattice();
  l->ctx = ctx;
  l->g.lx = dims[0];
  l->g.ly = dims[1];
  l->g.lz = dims[2];
  l->g.lt = dims[3];
  l->g.vol = (int)vol;
  l->g.sy = dims[0];
  l->g.sz = dims[0] * dims[1];
  l->g.st = dims[0] * dims[1] * dims[2];
  l->g.t_bc = t_bc;
  *out = l;
  return OVL_OK;
}

ovl_status ovl_destroy_lattice(ovl_lattice* lat) {
  clear_error();
  if (!lat) return OVL_OK;
  if (lat->servers.load() > 0) {
    set_error("ovl_destroy_lattice: the lattice is a field of a request server; destroy the server first");
    return OVL_EBUSY;
  }
  DeviceGuard dg(lat->ctx->device);
  free_direct_ws(lat->dws);
  free_multi_ws(lat->mws);
  if (lat->owns_links) {
    cudaFree(lat->u64);
    cudaFree(lat->u32);
    cudaFree(lat->u16);
    cudaFree(lat->defl.R);
    cudaFree(lat->defl.L);
  }
  delete lat;
  return OVL_OK;
}

int64_t ovl_lattice_n(const ovl_lattice* lat) { return lat ? (int64_t)12 * lat->g.vol : 0; }

ovl_status ovl_set_links(ovl_lattice* lat, const void* U, int32_t U_on_device, uint32_t formats) {
  clear_error();
  OVL_REQUIRE(lat && U, "ovl_set_links: NULL argument");
  OVL_REQUIRE((formats & ~(OVL_F64 | OVL_F32 | OVL_F16R12)) == 0, "ovl_set_links: unknown format bits 0x%x", formats);
  std::unique_lock<std::shared_mutex> excl(lat->guard, std::try_to_lock);
  if (!excl.owns_lock()) {
    set_error("ovl_set_links: a solve is using this lattice's links (retry when it has finished)");
    return OVL_EBUSY;
  }
  OVL_DEVICE_SCOPE(lat->ctx->device);
  const size_t nl = (size_t)36 * lat->g.vol;  // complex entries
  formats |= OVL_F64;
  // a copy held from an earlier call is refreshed too: no format may keep the previous field
  if (lat->u32) formats |= OVL_F32;
  if (lat->u16) formats |= OVL_F16R12;
  if (!lat->u64) OVL_CHECK_CUDA(cudaMalloc(&lat->u64, nl * 16));
  if ((formats & OVL_F32) && !lat->u32) OVL_CHECK_CUDA(cudaMalloc(&lat->u32, nl * 8));
  if ((formats & OVL_F16R12) && !lat->u16) OVL_CHECK_CUDA(cudaMalloc(&lat->u16, (size_t)24 * lat->g.vol * 4));
  const double* src = (const double*)U;
  double* tmp = nullptr;
  cudaStream_t st = lat->ctx->stream;
  if (!U_on_device) {
    OVL_CHECK_CUDA(cudaMalloc(&tmp, nl * 16));
    OVL_CHECK_CUDA(cudaMemcpyAsync(tmp, U, nl * 16, cudaMemcpyHostToDevice, st));
    src = tmp;
  }
  cudaError_t e = launch_ingest_links(lat->g, src, lat->u64, (formats & OVL_F32) ? lat->u32 : nullptr,
                                      (formats & OVL_F16R12) ? lat->u16 : nullptr, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (tmp) cudaFree(tmp);
  OVL_CHECK_CUDA(e);
  lat->formats |= formats;
  return OVL_OK;
}

ovl_status ovl_set_deflation(ovl_lattice* lat, double m_W, double mu, int32_t m, const void* R, const void* L,
                             const void* lambda, int32_t on_device) {
  clear_error();
  OVL_REQUIRE(lat, "ovl_set_deflation: NULL lattice");
  OVL_REQUIRE(m >= 0 && m <= 1024, "ovl_set_deflation: m must be in [0, 1024]");
  std::unique_lock<std::shared_mutex> excl(lat->guard, std::try_to_lock);
  if (!excl.owns_lock()) {
    set_error("ovl_set_deflation: a solve is using this lattice's deflation set (retry when it has finished)");
    return OVL_EBUSY;
  }
  OVL_DEVICE_SCOPE(lat->ctx->device);
  cudaFree(lat->defl.R);
  cudaFree(lat->defl.L);
  lat->defl = ovl_deflation();
  if (m == 0) return OVL_OK;
  OVL_REQUIRE(R && L && lambda, "ovl_set_deflation: NULL R, L or lambda");
  const size_t n = (size_t)12 * lat->g.vol;
  // biorthonormality check L^H R = I on the host (inputs are canonical complex128)
  std::vector<double> hr((size_t)m * n * 2), hl((size_t)m * n * 2), hlam(2 * (size_t)m);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  OVL_CHECK_CUDA(cudaMemcpy(hr.data(), R, hr.size() * 8, kind));
  OVL_CHECK_CUDA(cudaMemcpy(hl.data(), L, hl.size() * 8, kind));
  OVL_CHECK_CUDA(cudaMemcpy(hlam.data(), lambda, hlam.size() * 8, kind));
  double worst = 0;
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      double re = 0, im = 0;
      const double* la = &hl[(size_t)a * n * 2];
      const double* rb = &hr[(size_t)b * n * 2];
      for (size_t i = 0; i < n; ++i) {
        re += la[2 * i] * rb[2 * i] + la[2 * i + 1] * rb[2 * i + 1];
        im += la[2 * i] * rb[2 * i + 1] - la[2 * i + 1] * rb[2 * i];
      }
      double d = std::sqrt((re - (a == b)) * (re - (a == b)) + im * im);
      worst = std::max(worst, d);
    }
  OVL_REQUIRE(worst <= 1e-8, "ovl_set_deflation: max |L^H R - I| = %.3g > 1e-8", worst);
  double2 *dR = nullptr, *dL = nullptr, *tmp = nullptr;
  OVL_CHECK_CUDA(cudaMalloc(&dR, (size_t)m * n * 16));
  OVL_CHECK_CUDA(cudaMalloc(&dL, (size_t)m * n * 16));
  OVL_CHECK_CUDA(cudaMalloc(&tmp, (size_t)m * n * 16));
  cudaStream_t st = lat->ctx->stream;
  OVL_CHECK_CUDA(cudaMemcpyAsync(tmp, hr.data(), (size_t)m * n * 16, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(launch_to_native(lat->g, m, true, tmp, true, dR, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  OVL_CHECK_CUDA(cudaMemcpyAsync(tmp, hl.data(), (size_t)m * n * 16, cudaMemcpyHostToDevice, st));
  OVL_CHECK_CUDA(launch_to_native(lat->g, m, true, tmp, true, dL, st));
  OVL_CHECK_CUDA(cudaStreamSynchronize(st));
  cudaFree(tmp);
  lat->defl.m = m;
  lat->defl.m_w = m_W;
  lat->defl.mu = mu;
  lat->defl.R = dR;
  lat->defl.L = dL;
  lat->defl.lam = hlam;
  return OVL_OK;
}

ovl_status ovl_to_native(ovl_lattice* lat, int32_t dtype, int32_t nrhs, const void* in, void* out, void* stream) {
  clear_error();
  OVL_REQUIRE(lat && in && out && nrhs >= 1, "ovl_to_native: invalid arguments");
  OVL_REQUIRE(dtype == OVL_C128 || dtype == OVL_C64, "ovl_to_native: dtype");
  OVL_DEVICE_SCOPE(lat->ctx->device);
  bool f = dtype == OVL_C128;
  OVL_CHECK_CUDA(launch_to_native(lat->g, nrhs, f, in, f, out, (cudaStream_t)stream));
  return OVL_OK;
}

ovl_status ovl_from_native(ovl_lattice* lat, int32_t dtype, int32_t nrhs, const void* in, void* out, void* stream) {
  clear_error();
  OVL_REQUIRE(lat && in && out && nrhs >= 1, "ovl_from_native: invalid arguments");
  OVL_REQUIRE(dtype == OVL_C128 || dtype == OVL_C64, "ovl_from_native: dtype");
  OVL_DEVICE_SCOPE(lat->ctx->device);
  bool f = dtype == OVL_C128;
  OVL_CHECK_CUDA(launch_from_native(lat->g, nrhs, f, in, f, out, (cudaStream_t)stream));
  return OVL_OK;
}

ovl_status ovl_apply_DW(ovl_lattice* lat, double m_W, double mu, uint32_t flags, int32_t dtype, int32_t nrhs,
                        const void* in, void* out, void* stream) {
  clear_error();
  OVL_REQUIRE(lat && in && out && nrhs >= 1 && nrhs <= 65535, "ovl_apply_DW: invalid arguments");
  OVL_REQUIRE(in != out, "ovl_apply_DW: in and out must not alias");
  OVL_REQUIRE(dtype == OVL_C128 || dtype == OVL_C64, "ovl_apply_DW: dtype must be OVL_C128 or OVL_C64");
  OVL_REQUIRE((flags & ~(OVL_DAGGER | OVL_GAMMA5 | OVL_NATIVE | OVL_LINKS_F32 | OVL_LINKS_F16R12)) == 0,
              "ovl_apply_DW: unknown flags 0x%x", flags);
  OVL_REQUIRE(2.0 * m_W + 8.0 != 0.0, "ovl_apply_DW: m_W = -4 has no kappa");
  std::shared_lock<std::shared_mutex> shared(lat->src()->guard);
  OVL_DEVICE_SCOPE(lat->ctx->device);
  const bool f64 = dtype == OVL_C128;
  int lf = LINK_F64;
  if (f64) {
    OVL_REQUIRE(!(flags & (OVL_LINKS_F32 | OVL_LINKS_F16R12)), "ovl_apply_DW: FP64 uses FP64 links");
    OVL_REQUIRE(lat->src()->u64, "ovl_apply_DW: links not set");
  } else {
    lf = (flags & OVL_LINKS_F16R12) ? LINK_F16R12 : LINK_F32;
    OVL_REQUIRE(lf == LINK_F32 ? lat->src()->u32 != nullptr : lat->src()->u16 != nullptr,
                "ovl_apply_DW: links not set in the requested format");
  }
  const bool dag = flags & OVL_DAGGER, g5 = flags & OVL_GAMMA5, nat = flags & OVL_NATIVE;
  // D^H = g5 D(-mu) g5; output gamma5 count = dag xor g5
  OVL_CHECK_CUDA(launch_dslash(lat->g, lat->src()->links(), lf, f64, m_W, dag ? -mu : mu, dag, dag != g5, nat, nat, nrhs, in,
                               out, (cudaStream_t)stream));
  return OVL_OK;
}

void ovl_sign_params_default(ovl_sign_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->method = OVL_DIRECT_2SL;
  p->precision = OVL_PREC_F64;
  p->m_W = -2.0;
  p->mu = 0.0;
  p->tol = 1e-10;
  p->k_max = 600;
  p->check_every = 20;
  p->rational_kind = OVL_RAT_NEUBERGER;
  p->use_graphs = 1;
  p->restart_k = 40;
}

ovl_status ovl_apply_sign(ovl_lattice* lat, const ovl_sign_params* p, int32_t nrhs, const void* b, void* x,
                          ovl_sign_info* info, void* stream) {
  clear_error();
  OVL_REQUIRE(lat && p && b && x, "ovl_apply_sign: NULL argument");
  OVL_REQUIRE(nrhs >= 1 && nrhs <= 64, "ovl_apply_sign: nrhs must be in [1, 64]");
  OVL_REQUIRE(p->precision >= OVL_PREC_F64 && p->precision <= OVL_PREC_F32_F16LINKS, "ovl_apply_sign: precision");
  OVL_REQUIRE(p->tol >= 0, "ovl_apply_sign: tol must be >= 0");
  OVL_REQUIRE(2.0 * p->m_W + 8.0 != 0.0, "ovl_apply_sign: m_W = -4 has no kappa");
  std::shared_lock<std::shared_mutex> shared(lat->src()->guard);  // links / deflation set stay as they are
  OVL_DEVICE_SCOPE(lat->ctx->device);
  if (p->method == OVL_DIRECT_2SL)
    return solve_direct(lat, p, nrhs, (const double2*)b, (double2*)x, info, (cudaStream_t)stream);
  if (p->method == OVL_MULTISHIFT_BICG)
    return solve_multishift(lat, p, nrhs, (const double2*)b, (double2*)x, info, (cudaStream_t)stream);
  if (p->method == OVL_FOM_RESTARTED)
    return solve_fom(lat, p, nrhs, (const double2*)b, (double2*)x, info, (cudaStream_t)stream);
  set_error("ovl_apply_sign: unknown method %d", p->method);
  return OVL_EINVAL;
}

ovl_status ovl_get_tridiag(ovl_lattice* lat, int32_t rhs, int32_t k_cap, int32_t* k_out, void* alpha, void* beta,
                           void* delta) {
  clear_error();
  OVL_REQUIRE(lat && k_out, "ovl_get_tridiag: NULL argument");
  if (rhs < 0 || rhs >= (int)lat->last_alpha.size()) {
    set_error("ovl_get_tridiag: no direct solve with rhs %d on this lattice", rhs);
    return OVL_ENOTFOUND;
  }
  int k = (int)lat->last_alpha[rhs].size() / 2;
  *k_out = k;
  OVL_REQUIRE(k <= k_cap, "ovl_get_tridiag: capacity %d < k = %d", k_cap, k);
  if (alpha) std::memcpy(alpha, lat->last_alpha[rhs].data(), (size_t)k * 16);
  if (beta && k > 1) std::memcpy(beta, lat->last_beta[rhs].data(), (size_t)(k - 1) * 16);
  if (delta && k > 1) std::memcpy(delta, lat->last_delta[rhs].data(), (size_t)(k - 1) * 16);
  return OVL_OK;
}

}  // extern "C"
