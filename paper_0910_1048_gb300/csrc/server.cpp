// Request server: sign(H_W(mu)) b solves of mixed lattices, mu and tolerances as they arrive.
//
// Requests queue as they arrive. `max_slots` worker threads each take, among the queued
// requests whose device footprint (Krylov basis and work vectors of a direct two-sided Lanczos
// solve, Algorithm 4) fits in what the memory budget has left, the one with the least
// estimated work (sites x right-hand sides x k_max, FP32 at half weight) - unless the oldest
// request has waited longer than kMaxWait, which is then served first (no starvation of large
// requests; while it does not fit, smaller ones are not admitted past it). Requests that
// arrive while others run are admitted as soon as a slot and memory free up, and their work
// overlaps on the device (every slot solves on its own streams through a view of the field
// that shares the field's links but not its workspace). Workspaces are allocated and released
// stream-ordered, so admitting or retiring one request never stalls another. Each request's
// arithmetic is independent of what else runs: results are the same alone and in the mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "admission.h"
#include "common.h"

namespace ovl {
ovl_lattice* lattice_view(ovl_lattice* parent);
size_t direct_footprint(int vol, int nrhs, int kmax, bool f64, bool two_pass);
size_t multishift_footprint(int vol, int nrhs, int s, bool f64, bool refine);
void neuberger_for_spectrum(double lo, double hi, double eps, int* s_out, double* c_out, double* d_out);
constexpr double kFp32FloorHost = 2e-6;  // below it the reduced-precision multishift refines (FP64)
}  // namespace ovl

struct ovl_server {
  struct Request {
    uint64_t ticket = 0;
    ovl_request req{};
    std::vector<double> b, x;  // interleaved complex128
    std::vector<ovl_sign_info> info;
    size_t footprint = 0;
    double work = 0;  // estimated: sites x nrhs x k_max (FP32 at half weight)
    std::chrono::steady_clock::time_point arrived;
    ovl_status status = OVL_PENDING;
    bool done = false;
  };
  ovl_ctx* ctx = nullptr;
  ovl_server_cfg cfg{};
  std::vector<ovl_lattice*> fields;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  size_t in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  // (slot, field) -> the slot's view of the field (own workspaces, the field's links and
  // deflation set); created and looked up under `mu`, used outside it (the pointer is stable)
  std::map<std::pair<int, int>, ovl_lattice*> views;
};

namespace {

// Poles a multishift request will use: given, or Eq. no_of_poles for Neuberger (as the solver
// chooses them).
int request_poles(const ovl_request& r) {
  if (r.s > 0) return r.s;
  int s = 0;
  double c = 0, d = 0;
  ovl::neuberger_for_spectrum(r.spec_lo, r.spec_hi, std::max(r.tol, 1e-15), &s, &c, &d);
  return s;
}

size_t footprint(const ovl_server* s, const ovl_request& r) {
  const ovl_lattice* lat = s->fields[r.field_id];
  const bool f64 = r.precision == OVL_PREC_F64;
  if (r.method == OVL_MULTISHIFT_BICG)
    return ovl::multishift_footprint(lat->g.vol, r.nrhs, request_poles(r), f64,
                                     !f64 && r.tol < ovl::kFp32FloorHost);
  return ovl::direct_footprint(lat->g.vol, r.nrhs, r.k_max, f64, r.two_pass != 0);
}

constexpr double kMaxWait = 2.0;  // seconds after which the oldest request goes first

// Queue position of the next request to admit, or -1 (caller holds the lock); the policy is
// admission_pick (admission.h).
long pick(ovl_server* s) {
  if (s->queue.empty()) return -1;
  std::vector<ovl::PendingRequest> q(s->queue.size());
  for (size_t i = 0; i < q.size(); ++i) {
    const ovl_server::Request* r = s->reqs[s->queue[i]].get();
    q[i] = {r->footprint, r->work};
  }
  const ovl_server::Request* oldest = s->reqs[s->queue.front()].get();
  const double waited =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - oldest->arrived).count();
  return ovl::admission_pick(q.data(), q.size(), s->in_use, (size_t)s->cfg.mem_budget_bytes, waited, kMaxWait);
}

void worker(ovl_server* s, int slot) {
  cudaSetDevice(s->ctx->device);
  for (;;) {
    ovl_server::Request* job = nullptr;
    ovl_lattice* view = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      long at = -1;
      // re-checked at least every 100 ms so that a request passing kMaxWait is seen
      while (!s->stop && (at = pick(s)) < 0) s->cv.wait_for(lk, std::chrono::milliseconds(100));
      if (s->stop) return;
      job = s->reqs[s->queue[at]].get();
      s->queue.erase(s->queue.begin() + at);
      s->in_use += job->footprint;
      ovl_lattice*& v = s->views[{slot, job->req.field_id}];
      if (!v) v = ovl::lattice_view(s->fields[job->req.field_id]);
      view = v;
    }
    const ovl_request& r = job->req;
    ovl_sign_params p;
    ovl_sign_params_default(&p);
    p.method = r.method;
    p.precision = r.precision;
    p.m_W = r.m_W;
    p.mu = r.mu;
    p.tol = r.tol;
    p.k_max = r.k_max;
    p.use_deflation = r.use_deflation;
    p.rational_kind = r.rational_kind;
    p.s = r.s;
    p.spec_lo = r.spec_lo;
    p.spec_hi = r.spec_hi;
    p.two_pass = r.two_pass;
    p.host_io = 1;
    std::vector<ovl_sign_info> info(r.nrhs);
    std::vector<double> x(job->b.size());
    ovl_status st = ovl_apply_sign(view, &p, r.nrhs, job->b.data(), x.data(), info.data(), nullptr);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      job->x.swap(x);
      job->info = info;
      job->status = st;
      job->done = true;
      s->in_use -= job->footprint;
      job->b.clear();
      job->b.shrink_to_fit();
    }
    s->cv.notify_all();
  }
}

}  // namespace

extern "C" {

ovl_status ovl_server_create(ovl_ctx* ctx, const ovl_server_cfg* cfg, ovl_server** out) {
  ovl::clear_error();
  OVL_REQUIRE(ctx && cfg && out, "ovl_server_create: NULL argument");
  OVL_REQUIRE(cfg->mem_budget_bytes > 0 && cfg->max_slots >= 1 && cfg->max_slots <= 64,
              "ovl_server_create: need mem_budget_bytes > 0 and 1 <= max_slots <= 64");
  ovl_server* s = new ovl_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  for (int i = 0; i < cfg->max_slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return OVL_OK;
}

ovl_status ovl_server_add_field(ovl_server* s, ovl_lattice* lat, int32_t* field_id) {
  ovl::clear_error();
  OVL_REQUIRE(s && lat && field_id, "ovl_server_add_field: NULL argument");
  OVL_REQUIRE(lat->u64, "ovl_server_add_field: the lattice has no links");
  OVL_REQUIRE(lat->parent == nullptr, "ovl_server_add_field: not a field lattice");
  std::lock_guard<std::mutex> lk(s->mu);
  s->fields.push_back(lat);
  lat->servers.fetch_add(1);  // ovl_destroy_lattice refuses it until the server is destroyed
  *field_id = (int32_t)s->fields.size() - 1;
  return OVL_OK;
}

ovl_status ovl_submit(ovl_server* s, const ovl_request* r, uint64_t* ticket) {
  ovl::clear_error();
  OVL_REQUIRE(s && r && ticket && r->b, "ovl_submit: NULL argument");
  OVL_REQUIRE(r->nrhs >= 1 && r->nrhs <= 64 && r->k_max >= 1 && r->tol >= 0, "ovl_submit: invalid request");
  OVL_REQUIRE(r->precision >= OVL_PREC_F64 && r->precision <= OVL_PREC_F32_F16LINKS, "ovl_submit: precision");
  OVL_REQUIRE(r->method == OVL_DIRECT_2SL || r->method == OVL_MULTISHIFT_BICG, "ovl_submit: method");
  OVL_REQUIRE(r->two_pass == 0 || (r->two_pass == 1 && r->method == OVL_DIRECT_2SL),
              "ovl_submit: two_pass is 0, or 1 with the direct method");
  OVL_REQUIRE(r->method == OVL_DIRECT_2SL ||
                  (r->spec_lo > 0 && r->spec_hi > r->spec_lo &&
                   (r->rational_kind == OVL_RAT_NEUBERGER || r->rational_kind == OVL_RAT_ZOLOTAREV) &&
                   (r->rational_kind == OVL_RAT_NEUBERGER || r->s > 0) && r->s >= 0 && r->s <= 127),
              "ovl_submit: a multishift request needs 0 < spec_lo < spec_hi and a Neuberger or Zolotarev kind "
              "(Zolotarev with s > 0)");
  std::unique_lock<std::mutex> lk(s->mu);
  OVL_REQUIRE(r->field_id >= 0 && r->field_id < (int)s->fields.size(), "ovl_submit: unknown field %d", r->field_id);
  const ovl_lattice* lat = s->fields[r->field_id];
  const bool has_fmt = r->precision == OVL_PREC_F64 ||
                       (r->precision == OVL_PREC_F32 ? lat->u32 != nullptr : lat->u16 != nullptr);
  OVL_REQUIRE(has_fmt,
              "ovl_submit: field lacks the link format of this precision");
  OVL_REQUIRE(!r->use_deflation || (lat->defl.m > 0 && lat->defl.m_w == r->m_W && lat->defl.mu == r->mu),
              "ovl_submit: use_deflation needs the field's deflation set for (m_W, mu) = (%g, %g)", r->m_W, r->mu);
  auto job = std::make_unique<ovl_server::Request>();
  job->req = *r;
  job->footprint = footprint(s, *r);
  if (job->footprint > (size_t)s->cfg.mem_budget_bytes) {
    ovl::set_error("ovl_submit: request needs %zu bytes, budget is %lld", job->footprint,
                   (long long)s->cfg.mem_budget_bytes);
    return OVL_EINVAL;
  }
  const size_t nd = (size_t)2 * 12 * lat->g.vol * r->nrhs;
  job->b.assign((const double*)r->b, (const double*)r->b + nd);
  job->req.b = nullptr;
  job->work = (double)lat->g.vol * r->nrhs * r->k_max * (r->precision == OVL_PREC_F64 ? 1.0 : 0.5) *
              (r->two_pass ? 2.0 : 1.0);
  job->arrived = std::chrono::steady_clock::now();
  job->ticket = s->next_ticket++;
  *ticket = job->ticket;
  s->queue.push_back(job->ticket);
  s->reqs[job->ticket] = std::move(job);
  lk.unlock();
  s->cv.notify_all();
  return OVL_OK;
}

ovl_status ovl_poll(ovl_server* s, uint64_t ticket, ovl_sign_info* info, void* x_out) {
  ovl::clear_error();
  OVL_REQUIRE(s, "ovl_poll: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    ovl::set_error("ovl_poll: unknown ticket %llu", (unsigned long long)ticket);
    return OVL_ENOTFOUND;
  }
  ovl_server::Request* j = it->second.get();
  if (!j->done) return OVL_PENDING;
  if (info) std::memcpy(info, j->info.data(), j->info.size() * sizeof(ovl_sign_info));
  if (x_out && !j->x.empty()) std::memcpy(x_out, j->x.data(), j->x.size() * sizeof(double));
  ovl_status st = j->status;
  s->reqs.erase(it);  // results are handed out once
  return st;
}

ovl_status ovl_server_destroy(ovl_server* s) {
  ovl::clear_error();
  if (!s) return OVL_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->views)
    if (kv.second) ovl_destroy_lattice(kv.second);
  for (ovl_lattice* f : s->fields) f->servers.fetch_sub(1);
  delete s;
  return OVL_OK;
}

}  // extern "C"
