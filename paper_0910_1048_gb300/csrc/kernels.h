// Launchers of the library's CUDA kernels (implemented in kernels.cu).
#pragma once

#include <algorithm>

#include "common.h"

namespace ovl {

constexpr int kBlock = 128;     // threads per block of the site-parallel kernels
constexpr int kPairSites = 64;  // sites per block of the pair stencil (x2 threads)
constexpr int kLinkGroup = 4;     // sources that share one load of a site's links in the batched FP32 kernels
constexpr int kSplitVolume = 32768;  // below this many sites the pair stencils split each site over 8 threads
inline bool use_split(const Geom& g) { return g.vol < kSplitVolume; }
// Plain launch through cudaLaunchKernelEx (one call site per kernel shape, error returned).
// Programmatic dependent launch was measured here and dropped: blocks of a waiting successor
// hold SM slots that the concurrent solves of a step would otherwise use (8^4 FP64 pair stencil
// 50 -> 75 us inside the step).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plain(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Records a timing event around a launch: as an external event node while `st` is being captured
// into a graph (a plain record inside a capture only orders the graph's nodes and times nothing),
// as a plain record otherwise (the runtime refuses the external flag outside a capture).
inline cudaError_t record_timing(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, st);
}

// Pair-stencil variant chosen by the autotuner for (volume, precision): -1 none yet,
// 0 one thread per site (64 sites per block), 1 split over 8 threads, 2 / 3 one thread per site
// with 48 / 32 sites per block, 4 split held to 128 registers (two blocks per SM), 5 split with
// 16 sites per block held to 168 registers (three blocks per SM), 6 one thread per site, 32 sites,
// one stencil (H(mu) or H(-mu)) per one-warp block, 7 dynamically scheduled (warps of a resident
// grid claim 32-site tasks from a counter), 8 FP32 batches: each site's links loaded once for a
// group of 4 sources (one thread per site and stencil, 32 sites per block; as 3 otherwise). The
// FP64 stencil is bound by the FP64 pipe, so its time follows the most loaded SM: at 12^4 ncu
// counted SM active cycles of max 206K against a mean of 156K for variant 3 and 214K against 164K
// for variant 6. The multishift kernels run variants 0, 2, 3, 6, 7, 8 as 0 and 4, 5 as 1.
// Thread-safe, process-wide. (A 16-thread split, one hop per thread, measured 54 us against 32 us
// for FP64 at 8^4: more index and reduction work than the extra warps hide.)
constexpr int kPairVariants = 9;
int tuned_pair_variant(int vol, int prec);
// Returns the variant for the key, running `measure` (which returns the fastest variant, or -1)
// under the table's lock the first time, so that every solve in the process uses one decision per key.
int tune_pair_variant(int vol, int prec, int (*measure)(void*), void* arg);
// Sets the entry (variant >= 0) or removes it (-1).
void set_pair_variant(int vol, int prec, int variant);
constexpr int kVecBlock = 128;  // threads per block of the element-parallel vector kernels
constexpr int kBalBlock = 512;  // threads per block of the one-block-per-SM FP64 update
inline unsigned vec_blocks(const Geom& g) { return (unsigned)((12 * (size_t)g.vol + kVecBlock - 1) / kVecBlock); }
// Elements per thread of the element-parallel kernels: enough to amortise the per-thread set-up and
// the block reduction, while keeping at least about four (FP32) or two (FP64) blocks per SM over the
// whole grid. FP64 threads take more elements: every FP64 instruction of the reduction tree costs
// 64 FP32 ones on this GPU.
inline int vec_elts(const Geom& g, int nrhs, bool f64) {
  const size_t total = 12 * (size_t)g.vol * (size_t)nrhs;
  return (int)std::max<size_t>(1, std::min<size_t>(8, total / ((size_t)kVecBlock * (f64 ? 304 : 608))));
}
inline unsigned vec_blocks(const Geom& g, int elt) {
  return (unsigned)((12 * (size_t)g.vol + (size_t)kVecBlock * elt - 1) / ((size_t)kVecBlock * elt));
}
// partial-sum slots per rhs: the most blocks any reduction kernel launches (the element-parallel
// ones), plus kMaxFillSMs at the top for the one-block-per-SM FP64 update, whose block partials
// must not overwrite the pair stencil's chunk partials that its blocks are still reading
constexpr int kMaxFillSMs = 256;  // the one-block-per-SM kernels run on GPUs with at most this many SMs
inline int partial_slots(const Geom& g) { return (int)vec_blocks(g) + kMaxFillSMs; }

// Device state of the two-sided Lanczos recurrences for nrhs right-hand sides.
// Index conventions: column j = 1..kmax+1 of the basis, stored at slot (j - 1) % vcols; scalars
// indexed by j.
struct LzDev {
  int kmax = 0;
  int nrhs = 0;
  int nblk = 0;             // partial slots per rhs (>= blocks of any reduction kernel)
  int* j = nullptr;         // [nrhs] current step (1-based)
  int* status = nullptr;    // [nrhs] 0 running, 1 breakdown
  double* sv = nullptr;     // [nrhs][kmax+2] v_j = sv_j * vhat_j
  double2* sw = nullptr;    // [nrhs][kmax+2] w_j = sw_j * what_j
  double2* alpha = nullptr; // [nrhs][kmax+2]
  double2* beta = nullptr;  // [nrhs][kmax+2] super-diagonal beta_j = h_{j,j+1}
  double* delta = nullptr;  // [nrhs][kmax+2] sub-diagonal delta_j = h_{j+1,j}
  double* vnorm = nullptr;  // [nrhs][kmax+2] ||v_j||
  double* beta0 = nullptr;  // [nrhs] ||r||
  double* part = nullptr;   // [nrhs][nblk][4] block partials
  unsigned* count = nullptr;// [nrhs] last-block counters (kept at 0 between launches)
  unsigned* claim = nullptr;// [nrhs] task counters of the dynamically scheduled pair stencil (kept at 0)
  int* pending = nullptr;   // [nrhs] 1: the last update's sums await their finish (deferred mode)
  int vcols = 0;            // basis columns kept per rhs: kmax + 1, or 3 (two-pass: a rotating window)
  double2* xacc = nullptr;  // two-pass, second pass: [nrhs][12][V] FP64 sum of coef_j vhat_j so far
  const double2* xcoef = nullptr;  // two-pass: [nrhs][kmax + 2] coefficient of column j (0 beyond k)
  double2* ucoef = nullptr; // [nrhs][4] coefficients of the next update, written with alpha_j:
                            // sv_j alpha_j, sv_{j-1} beta_{j-1}, sw_j conj(alpha_j), delta_{j-1} sw_{j-1}
};

// Layout conversion canonical [nrhs][V][12] <-> native [nrhs][12][V]; element types by flag.
cudaError_t launch_to_native(const Geom& g, int nrhs, bool in_f64, const void* in, bool out_f64, void* out, cudaStream_t st);
cudaError_t launch_from_native(const Geom& g, int nrhs, bool in_f64, const void* in, bool out_f64, void* out, cudaStream_t st);

// Links: canonical complex128 [4][V][3][3] (device) -> [4][9][V] f64 / f32, [4][6][V] f16 rows 0-1.
cudaError_t launch_ingest_links(const Geom& g, const double* ucan, double2* u64, float2* u32, uint32_t* u16, cudaStream_t st);

// out = [g5^go] D_W(sign*mu) [g5^gi] in; dtype f64 (FP64 links) or f32 (lf = F32 / F16R12).
cudaError_t launch_dslash(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu,
                          bool g5_in, bool g5_out, bool native_in, bool native_out, int nrhs,
                          const void* in, void* out, cudaStream_t st);

// ---- direct two-sided Lanczos (Algorithm 4), per-step kernels
// vh: [nrhs][kmax+1][12][V], wh: [2][nrhs][12][V], av/aw: [nrhs][12][V]; element type by f64.
struct LzVecs {
  void* vh = nullptr;
  void* wh = nullptr;
  void* av = nullptr;
  void* aw = nullptr;
  double2* xp = nullptr;    // [nrhs][12][V] FP64 deflated part x_P (nullptr without deflation)
};

// c_i = l_i^H b, d_i = r_i^H b (dots[rhs][0..m) = c, [m..2m) = d); part >= nrhs*m*ceil(V/128)*4.
cudaError_t launch_defl_dots(const Geom& g, int nrhs, int m, const double2* b, const double2* R, const double2* L,
                             double* part, unsigned* count, double2* dots, cudaStream_t st);

// Start: from b (canonical complex128, device) build vhat_1 = r, what_1 = r~ and the scales.
// With m > 0 deflation vectors R, L (native FP64 [m][12][V]) and lam (host, 2m doubles):
// x_P = R sign(Lambda) L^H b, r = b - R L^H b, r~ = b - L R^H b (Algorithm 4, first lines).
cudaError_t launch_lanczos_start(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, const double2* b,
                                 int m, const double2* R, const double2* L, const double* lam_sign,
                                 double2* dots, cudaStream_t st);
// A step = pair stencil (+ alpha), then the biorthogonal update. `variant` is the pair shape of the
// solve (resolve_pair_variant once per solve, then the same value for every launch of it): with
// shape 7 in FP64 the step runs deferred (the update's sums are finished by a settle kernel that
// the next pair launch runs first, with the stencil launched early behind it; after a chunk's last
// step launch_lanczos_settle finishes them before the host reads the scalars).
int resolve_pair_variant(const Geom& g, int lf, bool f64);
// Kernels one Lanczos step launches.
int lanczos_step_launches(const Geom& g, int lf, bool f64, int variant);
// `mid`, when given, is recorded (record_timing) after the stencil or update kernel itself, before the
// one-block finishing kernel of the shapes that have one (or right after the single kernel).
// `first`, when given, is recorded right before the stencil kernel (after the settle kernel that
// precedes it in a deferred step).
cudaError_t launch_lanczos_pair(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu,
                                const LzDev& lz, const LzVecs& vec, cudaStream_t st, int variant,
                                cudaEvent_t mid = nullptr, cudaEvent_t first = nullptr);
cudaError_t launch_lanczos_update(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, cudaStream_t st,
                                  int variant, cudaEvent_t mid = nullptr);
// Finishes a deferred step (no-op otherwise): after the last step of a chunk, before the host or a
// later kernel reads alpha, beta, delta, the scales, |v|, j or the status.
cudaError_t launch_lanczos_settle(const Geom& g, bool f64, const LzDev& lz, cudaStream_t st, int variant);
int lanczos_settle_launches(bool f64, int variant);  // 1 where launch_lanczos_settle launches a kernel
// One step j (read from lz.j): pair stencil + alpha, then the biorthogonal update.
cudaError_t launch_lanczos_step(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu,
                                const LzDev& lz, const LzVecs& vec, cudaStream_t st, int variant);
// Element sampling of the stopping estimate: the norms ||V c|| of the change and of the iterate
// enter only as a ratio, so on large lattices they are taken over runs of 32 consecutive
// elements, one run in every 32 * stride (about 10^5 elements sampled; a fixed pattern, so the
// estimate is deterministic); the full basis read per evaluation would otherwise cost more than
// the steps between evaluations (16^4, 16 sources: 79 GB).
inline int vnorm_stride(const Geom& g) {
  const size_t n = 12 * (size_t)g.vol;
  int st = 1;
  while (st < 64 && n / (2 * st) >= 98304) st *= 2;
  return st;
}
// out[rhs][0..1] = ||sum_{j<k_r} d1_j vhat_j||^2, ||sum_{j<k_r} d2_j vhat_j||^2 over the sampled
// elements (own scratch part, count: part >= nrhs * 2 * ceil(12V/256) doubles, count >= nrhs zeros).
cudaError_t launch_lanczos_vnorms(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, const int* kr,
                                  const double2* d1, const double2* d2, int kcoef, double* part, unsigned* count,
                                  double* out, cudaStream_t st);
// x = x_P + sum_{j<=k_r} coef_j vhat_j, written canonical complex128; coef [nrhs][kcoef],
// kr [nrhs] (device) the Krylov dimension of each rhs.
cudaError_t launch_lanczos_combine(const Geom& g, bool f64, const LzDev& lz, const LzVecs& vec, const int* kr,
                                   const double2* coef, int kcoef, double2* x, cudaStream_t st);

}  // namespace ovl

namespace ovl {

// ---- multishift BiCG on M = A^2 (Algorithm 3 with Section 5's g(t) = t sum w_i/(t^2 - s_i))
// Seed system (M - sigma_1) x = r, sigma_1 the shift closest to 0; shifted systems
// (M - sigma_i) x = r share its Krylov space with residuals zeta^i_k r_k (collinear).
// Status: 0 running, 1 breakdown, 2 converged, 3 empty (r = 0), 4 final update pending.
constexpr int kMaxShifts = 128;
constexpr double kFp32Floor = 2e-6;   // relative residual the FP32 iteration reaches by itself
constexpr int kMaxRefineSweeps = 8;   // FP64 residual / FP32 correction rounds per shifted system
constexpr int kRefineGroup = 1024;    // correction systems solved together in one batch
constexpr size_t kRefineBytes = (size_t)48 << 30;  // buffer budget of that batch (at most a quarter
                                                    // of the free device memory)
struct MsDev {
  int nrhs = 0, s = 0, nblk = 0;
  int* k = nullptr;           // [nrhs] iterations done
  int* status = nullptr;      // [nrhs]
  double2* seed = nullptr;    // [nrhs][8]: rho, alpha_k, alpha_{k-1}, beta_{k-1}, (|r0|,|r|), beta_k
  double2* zeta = nullptr;    // [nrhs][s][3]: zeta_{k-1}, zeta_k, zeta_{k+1}
  double2* ash = nullptr;     // [nrhs][s] alpha^i_k
  double2* bsh = nullptr;     // [nrhs][s] beta^i_k
  int* active = nullptr;      // [nrhs][s] 1 running, 2 last update pending, 0 done
  const double* omega = nullptr;  // [s]
  const double* dsig = nullptr;   // [s] sigma_i - sigma_1
  double sigma1 = 0, tol = 0;
  const double* sig1v = nullptr;  // [nrhs] per-rhs seed shift (overrides sigma1; batched refinement)
  const double* tolv = nullptr;   // [nrhs] per-rhs tolerance (overrides tol)
  double* part = nullptr;     // [nrhs][nblk][4]
  unsigned* count = nullptr;  // [nrhs]
};

struct MsVecs {
  void *r = nullptr, *rt = nullptr, *p = nullptr, *pt = nullptr;  // [nrhs][12][V]
  void *t = nullptr, *tt = nullptr, *q = nullptr, *qt = nullptr;  // [nrhs][12][V]
  void* ps = nullptr;          // [nrhs][s][12][V] shifted directions
  double2* X = nullptr;        // [nrhs][12][V] FP64 sum_i omega_i x^(i)
  double2* xp = nullptr;       // [nrhs][12][V] FP64 x_P (nullptr without deflation)
  double2* xs = nullptr;       // [nrhs][s][12][V] per-shift solutions (refinement only; else X): float-float
                               // in the FP32 pass, FP64 after launch_ff_to_f64
  double2* r64 = nullptr;      // [nrhs][12][V] FP64 deflated residual r (refinement only)
};

cudaError_t launch_ms_start(const Geom& g, bool f64, const MsDev& ms, const MsVecs& v, const double2* b, int m,
                            const double2* R, const double2* L, const double* lam_sign, double2* dots, cudaStream_t st);
// One iteration (four launches). With timing events (may be null): ev[0] before the first
// pair stencil, ev[1] after it, ev[2] before the direction update, ev[3] after it.
// Whether the multishift iteration uses the eight-threads-per-site stencils (from the pair shape of
// (volume, key), key = link format, 0 for FP64); the solvers key their cached graphs on it.
bool ms_pair_split(const Geom& g, int key);
cudaError_t launch_ms_step(const Geom& g, const Links& U, int lf, bool f64, double m_w, double mu, const MsDev& ms,
                           const MsVecs& v, cudaStream_t st, cudaEvent_t* ev = nullptr);
// Reliable-update helpers. Residuals of the systems j0 .. j0+gn-1 of the flattened (rhs, shift)
// index j = rhs*s + i:
// res_j = r64[rhs] - (t2_j - sigma[i] x_j), |res_j|^2 -> out[j - j0]. t2, x, res hold gn vectors.
cudaError_t launch_ms_residual_batch(const Geom& g, int j0, int gn, int s, const double2* r64, const double2* t2,
                                     const double2* x, const double* sigma, double2* res, double* part,
                                     unsigned* count, double* out, cudaStream_t st);
// x_j += e_j for the gn vectors whose status[j] is not a breakdown (1).
cudaError_t launch_axpy_f64_masked(const Geom& g, int gn, const int* status, const double2* e, double2* x,
                                   cudaStream_t st);
// n complex values held as float-float (re hi, re lo, im hi, im lo) -> complex double, in place.
cudaError_t launch_ff_to_f64(size_t n, double2* x, cudaStream_t st);
// X = sum_i omega_i xs_i per rhs.
cudaError_t launch_ms_combine_shifts(const Geom& g, int nrhs, int s, const double* omega, const double2* xs,
                                     double2* X, cudaStream_t st);
// x (canonical complex128) = x_P + AX (AX native FP64, = H_W(mu) X)
cudaError_t launch_ms_finish(const Geom& g, int nrhs, const double2* ax, const double2* xp, double2* x, cudaStream_t st);

}  // namespace ovl
