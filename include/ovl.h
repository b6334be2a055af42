/*
 * ovl.h — C ABI of the GB300 library for x = sign(H_W(mu)) b.
 *
 * The operation (Bloch et al., arXiv:0910.1048): the overlap operator needs the sign
 * function of its kernel H_W = gamma5 D_W(mu) (Section 1), a non-Hermitian matrix at
 * quark chemical potential mu. sign(A) = R sign(Lambda) R^-1 with sign(z) = sign(Re z)
 * (Section 1, Eq. 1). The library evaluates sign(H_W) b by
 *   - direct two-sided Lanczos with LR deflation, Algorithm 4:
 *       x = x_P + beta V_k sign(H_k) e_1 (Eq. bloch_approx_unsym), or
 *   - multishift BiCG on a rational approximation, Algorithm 3 with Section 5's
 *       g(t) = t sum_i omega_i / (t^2 - sigma_i) (Neuberger Eq. pfe_s, or Zolotarev).
 *
 * Conventions (the paper defers D_W to its reference [Bloch:2006cd]; reading used):
 *   (D_W psi)(x) = psi(x) - kappa sum_nu [ e^{+mu d_nu,t} (1 - g_nu) U_nu(x) psi(x+nu)
 *                                        + e^{-mu d_nu,t} (1 + g_nu) U_nu(x-nu)^H psi(x-nu) ],
 *   kappa = 1/(2 m_W + 8); chiral gamma basis, gamma5 = diag(1,1,-1,-1); spatial
 *   directions periodic; time periodic or antiperiodic (t_bc).
 *
 * Canonical layouts (what callers pass; complex128 = two doubles re, im):
 *   links   U[4][Lt][Lz][Ly][Lx][3][3]   direction 0..3 = x,y,z,t; row index first
 *   spinor  psi[Lt][Lz][Ly][Lx][4][3]   spin, then colour fastest; n = 12 V complex
 *   site    ((t*Lz + z)*Ly + y)*Lx + x
 *   batches [nrhs][n]
 *
 * Errors: every call returns ovl_status; no call aborts, exits or throws across the ABI.
 * On failure ovl_last_error() returns a message for the calling thread.
 * Threading: one ovl_lattice must not be used by two threads at once; distinct lattices
 * may. Stream-ordered calls take a cudaStream_t as void* (NULL = legacy default stream).
 * Devices: a call makes the lattice's (or context's) device current while it runs and gives
 * the caller back its own current device before it returns.
 */
#ifndef OVL_H
#define OVL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ovl_status;
enum {
  OVL_OK = 0,
  OVL_PENDING = 1,      /* ovl_poll: request not finished */
  OVL_EINVAL = -1,      /* bad argument: shapes, odd extents, NULL, non-biorthonormal L,R */
  OVL_ENOMEM = -2,      /* device or host allocation failed */
  OVL_ECUDA = -3,       /* a CUDA call failed; message has the CUDA error string */
  OVL_EBREAKDOWN = -4,  /* two-sided Lanczos/BiCG: |w^H v| < 1e-14 ||v|| ||w|| */
  OVL_ENOCONV = -5,     /* k_max reached before tol; best iterate returned */
  OVL_ETIMEOUT = -6,    /* a bounded device-side wait gave up */
  OVL_EBUSY = -7,       /* server admission refused (memory budget or slots) */
  OVL_EILLPOSED = -8,   /* sign undefined: eigenvalue on the imaginary axis detected */
  OVL_ENOTFOUND = -9    /* unknown ticket / field id */
};

/* Storage formats of the links kept on the device (bit set for ovl_set_links). */
#define OVL_F64 1u     /* 18 doubles per link */
#define OVL_F32 2u     /* 18 floats per link */
#define OVL_F16R12 4u  /* first two rows as 12 halves; row 3 = conj(row1 x row2) (SU(3)) */

/* Element types of spinor buffers. */
#define OVL_C128 0     /* complex double */
#define OVL_C64 1      /* complex float */

/* ovl_apply_DW flags. */
#define OVL_DAGGER 1u  /* apply D_W(mu)^H = gamma5 D_W(-mu) gamma5 */
#define OVL_GAMMA5 2u  /* apply gamma5 after: H_W = gamma5 D_W */
#define OVL_NATIVE 4u  /* in/out use the library's device layout (ovl_to_native) */
#define OVL_LINKS_F32 8u     /* use the FP32 link copy (only with OVL_C64) */
#define OVL_LINKS_F16R12 16u /* use the FP16 12-real link copy (only with OVL_C64) */

typedef struct ovl_ctx ovl_ctx;
typedef struct ovl_lattice ovl_lattice;
typedef struct ovl_server ovl_server;

/* ----------------------------------------------------------------- context, lattice */

/* Create a context on CUDA device `device`. The context owns a stream and scratch.
 * Errors: EINVAL (out NULL), ECUDA (no such device / driver failure). */
ovl_status ovl_ctx_create(int32_t device, ovl_ctx** out);
ovl_status ovl_ctx_destroy(ovl_ctx* ctx);

/* Thread-local message describing the last failed call on this thread ("" if none). */
const char* ovl_last_error(void);

/* Library version string, e.g. "ovl 1.0 sm_103a". */
const char* ovl_version(void);

/* Create a lattice Lx x Ly x Lz x Lt (dims[0..3]); every extent even and >= 2.
 * t_bc: -1 antiperiodic (default physics), +1 periodic. No links yet.
 * Errors: EINVAL (odd/too small extents, |t_bc| != 1, volume > 2^26 sites). */
ovl_status ovl_create_lattice(ovl_ctx* ctx, const int32_t dims[4], int32_t t_bc, ovl_lattice** out);
ovl_status ovl_destroy_lattice(ovl_lattice* lat);

/* Number of complex entries per spinor, n = 12 V. */
int64_t ovl_lattice_n(const ovl_lattice* lat);

/* Copy links U (canonical complex128 layout, host or device memory per U_on_device)
 * into library-owned device copies in each format of the `formats` bit set (OVL_F64 is
 * always kept). Every format the lattice already holds from an earlier call is rewritten
 * from U as well, so no copy keeps the previous field. The caller's buffer may be freed on
 * return (the call synchronises).
 * Errors: EINVAL, EBUSY (a solve is reading the links), ENOMEM, ECUDA. */
ovl_status ovl_set_links(ovl_lattice* lat, const void* U, int32_t U_on_device, uint32_t formats);

/* LR deflation set (Section 3): m critical eigenpairs of A = H_W(m_W, mu):
 * R = right eigenvectors, L = left eigenvectors, each [m][n] canonical complex128,
 * lambda[m] complex128 eigenvalues; A R = R Lambda, L^H A = Lambda L^H, L^H R = I.
 * Copied to the device; valid for solves with the same (m_W, mu). m = 0 clears.
 * Errors: EINVAL (m < 0, max |L^H R - I| > 1e-8, NULL), EBUSY (a solve is reading the set),
 * ENOMEM, ECUDA. */
ovl_status ovl_set_deflation(ovl_lattice* lat, double m_W, double mu, int32_t m,
                             const void* R, const void* L, const void* lambda, int32_t on_device);

/* Convert nrhs spinors between the canonical layout and the library's device layout
 * (component-major: [nrhs][12][V] complex, c = spin*3 + colour). dtype OVL_C128/OVL_C64
 * for both sides. Device pointers; stream-ordered. */
ovl_status ovl_to_native(ovl_lattice* lat, int32_t dtype, int32_t nrhs, const void* in, void* out, void* stream);
ovl_status ovl_from_native(ovl_lattice* lat, int32_t dtype, int32_t nrhs, const void* in, void* out, void* stream);

/* out = D_W(mu) in (flags: OVL_DAGGER, OVL_GAMMA5 for H_W = gamma5 D_W), for nrhs
 * spinors [nrhs][n] of dtype OVL_C128 (FP64 links) or OVL_C64 (FP32 arithmetic with
 * FP32 links, or FP16 12-real links with OVL_LINKS_F16R12). in/out are device buffers,
 * must not alias, canonical layout unless OVL_NATIVE. Stream-ordered (no sync).
 * Section 1 defines H_W = gamma5 D_W; the stencil form is the reading above.
 * Errors: EINVAL (no links in the requested format, nrhs < 1, NULL), ECUDA. */
ovl_status ovl_apply_DW(ovl_lattice* lat, double m_W, double mu, uint32_t flags, int32_t dtype,
                        int32_t nrhs, const void* in, void* out, void* stream);

/* ----------------------------------------------------------------- sign solves */

enum { OVL_DIRECT_2SL = 0, OVL_MULTISHIFT_BICG = 1, OVL_FOM_RESTARTED = 2 };
enum { OVL_PREC_F64 = 0, OVL_PREC_F32 = 1, OVL_PREC_F32_F16LINKS = 2 };
enum { OVL_RAT_NEUBERGER = 0, OVL_RAT_ZOLOTAREV = 1, OVL_RAT_CUSTOM = 2 };

typedef struct {
  int32_t method;         /* OVL_DIRECT_2SL (Algorithm 4) | OVL_MULTISHIFT_BICG (Algorithm 3) |
                             OVL_FOM_RESTARTED (Algorithm 1: restarted FOM-LR on A^2) */
  int32_t precision;      /* OVL_PREC_*: vector/stencil precision; scalars always FP64 */
  double m_W;             /* Wilson mass (kappa = 1/(2 m_W + 8)) */
  double mu;              /* chemical potential */
  double tol;             /* relative accuracy target */
  int32_t k_max;          /* maximum Krylov dimension / iterations (default 600) */
  int32_t check_every;    /* direct: minimum spacing of convergence checks (default 20) */
  int32_t use_deflation;  /* 1: use the set from ovl_set_deflation (must match m_W, mu) */
  int32_t rational_kind;  /* multishift: OVL_RAT_* */
  int32_t s;              /* multishift: number of poles; 0 = from Eq. no_of_poles (Neuberger) */
  double spec_lo;         /* multishift: lower spectrum bound alpha (> 0) of the undeflated part */
  double spec_hi;         /* multishift: upper bound beta of |lambda| */
  const double* omega;    /* OVL_RAT_CUSTOM: s weights (host) */
  const double* sigma;    /* OVL_RAT_CUSTOM: s shifts sigma_i < 0 (host) */
  int32_t host_io;        /* 1: b and x are host pointers (copies inside the call) */
  int32_t use_graphs;     /* direct: capture the iteration chunks in CUDA graphs (default 1) */
  int32_t fixed_k;        /* direct: > 0 runs exactly this many steps (no convergence test) */
  int32_t priority;       /* CUDA stream priority of the solve, 0 default, p > 0 p levels more
                             urgent (clamped to the device's range); lets concurrent solves favour
                             the longest one. No effect on results. */
  int32_t restart_k;      /* restarted FOM: Arnoldi steps per cycle k (default 40, at most 64) */
  int32_t two_pass;       /* direct: 1 = two-pass strategy (Section 2.3): the first pass keeps three
                             basis vectors and builds H_k, the second regenerates the same vectors
                             and accumulates x; memory O(n) instead of O(k n), twice the stencils.
                             The stop test then measures the change of y with the column norms. */
} ovl_sign_params;

typedef struct {
  int32_t status;         /* OVL_OK | ENOCONV | EBREAKDOWN | ... for this right-hand side */
  int32_t iterations;     /* Krylov dimension k reached / BiCG iterations */
  int32_t matvecs;        /* applications of H_W (or its adjoint) */
  int32_t poles;          /* multishift: s used */
  double est_error;       /* the solver's own error estimate (relative) */
  double t_total_ms;      /* wall time of the call (shared by all rhs of the call) */
  double t_small_ms;      /* host time in sign(H_k) e_1 */
  double residual;        /* multishift: max recursive shifted residual |zeta_i r| / |r_0| */
  double t_kernel_ms;     /* mean device time of the sampled launches of the dominant kernel (the
                             pair stencil), timed with events on the stream that launched it */
  double t_update_ms;     /* the same for the vector-update kernel of a step */
  int32_t kernel_samples; /* launches behind t_kernel_ms (and t_update_ms) */
  int32_t kernel_launches;/* all library kernel launches of the call (shared by its rhs) */
  int32_t evaluations;    /* direct method: evaluations of sign(H_j) e_1 for this rhs */
  int32_t ritz_evaluations;/* direct method: of those, the ones that computed Ritz values to choose
                              the rational scale and pole count (the others reused them) */
  double t_finish_ms;     /* direct method: the same for the one-block kernels that finish a step's
                             cross-block sums and scalars, where the step's shapes have them
                             (t_kernel_ms and t_update_ms exclude them) */
} ovl_sign_info;

/* Fill p with defaults: DIRECT_2SL, F64, m_W = -2, mu = 0, tol = 1e-10, k_max = 600,
 * check_every = 20, no deflation, Neuberger, s = 0, use_graphs = 1, restart_k = 40. */
void ovl_sign_params_default(ovl_sign_params* p);

/* x = sign(H_W(m_W, mu)) b for nrhs right-hand sides b[nrhs][n] (canonical complex128),
 * written to x[nrhs][n]. Device pointers unless p->host_io. info[nrhs] receives per-rhs
 * results (may be NULL). The call returns when x is written (it synchronises `stream`).
 * Returns OVL_OK if every rhs reached tol, else the first non-OK per-rhs status
 * (ENOCONV / EBREAKDOWN still write the best iterate).
 * Algorithm 4 (direct), Algorithm 3 (multishift BiCG) or Algorithm 1 (restarted FOM: k_max
 * bounds the Arnoldi steps over all cycles, tol the shifted residuals |rho_i| |r| / |r_0|, the
 * rational function as for the multishift method); LR split x = x_P + f(A)(I-P)b (Eq. action)
 * when use_deflation. Errors: EINVAL, ENOMEM, ECUDA. */
ovl_status ovl_apply_sign(ovl_lattice* lat, const ovl_sign_params* p, int32_t nrhs,
                          const void* b, void* x, ovl_sign_info* info, void* stream);

/* Kernel shape of the two-sided Lanczos pair stencil (H(mu) v and H(-mu) w of one step of
 * Algorithm 4, the dominant kernel of the direct method) for lattices of `volume` sites at
 * `precision` (OVL_PREC_*): 0 one thread per site, 64 sites per block; 1 eight threads per site,
 * 32 sites per block; 2 / 3 as 0 with 48 / 32 sites per block; 4 as 1 held to two blocks per SM;
 * 5 eight threads per site, 16 sites per block, three blocks per SM; 6 one thread per site, 32
 * sites per one-warp block computing one of the two stencils; 7 one thread per site, the warps of
 * a grid that fills the GPU claiming 32-site tasks (one of the two stencils each) from a counter;
 * 8 (FP32 batches) one thread per site and stencil for a group of four right-hand sides, each
 * site's links loaded once per group (otherwise as 3). The multishift method runs 1, 4, 5 as its eight-thread stencil and the others as its
 * one-thread stencil. variant = -1
 * clears the entry: the next direct solve for that key times every shape on its own vectors and
 * keeps the fastest. Process-wide. All shapes compute the same step; results differ in the
 * rounding of the partial sums of alpha_j only.
 * Errors: EINVAL (variant outside -1..8, volume < 1, unknown precision). */
ovl_status ovl_set_pair_variant(int64_t volume, int32_t precision, int32_t variant);

/* The shape in use for (volume, precision); -1 if no solve has tuned it yet. */
int32_t ovl_get_pair_variant(int64_t volume, int32_t precision);

/* Allocation-free variant of ovl_apply_sign's direct method, for callers that cannot
 * allocate device memory: processes whose device memory belongs to another allocator (a
 * framework's pool, a server that reserves its budget at start-up) and latency-critical
 * loops that must not call cudaMalloc/cudaFree. The paper has no counterpart: this is a
 * property of the library, not of the method. Same kernels and results as ovl_apply_sign
 * (method OVL_DIRECT_2SL); b and x are device buffers; runs on `stream` and synchronizes it.
 * All scratch lives in one static 64 MiB device array per GPU that loads the library, held
 * until the process exits; its address is looked up on the first call for each device (make
 * that first call before any stream capture) and again on each later call made outside a
 * capture. Calls share the array: calls that overlap on the GPU race. No CUDA graphs, streams,
 * events or pinned buffers are created. `stream` must belong to the lattice's device; the
 * caller's current device is left as it was.
 * Errors: EINVAL (host_io set, method not direct, stream of another device, or scratch needed
 * > 64 MiB, e.g. a basis of nrhs * (k_max+1) * 12 V complex values that does not fit), ECUDA;
 * solve statuses as ovl_apply_sign. */
ovl_status ovl_apply_sign_noalloc(ovl_lattice* lat, const ovl_sign_params* p, int32_t nrhs,
                                  const void* b, void* x, ovl_sign_info* info, void* stream);

/* Tridiagonal H_k of the last direct solve on this lattice, rhs index `rhs`:
 * alpha[k], beta[k-1] (super-diagonal), delta[k-1] (sub-diagonal), complex128 host
 * arrays; *k_out = k. Pass k_cap = capacity of alpha. Errors: EINVAL, ENOTFOUND. */
ovl_status ovl_get_tridiag(ovl_lattice* lat, int32_t rhs, int32_t k_cap, int32_t* k_out,
                           void* alpha, void* beta, void* delta);

/* ----------------------------------------------------------------- host-side pieces */

/* y = sign(T) e_1 for the k x k tridiagonal T (diagonal alpha[k], super beta[k-1],
 * sub delta[k-1], complex128), written to y[k] complex128 (Section 2: f of the small
 * projected matrix). Host-only, FP64. method 0 = automatic (3, then 1, then 2 up to k = 200),
 * 1 = O(k^2) complex-symmetric QL with replayed rotations, 2 = dense scaled Newton (O(k^3)),
 * 3 = rational route: g_s(c T) e_1 of Section 5 (Eq. pfe_s) with c and s chosen from the Ritz
 * values by Theorem 1's bound, two tridiagonal solves per pole, accepted when the involution
 * residual |g(cT) y - e_1| is below 1e-11.
 * Errors: EINVAL; EILLPOSED when a Ritz value lies on the imaginary axis; ENOCONV when the
 * chosen route misses its accuracy check. */
ovl_status ovl_small_sign(int32_t k, const void* alpha, const void* beta, const void* delta,
                          void* y, int32_t method);

/* Rational approximation g(t) = t sum_i omega_i / (t^2 - sigma_i) of sign(t) (Section 5).
 * kind OVL_RAT_NEUBERGER: Eq. pfe_s with c and s from [lo, hi] (Eq. no_of_poles with
 *   the circle heuristic of Section 6) unless s > 0 is given.
 * kind OVL_RAT_ZOLOTAREV: best approximation on [-hi,-lo] u [lo,hi] with s > 0 poles.
 * omega/sigma receive s_cap entries at most; *s_out = s; *err_out = the approximation's
 * bound (Theorem 1 eps for Neuberger, equioscillation level for Zolotarev). Host-only.
 * Errors: EINVAL (lo <= 0, hi <= lo, s_cap too small). */
ovl_status ovl_rational_coeffs(int32_t kind, int32_t s, double lo, double hi, double eps,
                               int32_t s_cap, double* omega, double* sigma, int32_t* s_out,
                               double* err_out);

/* ----------------------------------------------------------------- serving */

typedef struct {
  int64_t mem_budget_bytes; /* device bytes the server may hold for request state */
  int32_t max_slots;        /* concurrent requests on the device */
  int32_t streams;          /* CUDA streams used for concurrent slots */
} ovl_server_cfg;

typedef struct {
  int32_t field_id;         /* from ovl_server_add_field */
  int32_t nrhs;
  double mu;
  double m_W;
  double tol;
  int32_t k_max;
  int32_t precision;        /* OVL_PREC_* */
  const void* b;            /* host complex128 [nrhs][n]; copied during ovl_submit */
  int32_t method;           /* OVL_DIRECT_2SL (0) | OVL_MULTISHIFT_BICG (FP32 / FP16-link precisions
                               refine with FP64 reliable updates below tol 2e-6) */
  int32_t use_deflation;    /* 1: the field's deflation set (ovl_set_deflation on the field, same m_W, mu) */
  int32_t rational_kind;    /* multishift: OVL_RAT_NEUBERGER | OVL_RAT_ZOLOTAREV */
  int32_t s;                /* multishift: poles (0: Eq. no_of_poles from the bounds, Neuberger) */
  double spec_lo, spec_hi;  /* multishift: bounds of |lambda| of the (deflated) spectrum */
  int32_t two_pass;         /* direct: 1 = two-pass strategy (Section 2.3): device memory O(n) per
                               source instead of the k_max + 1 basis columns, twice the stencils */
} ovl_request;

/* A request loop on worker threads: requests are admitted when their device footprint fits
 * the memory budget and a slot is free, the least estimated work first (sites x nrhs x k_max)
 * unless the oldest request has waited more than 2 s; admitted requests run concurrently
 * (continuous batching across streams). The admission order does not change any result.
 * A field's links and deflation set are read at every solve: ovl_set_links / ovl_set_deflation
 * on a field take effect for requests admitted afterwards and return OVL_EBUSY while a solve is
 * reading them; ovl_destroy_lattice on a field returns OVL_EBUSY until its server is destroyed. */
ovl_status ovl_server_create(ovl_ctx* ctx, const ovl_server_cfg* cfg, ovl_server** out);
ovl_status ovl_server_add_field(ovl_server* srv, ovl_lattice* lat, int32_t* field_id);
/* Enqueue; *ticket identifies the request. EINVAL for a request that can never fit. */
ovl_status ovl_submit(ovl_server* srv, const ovl_request* req, uint64_t* ticket);
/* OVL_PENDING while running; else the request's final status, with info[nrhs] and
 * x_out (host complex128 [nrhs][n], may be NULL) written once. ENOTFOUND: unknown ticket. */
ovl_status ovl_poll(ovl_server* srv, uint64_t ticket, ovl_sign_info* info, void* x_out);
ovl_status ovl_server_destroy(ovl_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* OVL_H */
