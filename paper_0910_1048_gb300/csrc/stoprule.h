// Stopping rule and evaluation schedule of the direct method (shared by the allocating and the
// allocation-free drivers so that both stop at the same k).
//
// The paper fixes k a priori (Algorithm 4). Here y_j = sign(H_j) e_1 is evaluated at a sparse
// set of steps k_1 < k_2 < ...; at each, d_i = ||V(y_{k_i} - [y_{k_{i-1}}; 0])|| / ||V y_{k_i}|| is
// the relative change of x since the previous evaluation. Krylov approximations of sign(A) b
// converge roughly geometrically, e(k) ~ C rho^k, so d_i ~ e(k_{i-1}) (1 - rho^{D_i}) with
// D_i = k_i - k_{i-1}, and the error at k_i is estimated as
//     e_i = d_i rho^{D_i} / (1 - rho^{D_i}),
// with log rho from the last two changes (log(d_i/d_{i-1}) over the mean spacing). A rhs stops
// when d_i <= tol (the change itself is small) or, with a rate, when 2 e_i <= tol. Each rhs keeps
// its own schedule: its next evaluation goes where it is predicted to reach tol/2, within
// [k+chunk, 1.5 k]; without a rate it is 1.25 k. A rhs therefore stops at the same k whether it
// is solved alone or in a batch.
#pragma once

#include <algorithm>
#include <cmath>

namespace ovl {

struct StopTrack {
  int k_prev = 0;        // step of the previous evaluation
  double d_prev = 0;     // its relative change (0: none yet)
  int dk_prev = 0;       // its spacing
  double log_rho = 0;    // per-step log rate (< 0 when known)
  double err = 1e300;    // current error estimate
  int next = 0;          // step count at which this rhs is evaluated next
};

// Record evaluation at step k with relative change d (d < 0: first evaluation, no change yet).
inline void stop_record(StopTrack& t, int k, double d) {
  if (d < 0) {
    t.k_prev = k;
    t.err = 1e300;
    return;
  }
  const int dk = k - t.k_prev;
  t.log_rho = 0;
  if (t.d_prev > 0 && d > 0 && d < t.d_prev && dk > 0 && t.dk_prev > 0)
    t.log_rho = std::log(d / t.d_prev) / (0.5 * (dk + t.dk_prev));
  if (t.log_rho < 0) {
    double q = std::exp(t.log_rho * dk);  // rho^D
    t.err = d * q / (1.0 - q);
  } else {
    t.err = d;
  }
  t.d_prev = d;
  t.dk_prev = dk;
  t.k_prev = k;
}

inline bool stop_converged(const StopTrack& t, double tol) {
  return t.d_prev > 0 && (t.d_prev <= tol || (t.log_rho < 0 && 2.0 * t.err <= tol));
}

// Steps after k at which this rhs is predicted to reach tol / 2 (or -1 without a rate).
inline double stop_predict(const StopTrack& t, double tol) {
  if (!(t.log_rho < 0) || !(t.err < 1e299)) return -1;
  return std::max(0.0, std::log(0.5 * tol / t.err) / t.log_rho);
}

inline int stop_next_eval(int k, int chunk, double steps_needed) {
  double jn = steps_needed < 0 ? 1.25 * k : std::min(1.5 * k, std::max((double)k + chunk, k + steps_needed));
  return std::max(k + chunk, (int)jn);
}

// Schedule the next evaluation of a rhs evaluated at step k.
inline void stop_schedule(StopTrack& t, int k, int chunk, double tol) {
  t.next = stop_next_eval(k, chunk, stop_predict(t, tol));
}

// Is a rhs due for evaluation at a snapshot of k steps? (Always at the last snapshot, and at once
// when it stopped on the device.)
inline bool stop_due(const StopTrack& t, int k, bool final_snapshot, bool stopped_on_device) {
  return final_snapshot || stopped_on_device || k >= t.next;
}

}  // namespace ovl
