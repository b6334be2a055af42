// Host-only checks of the direct method's stopping rule (csrc/stoprule.h), built by
// tests/test_stoprule_host.py with the host compiler and driven through ctypes.
#include <cmath>

#include "../../paper_0910_1048_gb300/csrc/stoprule.h"

extern "C" {

// Feed the changes d_i = e(k_{i-1}) - e(k_i) of an error that decays exactly as e(k) = C rho^k
// at the steps k[0..n-1] (k[0]: first evaluation, no change yet); return the last estimate, the
// rate it found, whether it stopped at tol, and the predicted steps to tol / 2.
void feed_geometric(double c, double rho, const int* k, int n, double tol, double* est, double* log_rho,
                    int* converged, double* predict) {
  ovl::StopTrack t;
  ovl::stop_record(t, k[0], -1.0);
  for (int i = 1; i < n; ++i) {
    const double d = c * (std::pow(rho, k[i - 1]) - std::pow(rho, k[i]));
    ovl::stop_record(t, k[i], d);
  }
  *est = t.err;
  *log_rho = t.log_rho;
  *converged = ovl::stop_converged(t, tol) ? 1 : 0;
  *predict = ovl::stop_predict(t, tol);
}

int next_eval(int k, int chunk, double steps_needed) { return ovl::stop_next_eval(k, chunk, steps_needed); }

int due(int next, int k, int final_snapshot, int stopped) {
  ovl::StopTrack t;
  t.next = next;
  return ovl::stop_due(t, k, final_snapshot != 0, stopped != 0) ? 1 : 0;
}

}
