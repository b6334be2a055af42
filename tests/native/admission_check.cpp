// Host-only driver of the request server's admission policy (csrc/admission.h), built by
// tests/test_admission_host.py with the host compiler and called through ctypes.
#include <cstddef>
#include <vector>

#include "../../paper_0910_1048_gb300/csrc/admission.h"

extern "C" long pick(const double* footprint, const double* work, long n, double in_use, double budget,
                     double waited_oldest, double max_wait) {
  std::vector<ovl::PendingRequest> q((size_t)n);
  for (long i = 0; i < n; ++i) q[(size_t)i] = {(size_t)footprint[i], work[i]};
  return ovl::admission_pick(q.data(), q.size(), (size_t)in_use, (size_t)budget, waited_oldest, max_wait);
}
