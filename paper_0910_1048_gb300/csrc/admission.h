// Admission policy of the request server (host-only, no CUDA): which queued request a free
// slot takes next.
//
// Among the queued requests whose device footprint fits what the memory budget has left, the one
// with the least estimated work; but once the oldest request has waited longer than max_wait it
// goes first, and while it does not fit nothing is admitted past it (no starvation of large
// requests).
#pragma once

#include <cstddef>

namespace ovl {

struct PendingRequest {
  size_t footprint;  // device bytes while it runs
  double work;       // estimated work (sites x right-hand sides x k_max, FP32 at half weight)
};

// q[0..n-1] in arrival order; waited_oldest: seconds the oldest (q[0]) has waited. Returns the
// queue position to admit, or -1 when nothing may be admitted now.
inline long admission_pick(const PendingRequest* q, size_t n, size_t in_use, size_t budget, double waited_oldest,
                           double max_wait) {
  if (n == 0) return -1;
  if (waited_oldest > max_wait) return in_use + q[0].footprint <= budget ? 0 : -1;
  long best = -1;
  double best_work = 0;
  for (size_t i = 0; i < n; ++i) {
    if (in_use + q[i].footprint > budget) continue;
    if (best < 0 || q[i].work < best_work) best = (long)i, best_work = q[i].work;
  }
  return best;
}

}  // namespace ovl
