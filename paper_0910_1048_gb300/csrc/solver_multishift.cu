// Multishift BiCG on A^2 with a rational sign approximation (Algorithm 3 + Section 5).
#include "kernels.h"

namespace ovl {

struct MultiWS {};
void free_multi_ws(MultiWS* w) { delete w; }

ovl_status solve_multishift(ovl_lattice*, const ovl_sign_params*, int, const double2*, double2*, ovl_sign_info*,
                            cudaStream_t) {
  set_error("apply_sign: multishift method not available in this build");
  return OVL_EINVAL;
}

}  // namespace ovl
