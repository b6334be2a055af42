// Request server (continuous batching).
#include "common.h"

extern "C" {
ovl_status ovl_server_create(ovl_ctx*, const ovl_server_cfg*, ovl_server**) { ovl::set_error("server: not available"); return OVL_EINVAL; }
ovl_status ovl_server_add_field(ovl_server*, ovl_lattice*, int32_t*) { return OVL_EINVAL; }
ovl_status ovl_submit(ovl_server*, const ovl_request*, uint64_t*) { return OVL_EINVAL; }
ovl_status ovl_poll(ovl_server*, uint64_t, ovl_sign_info*, void*) { return OVL_EINVAL; }
ovl_status ovl_server_destroy(ovl_server*) { return OVL_OK; }
}
