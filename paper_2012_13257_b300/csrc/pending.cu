// Entry points whose kernels are not built yet: they reject every call.
#include "api_internal.h"


extern "C" {
gmi_status gmi_server_config_default(gmi_server_config*) { return GMI_ERR_UNSUPPORTED; }
gmi_status gmi_server_create(const gmi_server_config*, gmi_server** out) {
  if (out) *out = nullptr;
  return GMI_ERR_UNSUPPORTED;
}
gmi_status gmi_server_submit(gmi_server*, const float*, const float*, int64_t, int, int, float, float*, uint64_t*) { return GMI_ERR_UNSUPPORTED; }
gmi_status gmi_server_wait(gmi_server*, uint64_t, int, double*) { return GMI_ERR_UNSUPPORTED; }
gmi_status gmi_server_poll(gmi_server*, uint64_t) { return GMI_ERR_UNSUPPORTED; }
gmi_status gmi_server_stats(gmi_server*, uint64_t*, uint64_t*, uint64_t*, size_t*) { return GMI_ERR_UNSUPPORTED; }
gmi_status gmi_server_destroy(gmi_server*) { return GMI_OK; }
}
