// Batched evaluation of many problems of one model in one persistent launch.
#include "ocp_internal.h"

using namespace ocpg;

extern "C" {

ocp_status ocp_batch_create(ocp_t* const* items, int count, ocp_batch_t** out) {
  (void)items; (void)count;
  if (out) *out = nullptr;
  return set_err(nullptr, OCP_EMODEL, "batched evaluation is not available in this build");
}

void ocp_batch_destroy(ocp_batch_t* b) { delete b; }

ocp_status ocp_batch_offsets(const ocp_batch_t* b, int64_t*, int64_t*, int64_t*, int64_t*) {
  return b ? OCP_EMODEL : OCP_EINVAL;
}

ocp_status ocp_batch_set_config(ocp_batch_t* b, int, int) { return b ? OCP_EMODEL : OCP_EINVAL; }

ocp_status ocp_batch_eval_all(ocp_batch_t* b, const double*, const double*, double, double*, double*, double*,
                              double*, void*) {
  return b ? OCP_EMODEL : OCP_EINVAL;
}

}  // extern "C"
