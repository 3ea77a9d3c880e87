// Batched execution of independent problems (placeholder until the batched scheduler lands).
#include "sidp.h"

struct sidp_batch {
  int unused;
};

extern "C" {
sidp_status sidp_batch_create(sidp_batch** out, const sidp_config*, int, void*) {
  if (out) *out = nullptr;
  return SIDP_ERR_ARG;
}
sidp_status sidp_batch_destroy(sidp_batch*) { return SIDP_OK; }
sidp_status sidp_batch_sizes(const sidp_batch*, int, long long*, int*) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_total_nodes(const sidp_batch*, long long*) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_node_coords(const sidp_batch*, int, double*, double*) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_set_state(sidp_batch*, int, const double*) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_get_state(sidp_batch*, int, double*) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_step(sidp_batch*, int) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_get_diag(sidp_batch*, int, sidp_diag*) { return SIDP_ERR_ARG; }
sidp_status sidp_batch_synchronize(sidp_batch*) { return SIDP_ERR_ARG; }
const char* sidp_batch_last_error(const sidp_batch*) { return "batched execution not built yet"; }
}
