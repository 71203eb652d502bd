// Batched independent states: apply plans[i] to states[i] for all i.
#include "internal.h"

using namespace pr;

extern "C" {

int batch_run(sv_state **states, sv_plan **plans, size_t count, int use_graph) {
  (void)use_graph;
  if (count && (!states || !plans)) return fail(SV_EINVAL, "NULL arrays");
  for (size_t i = 0; i < count; ++i) {
    if (!states[i] || !plans[i]) return fail(SV_EINVAL, "NULL entry %zu", i);
    int rc = apply_plan(states[i], plans[i]);
    if (rc) return rc;
  }
  return SV_OK;
}

}  // extern "C"
