// Learned right preconditioner (placeholder state until a network is set).
#include "vie_internal.cuh"

namespace vie {

void free_precond(vie_plan* p) { (void)p; }

vie_status precond_get(vie_plan* p, vie_precond_fn* fn, void** ctx) {
  (void)p;
  *fn = nullptr;
  *ctx = nullptr;
  set_error("no preconditioner has been set on this plan");
  return VIE_ERR_INVALID;
}

}  // namespace vie
