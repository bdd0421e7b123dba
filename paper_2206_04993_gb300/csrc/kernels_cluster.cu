// Cluster path: placeholder until the fused kernel lands.
#include "internal.h"

namespace sgep {
bool cluster_supported(const Ctx&, const char** why) {
  if (why) *why = "not built yet";
  return false;
}
int cluster_alloc(Ctx&) { return SGEP_ENOTSUP; }
void cluster_free(Ctx&) {}
int cluster_step(Ctx&, const void*, const void*, int64_t, float, float, cudaStream_t) { return SGEP_ENOTSUP; }
int cluster_flush(Ctx&, cudaStream_t) { return SGEP_ENOTSUP; }
int cluster_products(Ctx&, float*, float*, cudaStream_t) { return SGEP_ENOTSUP; }
}  // namespace sgep
