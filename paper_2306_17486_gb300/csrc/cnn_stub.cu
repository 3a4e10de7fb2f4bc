// Placeholder for the CNN preconditioner hooks until the network kernels land.
#include "problem.h"

namespace helm {
int launch_cnn_precond(const helm_problem*, const helm_cnn*, const float2*, float2*, int, Carve&,
                       const VcycleScratch&, const int*, cudaStream_t) {
  set_error("CNN preconditioner not built");
  return HELM_EINVAL;
}
size_t cnn_workspace_bytes(const helm_problem*, const helm_cnn*, int) { return 0; }
}  // namespace helm
