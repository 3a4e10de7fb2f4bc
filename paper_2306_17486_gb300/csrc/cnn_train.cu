// Training forward and backward of the network (filled in with the training kernels).
#include "cnn_impl.h"

namespace helm {

int cnn_forward_train(helm_cnn*, const helm_problem*, const float2*, float2*, int, Carve&, cudaStream_t) {
  set_error("cnn: training forward not built");
  return HELM_EINVAL;
}

}  // namespace helm
