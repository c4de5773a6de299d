// GPU factorization (placeholder until the batched setup kernels land).
#include "internal.h"

namespace hifcn {
int gpu_setup(Handle *h, const double *a_nodes, cudaStream_t s) {
  (void)h; (void)a_nodes; (void)s;
  set_last_error("GPU setup not available in this build");
  return HIF_EINVAL;
}
}  // namespace hifcn
