// FP64 instantiation of the adjoint through the unrolled CADMM iterations.
#include "top_stream.cuh"
#include "top_adjoint.cuh"

namespace top {
int launch_adjoint_f64(const StreamArgs &f, const AdjArgs &a, int ckpt, void *const *ck, void *const *tape,
                       const size_t *bytes, double *dw, double *dT, void *stream) {
  return run_adjoint_t<double>(f, a, ckpt, ck, tape, bytes, dw, dT, stream);
}
}  // namespace top
