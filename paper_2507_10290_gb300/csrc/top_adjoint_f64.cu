// FP64 instantiation of the adjoint through the unrolled CADMM iterations.
#include "top_stream.cuh"
#include "top_adjoint.cuh"
#include "top_adjres.cuh"

namespace top {
int launch_adjoint_f64(const StreamArgs &f, const AdjArgs &a, int fam, int ckpt, void *const *ck, void *const *tape,
                       const size_t *bytes, double *dw, double *dT, void *stream) {
  return run_adjoint_t<double>(f, a, fam, ckpt, ck, tape, bytes, dw, dT, stream);
}
int launch_adjres_f64(const AdjResArgs &a, int nblocks, int C, size_t smem, void *stream) {
  return launch_adjres_t<double>(a, nblocks, C, smem, stream);
}
}  // namespace top
