// FP32 instantiations of the resident CADMM kernel (FP32 state and arithmetic,
// FP64 residual and cost reductions).
#include "top_resident.cuh"

namespace top {
int launch_resident_f32(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream) {
  return launch_resident_t<float>(a, nblocks, C, smem, fam, stream);
}
}  // namespace top
