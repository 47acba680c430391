// FP32 instances of the resident CADMM kernel with the stall rule
// (top_problem.stall_checks; fixed rho).
#include "top_resident.cuh"

namespace top {
int launch_resident_stall_f32(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream) {
  return launch_resident_stall_t<float>(a, nblocks, C, smem, fam, stream);
}
}  // namespace top
