// FP64 instantiations of the resident CADMM kernel.
#include "top_resident.cuh"

namespace top {
int launch_resident_f64(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream) {
  return launch_resident_t<double>(a, nblocks, C, smem, fam, stream);
}
}  // namespace top
