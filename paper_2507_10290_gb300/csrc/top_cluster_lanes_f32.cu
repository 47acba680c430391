// FP32 instantiations of the cluster-resident kernel with 2 or 4 lanes per
// segment (top_cluster.cuh: the sample rows of the box / ball / velocity-norm
// families split over a segment's lanes; fixed rho).
#include "top_cluster.cuh"

namespace top {
template <int LN>
static void *lanes_kernel(int fam) {
  switch (fam) {
    case 1: return (void *)cluster_kernel<float, 1, false, LN>;
    case 2: return (void *)cluster_kernel<float, 2, false, LN>;
    case 3: return (void *)cluster_kernel<float, 3, false, LN>;
    case 4: return (void *)cluster_kernel<float, 4, false, LN>;
    case 5: return (void *)cluster_kernel<float, 5, false, LN>;
    case 6: return (void *)cluster_kernel<float, 6, false, LN>;
    case 7: return (void *)cluster_kernel<float, 7, false, LN>;
    default: return nullptr;
  }
}

void *cluster_lanes_kernel_f32(int fam, int ln) {
  return ln == 2 ? lanes_kernel<2>(fam) : ln == 4 ? lanes_kernel<4>(fam) : nullptr;
}
}  // namespace top
