// FP32 instantiations of the cluster-resident kernel with 2 lanes per segment
// (top_cluster.cuh: a segment's sample rows of the box / ball / velocity-norm
// and polytope families split over its lanes; fixed rho).
#include "top_cluster.cuh"

namespace top {
void *cluster_lanes2_kernel_f32(int fam) {
  switch (fam) {
    case 1: return (void *)cluster_kernel<float, 1, false, 2>;
    case 2: return (void *)cluster_kernel<float, 2, false, 2>;
    case 3: return (void *)cluster_kernel<float, 3, false, 2>;
    case 4: return (void *)cluster_kernel<float, 4, false, 2>;
    case 5: return (void *)cluster_kernel<float, 5, false, 2>;
    case 6: return (void *)cluster_kernel<float, 6, false, 2>;
    case 7: return (void *)cluster_kernel<float, 7, false, 2>;
    case 16: return (void *)cluster_kernel<float, 16, false, 2>;
    case 17: return (void *)cluster_kernel<float, 17, false, 2>;
    case 18: return (void *)cluster_kernel<float, 18, false, 2>;
    case 19: return (void *)cluster_kernel<float, 19, false, 2>;
    case 20: return (void *)cluster_kernel<float, 20, false, 2>;
    case 21: return (void *)cluster_kernel<float, 21, false, 2>;
    case 22: return (void *)cluster_kernel<float, 22, false, 2>;
    case 23: return (void *)cluster_kernel<float, 23, false, 2>;
    default: return nullptr;
  }
}
}  // namespace top
