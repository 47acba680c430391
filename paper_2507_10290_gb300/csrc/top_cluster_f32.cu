// FP32 instantiations of the cluster-resident kernel (top_cluster.cuh).
#include "top_cluster.cuh"

namespace top {
int launch_cluster_f32(const ClusterArgs &a, int nclusters, int csz, int C, int ln, size_t smem, int fam,
                       void *stream) {
  return launch_cluster_t<float>(a, nclusters, csz, C, ln, smem, fam, stream);
}
int cluster_max_size_f32(int C, int ln, size_t smem, int fam) { return cluster_max_size_t<float>(C, ln, smem, fam); }
void *cluster_lanes_kernel_f32(int fam, int ln) {
  return ln == 2 ? cluster_lanes2_kernel_f32(fam) : ln == 4 ? cluster_lanes4_kernel_f32(fam) : nullptr;
}
}  // namespace top
