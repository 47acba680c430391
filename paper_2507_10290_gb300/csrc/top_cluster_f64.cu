// FP64 instantiations of the cluster-resident kernel (top_cluster.cuh).
#include "top_cluster.cuh"

namespace top {
int launch_cluster_f64(const ClusterArgs &a, int nclusters, int csz, int C, int ln, size_t smem, int fam,
                       void *stream) {
  return launch_cluster_t<double>(a, nclusters, csz, C, ln, smem, fam, stream);
}
int cluster_max_size_f64(int C, int ln, size_t smem, int fam) { return cluster_max_size_t<double>(C, ln, smem, fam); }
int cluster_max_size(int C, int ln, size_t smem, int fam, bool fp64) {
  return fp64 ? cluster_max_size_f64(C, ln, smem, fam) : cluster_max_size_f32(C, ln, smem, fam);
}
}  // namespace top
