// top_kinv.cu -- FP64 assembly and inversion of the local KKT matrix of
// Eq. 18a, one matrix per segment.
//
// The 24x24 matrix 2 Qt + rho Mt^T E Mt + rho Ao^T Ao + rho sum_j A_j^T A_j is
// I_3 (x) K8 for every constraint family the library supports (the box rows
// are per-axis and the ball / velocity sample matrices are I_3 (x) beta^T),
// so one 8x8 block per segment is formed, in the normalised coordinates
// ch_k = c_k T^k (see top_math.cuh):
//   Kh = 2 T^-7 Qh
//      + rho sum_{start rows r} (r! s_r)^2 e_r e_r^T
//      + rho sum_{end rows r}   s_r^2 F(.,r) F(.,r)^T
//      + 2 rho s_1^2 sum_j a_j a_j^T          (box: rows +-e_a (x) beta'(t_j))
//      +   rho       sum_j b_j b_j^T          (ball: position samples)
//      +   rho s_1^2 sum_j a_j a_j^T          (velocity-norm samples)
// with a_j[k] = k tau_j^{k-1}, b_j[k] = tau_j^k, tau_j = j / M, and the
// consensus rows of order >= p dropped at the trajectory's two ends.  Kh is
// Jacobi-equilibrated, factorised by Cholesky and inverted in FP64; the
// packed inverse is written in FP64 and rounded to FP32 for the FP32 path.
#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"

namespace top {

__device__ __forceinline__ int find_traj(const int32_t *off, int B, int g) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void kinv_kernel(const DevProblem p, double rho, float *__restrict__ G32,
                            double *__restrict__ G64, int *__restrict__ err) {
  const int S = p.S;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < S; g += gridDim.x * blockDim.x) {
    const int b = find_traj(p.seg_offset, p.B, g);
    const int i = g - p.seg_offset[b];
    const int N = p.seg_offset[b + 1] - p.seg_offset[b];
    const bool first = (i == 0), last = (i == N - 1);
    const double T = p.durations[g];
    if (!(T > 0.0) || !(T < 1e30)) {
      atomicOr(err, 1);
      continue;
    }
    double s[NC];
    s[0] = 1.0;
    for (int r = 1; r < NC; ++r) s[r] = s[r - 1] / T;
    double K[NC][NC];
    const double t7 = s[7];
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
      for (int l = 0; l < NC; ++l) K[k][l] = 2.0 * t7 * qhat(k, l);
    // consensus rows (Mt^T E Mt)
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      if (!(first && r >= PO)) {
        const double v = double(fact(r)) * s[r];
        K[r][r] += rho * v * v;
      }
      if (!(last && r >= PO)) {
        const double w = rho * s[r] * s[r];
#pragma unroll
        for (int k = r; k < NC; ++k)
#pragma unroll
          for (int l = r; l < NC; ++l) K[k][l] += w * double(falling(k, r)) * double(falling(l, r));
      }
    }
    auto add_samples = [&](int M, int order, double weight) {
      for (int j = 1; j <= M; ++j) {
        const double tau = double(j) / double(M);
        double a[NC];
        for (int k = 0; k < NC; ++k) {
          if (order == 0) {
            double t = 1.0;
            for (int q = 0; q < k; ++q) t *= tau;
            a[k] = t;
          } else {
            double t = 1.0;
            for (int q = 0; q < k - 1; ++q) t *= tau;
            a[k] = (k == 0) ? 0.0 : double(k) * t;
          }
        }
        for (int k = 0; k < NC; ++k)
          for (int l = 0; l < NC; ++l) K[k][l] += weight * a[k] * a[l];
      }
    };
    if (p.inner == 0) {
      if (p.M_box > 0) add_samples(p.M_box, 1, 2.0 * rho * s[1] * s[1]);
      if (p.M_ball > 0) add_samples(p.M_ball, 0, rho);
      if (p.M_vn > 0) add_samples(p.M_vn, 1, rho * s[1] * s[1]);
    }
    // Jacobi equilibration + Cholesky + inverse, all FP64
    double d[NC];
    bool ok = true;
    for (int k = 0; k < NC; ++k) {
      ok = ok && (K[k][k] > 0.0);
      d[k] = ok ? 1.0 / sqrt(K[k][k]) : 0.0;
    }
    double L[NC][NC];
    for (int k = 0; k < NC; ++k)
      for (int l = 0; l < NC; ++l) L[k][l] = 0.0;
    for (int j = 0; j < NC && ok; ++j) {
      double dd = d[j] * K[j][j] * d[j];
      for (int q = 0; q < j; ++q) dd -= L[j][q] * L[j][q];
      if (!(dd > 0.0)) { ok = false; break; }
      const double ljj = sqrt(dd);
      L[j][j] = ljj;
      for (int r = j + 1; r < NC; ++r) {
        const double kk = (r > j) ? K[j][r] : K[r][j];  // K upper part is complete (symmetric fill)
        double a = d[r] * kk * d[j];
        for (int q = 0; q < j; ++q) a -= L[r][q] * L[j][q];
        L[r][j] = a / ljj;
      }
    }
    if (!ok) {
      atomicOr(err, 2);
      continue;
    }
    // inverse of L (lower), then (L L^T)^-1 = L^-T L^-1
    double Li[NC][NC];
    for (int c = 0; c < NC; ++c) {
      for (int r = 0; r < NC; ++r) {
        if (r < c) { Li[r][c] = 0.0; continue; }
        double a = (r == c) ? 1.0 : 0.0;
        for (int q = c; q < r; ++q) a -= L[r][q] * Li[q][c];
        Li[r][c] = a / L[r][r];
      }
    }
    for (int k = 0; k < NC; ++k)
      for (int l = k; l < NC; ++l) {
        double a = 0.0;
        for (int q = l; q < NC; ++q) a += Li[q][k] * Li[q][l];
        const double v = d[k] * a * d[l];
        const int idx = gidx(k, l);
        if (G64) G64[size_t(idx) * S + g] = v;
        if (G32) G32[size_t(idx) * S + g] = float(v);
      }
  }
}

int launch_kinv(const DevProblem &p, double rho, void *G32, void *G64, int *err_flag, void *stream) {
  if (p.S == 0) return 0;
  const int threads = 128;
  int blocks = (p.S + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  kinv_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(p, rho, (float *)G32, (double *)G64, err_flag);
  return (int)cudaGetLastError();
}

}  // namespace top
