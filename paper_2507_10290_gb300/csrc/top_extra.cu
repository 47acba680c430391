// top_extra.cu -- kernels around the iteration: sampling trajectories at
// uniform times (the evaluation behind the similarity metric of Sec. IV-A.2)
// and the log-space duration step of the outer time allocation.
#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"

namespace top {

// start time of every segment within its trajectory and each trajectory's
// total duration (one thread per trajectory, in segment order)
__global__ void traj_times_kernel(const int32_t *__restrict__ off, const double *__restrict__ T, int B,
                                  double *__restrict__ tstart, double *__restrict__ ttot) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int g = off[b]; g < off[b + 1]; ++g) {
      tstart[g] = acc;
      acc += T[g];
    }
    ttot[b] = acc;
  }
}

// derivative `order` of sigma_i(t) = sum_k c_k (t - t_{i-1})^k at the M times
// t_m = m T_b / (M - 1); at a junction the later segment is used
__global__ void sample_kernel(const int32_t *__restrict__ off, const double *__restrict__ tstart,
                              const double *__restrict__ ttot, const double *__restrict__ coeffs, int B, int M,
                              int order, double *__restrict__ out) {
  const long long n = (long long)B * M;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = int(q / M), m = int(q % M);
    const int g0 = off[b], g1 = off[b + 1];
    double *o = out + q * 3;
    if (g1 <= g0) {
      o[0] = o[1] = o[2] = 0.0;
      continue;
    }
    const double t = (m == M - 1) ? ttot[b] : double(m) * ttot[b] / double(M - 1);
    int lo = g0, hi = g1 - 1;  // last segment whose start is <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tstart[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const double tau = t - tstart[lo];
    for (int a = 0; a < 3; ++a) {
      const double *c = coeffs + ((size_t)lo * 3 + a) * NC;
      double acc = 0.0;  // Horner over k = order..7 of F(k, order) c_k tau^(k - order)
      for (int k = NC - 1; k >= order; --k) acc = acc * tau + double(falling(k, order)) * c[k];
      o[a] = acc;
    }
  }
}

// T_i <- T_i exp(-clamp(lr T_i (dJ/dT_i + k_T), -0.5, 0.5)): a gradient step in log T
__global__ void time_step_kernel(double *__restrict__ T, const double *__restrict__ dT, int S, double kT, double lr) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < S; g += gridDim.x * blockDim.x) {
    double x = lr * T[g] * (dT[g] + kT);
    x = x > 0.5 ? 0.5 : (x < -0.5 ? -0.5 : x);
    T[g] = T[g] * exp(-x);
  }
}

int launch_sample(const int32_t *off, const double *T, int B, int M, int order, const double *coeffs,
                  double *tstart, double *ttot, double *out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (B <= 0) return 0;
  int bt = (B + 127) / 128;
  if (bt > sm_count() * 8) bt = sm_count() * 8;
  traj_times_kernel<<<bt, 128, 0, st>>>(off, T, B, tstart, ttot);
  const long long n = (long long)B * M;
  long long bs = (n + 255) / 256;
  if (bs > sm_count() * 16) bs = sm_count() * 16;
  sample_kernel<<<(int)bs, 256, 0, st>>>(off, tstart, ttot, coeffs, B, M, order, out);
  return (int)cudaGetLastError();
}

int launch_time_step(double *T, const double *dT, int S, double kT, double lr, void *stream) {
  if (S <= 0) return 0;
  int blocks = (S + 255) / 256;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  time_step_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(T, dT, S, kT, lr);
  return (int)cudaGetLastError();
}

}  // namespace top
