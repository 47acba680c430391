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
// Jacobi-equilibrated, factorised by Cholesky and inverted in FP64, all in
// one packed lower triangle held in registers (the factor and its inverse
// overwrite the matrix); the packed inverse is written in FP64 or rounded to
// FP32 for the FP32 path.
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

// packed lower triangle, i >= j
__host__ __device__ constexpr int lidx(int i, int j) { return i * (i + 1) / 2 + j; }

__device__ __forceinline__ void add_sample_rows(double (&A)[NG], int M, int order, double weight) {
  for (int j = 1; j <= M; ++j) {
    const double tau = double(j) / double(M);
    double a[NC];
    double t = 1.0;  // tau^(k - order) built incrementally
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if (order == 0) {
        a[k] = t;
        t *= tau;
      } else {
        a[k] = (k == 0) ? 0.0 : double(k) * t;
        if (k >= 1) t *= tau;
      }
    }
#pragma unroll
    for (int r = 0; r < NC; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) A[lidx(r, c)] += weight * a[r] * a[c];
  }
}

// column J of the in-place Cholesky factorisation (recursion keeps every
// index a compile-time constant, so the packed matrix stays in registers)
template <int J>
__device__ __forceinline__ void chol_col(double (&A)[NG], double (&inv)[NC], bool &ok) {
  double dd = A[lidx(J, J)];
#pragma unroll
  for (int k = 0; k < J; ++k) dd -= A[lidx(J, k)] * A[lidx(J, k)];
  ok = ok && (dd > 0.0);
  const double ddp = dd > 0.0 ? dd : 1.0;
  inv[J] = rsqrt(ddp);          // 1 / L_JJ
  A[lidx(J, J)] = ddp * inv[J];  // L_JJ = sqrt(dd)
#pragma unroll
  for (int r = J + 1; r < NC; ++r) {
    double a = A[lidx(r, J)];
#pragma unroll
    for (int k = 0; k < J; ++k) a -= A[lidx(r, k)] * A[lidx(J, k)];
    A[lidx(r, J)] = a * inv[J];
  }
  if constexpr (J + 1 < NC) chol_col<J + 1>(A, inv, ok);
}

// the rho-weighted terms of the local matrix: consensus rows (Mt^T E Mt) and
// the sample rows of the closed-form constraint families, each times `rho`
template <bool SAMPLES>
__device__ __forceinline__ void add_rho_terms(const DevProblem &p, const double (&s)[NC], bool first, bool last,
                                              double rho, double (&A)[NG]) {
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    if (!(first && q >= PO)) {
      const double v = double(fact(q)) * s[q];
      A[lidx(q, q)] += rho * v * v;
    }
    if (!(last && q >= PO)) {
      const double w = rho * s[q] * s[q];
      // F(r,q) F(c,q) is an integer below 2^25, formed at compile time: one FMA per entry
#pragma unroll
      for (int r = q; r < NC; ++r)
#pragma unroll
        for (int c = q; c <= r; ++c) A[lidx(r, c)] += w * double(falling(r, q) * falling(c, q));
    }
  }
  if (SAMPLES && p.inner == 0) {
    if (p.M_box > 0) add_sample_rows(A, p.M_box, 1, 2.0 * rho * s[1] * s[1]);
    if (p.M_ball > 0) add_sample_rows(A, p.M_ball, 0, rho);
    if (p.M_vn > 0) add_sample_rows(A, p.M_vn, 1, rho * s[1] * s[1]);
  }
}

// segment g's place in its trajectory and its powers s_r = T^-r; false for a
// duration that is not positive and finite
__device__ __forceinline__ bool segment_powers(const DevProblem &p, int g, double (&s)[NC]) {
  const double T = p.durations[g];
  if (!(T > 0.0) || !(T < 1e30)) return false;
  const double it = 1.0 / T;
  s[0] = 1.0;
#pragma unroll
  for (int r = 1; r < NC; ++r) s[r] = s[r - 1] * it;
  return true;
}

__device__ __forceinline__ bool segment_setup(const DevProblem &p, int g, bool &first, bool &last,
                                              double (&s)[NC]) {
  const int b = find_traj(p.seg_offset, p.B, g);
  const int i = g - p.seg_offset[b];
  const int N = p.seg_offset[b + 1] - p.seg_offset[b];
  first = (i == 0);
  last = (i == N - 1);
  const double T = p.durations[g];
  if (!(T > 0.0) || !(T < 1e30)) return false;
  const double it = 1.0 / T;
  s[0] = 1.0;
#pragma unroll
  for (int r = 1; r < NC; ++r) s[r] = s[r - 1] * it;
  return true;
}

// Jacobi equilibration (A <- D A D, D = diag(A)^-1/2), Cholesky and inversion
// of the factor, all in place: A ends as L^-1 of D A D (packed lower).
// Returns false if A is not positive definite.
__device__ __forceinline__ bool equil_chol_inv(double (&A)[NG], double (&d)[NC]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const double akk = A[lidx(k, k)];
    ok = ok && (akk > 0.0);
    d[k] = ok ? rsqrt(akk) : 0.0;
  }
  if (!ok) return false;
#pragma unroll
  for (int r = 0; r < NC; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) A[lidx(r, c)] *= d[r] * d[c];
  // Cholesky in place: A <- L (lower), inv[j] = 1 / L_jj
  double inv[NC];
  chol_col<0>(A, inv, ok);
  if (!ok) return false;
  // invert L in place, column by column: X_jj = 1/L_jj,
  // X_rj = -(1/L_rr) (L_rj X_jj + sum_{j<k<r} L_rk X_kj)
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    A[lidx(j, j)] = inv[j];
#pragma unroll
    for (int r = j + 1; r < NC; ++r) {
      double a = A[lidx(r, j)] * A[lidx(j, j)];
#pragma unroll
      for (int k = j + 1; k < r; ++k) a += A[lidx(r, k)] * A[lidx(k, j)];
      A[lidx(r, j)] = -inv[r] * a;
    }
  }
  return true;
}

// K^-1 from A = L^-1 of D K D (packed lower) and the scaling d:
// (D K D)^-1 = L^-T L^-1, so K^-1 = D L^-T L^-1 D; packed symmetric entries
// written to rows base + gidx(k, l) of the [rows][S] output
__device__ __forceinline__ void store_inverse(const double (&A)[NG], const double (&d)[NC], int S, int g, int base,
                                              float *G32, double *G64) {
  double X[NG];  // L^-1 D: column k of L^-1 times d_k, so K^-1 = X^T X
#pragma unroll
  for (int q = 0; q < NC; ++q)
#pragma unroll
    for (int k = 0; k <= q; ++k) X[lidx(q, k)] = A[lidx(q, k)] * d[k];
#pragma unroll
  for (int k = 0; k < NC; ++k)
#pragma unroll
    for (int l = k; l < NC; ++l) {
      double v = 0.0;
#pragma unroll
      for (int q = l; q < NC; ++q) v += X[lidx(q, k)] * X[lidx(q, l)];
      const size_t idx = size_t(base + gidx(k, l)) * S + g;
      if (G64) G64[idx] = v;
      if (G32) G32[idx] = float(v);
    }
}

// Interior segments of a trajectory with the same duration as its first
// interior segment have the same local matrix (it depends on T, rho, the
// sample counts and the end masks only).  kinv_mark_kernel marks them
// copy[g] = that segment and lists every other segment in `list` (list[0] =
// count, warp-aggregated appends, so a warp's entries stay in segment order;
// an entry is g with the segment's first / last flags in bits 30 / 31, so the
// inversion kernel needs no search of the offsets; g < 2^30 since the host
// keeps 108 S below 2^31);
// kinv_kernel then inverts the listed segments only and kinv_copy_kernel
// fills in the rest: a trajectory whose segments share one duration costs
// three inversions instead of N.
__global__ void kinv_mark_kernel(const DevProblem p, int *__restrict__ copy, int *__restrict__ list) {
  const int S = p.S, lane = threadIdx.x & 31;
  for (long long w0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < S;
       w0 += (long long)gridDim.x * blockDim.x) {
    const int g = int(w0) + lane;
    bool rep = false;
    unsigned entry = 0u;
    if (g < S) {
      const int b = find_traj(p.seg_offset, p.B, g);
      const int g0 = p.seg_offset[b], N = p.seg_offset[b + 1] - g0, i = g - g0;
      const bool same = i >= 2 && i <= N - 2 && p.durations[g] == p.durations[g0 + 1];
      copy[g] = same ? g0 + 1 : -1;
      rep = !same;
      entry = unsigned(g) | (i == 0 ? 1u << 30 : 0u) | (i == N - 1 ? 1u << 31 : 0u);
    }
    const unsigned m = __ballot_sync(0xffffffffu, rep);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(list, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (rep) list[1 + base + __popc(m & ((1u << lane) - 1u))] = int(entry);
  }
}

// one thread per listed segment (every segment when `list` is null)
template <bool SAMPLES>
__global__ void __launch_bounds__(128) kinv_kernel(const DevProblem p, double rho, float *__restrict__ G32,
                                                   double *__restrict__ G64, int *__restrict__ err,
                                                   const int *__restrict__ list) {
  const int S = p.S;
  const int n = list ? list[0] : S;
  if (!TOP_IN_BOUNDS(p.err, n >= 0 && n <= S)) return;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const unsigned e = list ? unsigned(list[1 + x]) : 0u;
    const int g = list ? int(e & 0x3fffffffu) : x;
    if (!TOP_IN_BOUNDS(p.err, g >= 0 && g < S)) continue;
    bool first = (e >> 30) & 1u, last = (e >> 31) & 1u;
    double s[NC];
    if (!(list ? segment_powers(p, g, s) : segment_setup(p, g, first, last, s))) {
      atomicOr(err, 1);
      continue;
    }
    double A[NG];
    const double t7x2 = 2.0 * s[7];  // the cost block 2 T^-7 Qh lives on coefficients 4..7
#pragma unroll
    for (int r = 0; r < NC; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) A[lidx(r, c)] = (r >= PO && c >= PO) ? t7x2 * qhat(r, c) : 0.0;
    add_rho_terms<SAMPLES>(p, s, first, last, rho, A);
    double d[NC];
    if (!equil_chol_inv(A, d)) {
      atomicOr(err, 2);
      continue;
    }
    store_inverse(A, d, S, g, 0, G32, G64);
  }
}

// one cyclic-Jacobi rotation of the symmetric D x D matrix C zeroing C[P][Q]
// (textbook symmetric Schur decomposition, e.g. Golub & Van Loan, Sec. 8.5),
// accumulated into the eigenvector columns of V
template <int P, int Q, int D>
__device__ __forceinline__ void jacobi_rot(double (&C)[D][D], double (&V)[D][D]) {
  const double apq = C[P][Q];
  if (apq == 0.0) return;
  const double theta = (C[Q][Q] - C[P][P]) / (2.0 * apq);
  const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
  const double c = rsqrt(1.0 + t * t), sn = t * c;
#pragma unroll
  for (int k = 0; k < D; ++k) {  // columns P, Q of C J
    const double ckp = C[k][P], ckq = C[k][Q];
    C[k][P] = c * ckp - sn * ckq;
    C[k][Q] = sn * ckp + c * ckq;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {  // rows P, Q of J^T (C J)
    const double cpk = C[P][k], cqk = C[Q][k];
    C[P][k] = c * cpk - sn * cqk;
    C[Q][k] = sn * cpk + c * cqk;
  }
  C[P][Q] = C[Q][P] = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double vkp = V[k][P], vkq = V[k][Q];
    V[k][P] = c * vkp - sn * vkq;
    V[k][Q] = sn * vkp + c * vkq;
  }
}

// Adaptive-rho data of every segment (FP64).  With H the rho-weighted part of
// the local matrix and D its Jacobi scaling, D H D = L L^T and M = L^-1 D
// (lower triangular).  The cost block 2 T^-7 Qh lives on coefficients 4..7
// only, so  M K(rho) M^T = rho I + blockdiag(0, C4),  C4 = M44 Q4 M44^T, and
// with C4 = V diag(lambda) V^T:
//   K(rho)^-1 = M^T blockdiag(I / rho, V diag(1 / (lambda + rho)) V^T) M
//             = A0 / rho + Y diag(1 / (lambda + rho)) Y^T,
//   A0 = M_top^T M_top (rows 0..3 of M, columns 0..3 only),  Y = M_bot^T V.
template <bool SAMPLES>
__global__ void __launch_bounds__(128) keig_kernel(const DevProblem p, float *__restrict__ E32,
                                                   double *__restrict__ E64, int *__restrict__ err) {
  const int S = p.S;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < S; g += gridDim.x * blockDim.x) {
    bool first, last;
    double s[NC];
    if (!segment_setup(p, g, first, last, s)) {
      atomicOr(err, 1);
      continue;
    }
    double A[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) A[q] = 0.0;
    add_rho_terms<SAMPLES>(p, s, first, last, 1.0, A);
    double d[NC];
    if (!equil_chol_inv(A, d)) {
      atomicOr(err, 2);
      continue;
    }
    // M = L^-1 D in place (lower triangular)
#pragma unroll
    for (int r = 0; r < NC; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) A[lidx(r, c)] *= d[c];
    // C4 = M44 Q4 M44^T with Q4 = 2 s_7 Qh[4..7][4..7]
    double W[4][4];  // W = M44 Q4
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double a = 0.0;
#pragma unroll
        for (int k = 0; k <= i; ++k) a += A[lidx(PO + i, PO + k)] * (2.0 * s[7] * qhat(PO + k, PO + j));
        W[i][j] = a;
      }
    double Cm[4][4], V[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double a = 0.0;
#pragma unroll
        for (int k = 0; k <= j; ++k) a += W[i][k] * A[lidx(PO + j, PO + k)];
        Cm[i][j] = a;
        V[i][j] = (i == j) ? 1.0 : 0.0;
      }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < i; ++j) Cm[i][j] = Cm[j][i] = 0.5 * (Cm[i][j] + Cm[j][i]);
    // cyclic Jacobi sweeps (quadratic convergence; a 4x4 needs a handful)
    for (int sweep = 0; sweep < 16; ++sweep) {
      double off = 0.0, dia = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        dia += Cm[i][i] * Cm[i][i];
#pragma unroll
        for (int j = i + 1; j < 4; ++j) off += Cm[i][j] * Cm[i][j];
      }
      if (!(off > 1e-34 * dia)) break;
      jacobi_rot<0, 1>(Cm, V); jacobi_rot<0, 2>(Cm, V); jacobi_rot<0, 3>(Cm, V);
      jacobi_rot<1, 2>(Cm, V); jacobi_rot<1, 3>(Cm, V); jacobi_rot<2, 3>(Cm, V);
    }
    double out[NE];
    // A0 = M_top^T M_top on the top-left 4x4 block (packed lower)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        double a = 0.0;
#pragma unroll
        for (int r = i; r < 4; ++r) a += A[lidx(r, i)] * A[lidx(r, j)];
        out[NE_A0 + lidx(i, j)] = a;
      }
    // Y = M_bot^T V
#pragma unroll
    for (int i = 0; i < NC; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double a = 0.0;
#pragma unroll
        for (int r = (i > PO ? i : PO); r < NC; ++r) a += A[lidx(r, i)] * V[r - PO][k];
        out[NE_Y + i * 4 + k] = a;
      }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[NE_L + k] = Cm[k][k] > 0.0 ? Cm[k][k] : 0.0;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      if (E64) E64[size_t(q) * S + g] = out[q];
      if (E32) E32[size_t(q) * S + g] = float(out[q]);
    }
  }
}

// Polytope family (FP64, once per solve).  N3 = sum_f n_f n_f^T = U diag(nu) U^T
// by cyclic Jacobi; in the rotated axes the polytope rows add rho nu_b B_pos to
// the isotropic 8x8 local matrix of axis b (B_pos = sum_j b_j b_j^T, position
// samples b_j[k] = tau_j^k), so each rotated axis gets its own 8x8 inverse.
// The normals and offsets are also stored in the iteration type.
template <bool SAMPLES, class R>
__global__ void __launch_bounds__(128) kinv_poly_kernel(const DevProblem p, double rho, R *__restrict__ PG,
                                                        R *__restrict__ PU, R *__restrict__ PN, R *__restrict__ PH,
                                                        int *__restrict__ err) {
  const int S = p.S, F = p.F_poly;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < S; g += gridDim.x * blockDim.x) {
    bool first, last;
    double s[NC];
    if (!segment_setup(p, g, first, last, s)) {
      atomicOr(err, 1);
      continue;
    }
    double C3[3][3], U[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { C3[a][b] = 0.0; U[a][b] = (a == b) ? 1.0 : 0.0; }
    for (int f = 0; f < F; ++f) {
      const double *nf = p.poly_n + ((size_t)g * F + f) * 3;
      const double n0 = nf[0], n1 = nf[1], n2 = nf[2], hf = p.poly_h[(size_t)g * F + f];
      if (!(n0 == n0 && n1 == n1 && n2 == n2 && hf == hf)) atomicOr(err, 1);
      C3[0][0] += n0 * n0; C3[0][1] += n0 * n1; C3[0][2] += n0 * n2;
      C3[1][1] += n1 * n1; C3[1][2] += n1 * n2; C3[2][2] += n2 * n2;
      PN[(size_t)(f * 3 + 0) * S + g] = R(n0);
      PN[(size_t)(f * 3 + 1) * S + g] = R(n1);
      PN[(size_t)(f * 3 + 2) * S + g] = R(n2);
      PH[(size_t)f * S + g] = R(hf);
    }
    C3[1][0] = C3[0][1]; C3[2][0] = C3[0][2]; C3[2][1] = C3[1][2];
    for (int sweep = 0; sweep < 16; ++sweep) {
      double off = 0.0, dia = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dia += C3[i][i] * C3[i][i];
#pragma unroll
        for (int j = i + 1; j < 3; ++j) off += C3[i][j] * C3[i][j];
      }
      if (!(off > 1e-34 * dia)) break;
      jacobi_rot<0, 1>(C3, U); jacobi_rot<0, 2>(C3, U); jacobi_rot<1, 2>(C3, U);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) PU[(size_t)(a * 3 + b) * S + g] = R(U[a][b]);
    for (int b = 0; b < 3; ++b) {
      const double nu = C3[b][b] > 0.0 ? C3[b][b] : 0.0;
      double A[NG];
      const double t7x2 = 2.0 * s[7];
#pragma unroll
      for (int r = 0; r < NC; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) A[lidx(r, c)] = (r >= PO && c >= PO) ? t7x2 * qhat(r, c) : 0.0;
      add_rho_terms<SAMPLES>(p, s, first, last, rho, A);
      if (nu > 0.0) add_sample_rows(A, p.M_poly, 0, rho * nu);
      double d[NC];
      if (!equil_chol_inv(A, d)) {
        atomicOr(err, 2);
        break;
      }
      if (sizeof(R) == 8) store_inverse(A, d, S, g, b * NG, nullptr, (double *)PG);
      else store_inverse(A, d, S, g, b * NG, (float *)PG, nullptr);
    }
  }
}

int launch_kinv_poly(const DevProblem &p, double rho, bool fp64, const PolyData &out, int *err_flag, void *stream) {
  if (p.S == 0) return 0;
  const int threads = 128;
  int blocks = (p.S + threads - 1) / threads;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  cudaStream_t st = (cudaStream_t)stream;
  const bool samples = p.inner == 0 && (p.M_box > 0 || p.M_ball > 0 || p.M_vn > 0);
#define TOP_KP(SMP, R)                                                                                   \
  kinv_poly_kernel<SMP, R><<<blocks, threads, 0, st>>>(p, rho, (R *)out.G, (R *)out.U, (R *)out.N, (R *)out.H, \
                                                       err_flag)
  if (fp64) {
    if (samples) TOP_KP(true, double); else TOP_KP(false, double);
  } else {
    if (samples) TOP_KP(true, float); else TOP_KP(false, float);
  }
#undef TOP_KP
  return (int)cudaGetLastError();
}

int launch_keig(const DevProblem &p, void *E32, void *E64, int *err_flag, void *stream) {
  if (p.S == 0) return 0;
  const int threads = 128;
  int blocks = (p.S + threads - 1) / threads;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  const bool samples = p.inner == 0 && (p.M_box > 0 || p.M_ball > 0 || p.M_vn > 0);
  if (samples)
    keig_kernel<true><<<blocks, threads, 0, (cudaStream_t)stream>>>(p, (float *)E32, (double *)E64, err_flag);
  else
    keig_kernel<false><<<blocks, threads, 0, (cudaStream_t)stream>>>(p, (float *)E32, (double *)E64, err_flag);
  return (int)cudaGetLastError();
}

__global__ void fill_kernel(double *x, int n, double v) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) x[q] = v;
}

int launch_fill(double *x, int n, double v, void *stream) {
  if (n <= 0) return 0;
  int blocks = (n + 255) / 256;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  fill_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, n, v);
  return (int)cudaGetLastError();
}

__global__ void kinv_copy_kernel(const int *__restrict__ copy, int S, float *__restrict__ G32,
                                 double *__restrict__ G64) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < S; g += gridDim.x * blockDim.x) {
    const int src = copy[g];
    if (src < 0) continue;
#pragma unroll 4
    for (int q = 0; q < NG; ++q) {
      if (G64) G64[(size_t)q * S + g] = G64[(size_t)q * S + src];
      if (G32) G32[(size_t)q * S + g] = G32[(size_t)q * S + src];
    }
  }
}

int launch_kinv(const DevProblem &p, double rho, void *G32, void *G64, int *err_flag, void *stream, int *copy) {
  if (p.S == 0) return 0;
  const int threads = 128;
  int blocks = (p.S + threads - 1) / threads;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  const bool samples = p.inner == 0 && (p.M_box > 0 || p.M_ball > 0 || p.M_vn > 0);
  cudaStream_t st = (cudaStream_t)stream;
  int *list = copy ? copy + p.S : nullptr;
  if (copy) {
    cudaError_t e = cudaMemsetAsync(list, 0, sizeof(int), st);
    if (e != cudaSuccess) return (int)e;
    int mb = (p.S + 255) / 256;
    if (mb > sm_count() * 16) mb = sm_count() * 16;
    kinv_mark_kernel<<<mb, 256, 0, st>>>(p, copy, list);
  }
  if (samples)
    kinv_kernel<true><<<blocks, threads, 0, st>>>(p, rho, (float *)G32, (double *)G64, err_flag, list);
  else
    kinv_kernel<false><<<blocks, threads, 0, st>>>(p, rho, (float *)G32, (double *)G64, err_flag, list);
  if (copy) {
    int cb = (p.S + 255) / 256;
    if (cb > sm_count() * 16) cb = sm_count() * 16;
    kinv_copy_kernel<<<cb, 256, 0, st>>>(copy, p.S, (float *)G32, (double *)G64);
  }
  return (int)cudaGetLastError();
}

}  // namespace top
