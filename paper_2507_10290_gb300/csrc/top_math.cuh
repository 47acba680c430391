// top_math.cuh -- per-segment algebra of the CADMM iteration in the
// time-normalised basis used by every kernel of the library.
//
// The paper's segment polynomial is sigma_i(t) = c_i^T beta(t), beta(t) =
// (1, t, ..., t^7) (Sec. III-D.1).  The kernels work with the normalised
// coefficients  ch_k = c_k T^k, i.e. sigma(t) = sum_k ch_k (t/T)^k, so that
// every basis constant becomes an integer and only the powers s_r = T^{-r}
// carry the duration:
//   derivative r at t = 0 :  r! s_r ch_r
//   derivative r at t = T :  s_r sum_{k>=r} F(k,r) ch_k,     F(k,r) = k!/(k-r)!
//   velocity at t = tau T :  s_1 sum_k k tau^{k-1} ch_k
//   position at t = tau T :  sum_k tau^k ch_k
// The local matrix of Eq. 18a in these coordinates is D K D with
// D = diag(s_k); its inverse G = (D K D)^{-1} is what the FP64 precompute
// kernel stores, and c = D G D r becomes ch = G (D r).
#pragma once

#include <cstdint>

namespace top {

constexpr int AX = 3;    // flat-output axes
constexpr int PO = 4;    // control order p (minimum snap)
constexpr int NC = 8;    // coefficients per axis (degree 2p-1)
constexpr int ND = 7;    // consensus derivative orders 0..2p-2
constexpr int NJ = AX * ND;  // consensus values per junction (21)
constexpr int NG = NC * (NC + 1) / 2;  // packed symmetric 8x8 (36)

__host__ __device__ constexpr int falling(int k, int r) {
  int f = 1;
  for (int i = 0; i < r; ++i) f *= (k - i);
  return f;
}

__host__ __device__ constexpr int fact(int r) { return falling(r, r); }

// index of (k, l), k <= l, in the packed upper triangle
__host__ __device__ constexpr int gidx(int k, int l) {
  return k <= l ? k * NC - (k * (k - 1)) / 2 + (l - k) : l * NC - (l * (l - 1)) / 2 + (k - l);
}

// (s_0 .. s_7) = T^{-r}
template <class R>
__device__ __forceinline__ void inv_powers(R T, R (&s)[NC]) {
  R it = R(1) / T;
  s[0] = R(1);
#pragma unroll
  for (int r = 1; r < NC; ++r) s[r] = s[r - 1] * it;
}

// rhs_k += rho * ( k! wS_k + sum_{r<=min(k,6)} F(k,r) wE_r ), where wS, wE
// are already multiplied by s_r (the consensus part of D r, Eq. 18a).
template <class R>
__device__ __forceinline__ void consensus_rhs(const R (&wS)[ND], const R (&wE)[ND], R rho,
                                              R (&rhs)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    R acc = (k < ND) ? R(fact(k)) * wS[k] : R(0);
#pragma unroll
    for (int r = 0; r < ND; ++r)
      if (r <= k) acc += R(falling(k, r)) * wE[r];
    rhs[k] += rho * acc;
  }
}

// as consensus_rhs, with the start-side targets already multiplied by k!
template <class R>
__device__ __forceinline__ void consensus_rhs_f(const R (&wSf)[ND], const R (&wE)[ND], R rho, R (&rhs)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    R acc = (k < ND) ? wSf[k] : R(0);
#pragma unroll
    for (int r = 0; r < ND; ++r)
      if (r <= k) acc += R(falling(k, r)) * wE[r];
    rhs[k] += rho * acc;
  }
}

// derivatives 0..6 at both ends of one axis: eS_r = r! s_r ch_r,
// eE_r = s_r sum_{k>=r} F(k,r) ch_k  (the rows of M(T) c, Sec. III-D.1)
template <class R>
__device__ __forceinline__ void end_derivs(const R (&ch)[NC], const R (&s)[NC], R (&eS)[ND],
                                           R (&eE)[ND]) {
#pragma unroll
  for (int r = 0; r < ND; ++r) {
    eS[r] = R(fact(r)) * s[r] * ch[r];
    R acc = R(0);
#pragma unroll
    for (int k = r; k < NC; ++k) acc += R(falling(k, r)) * ch[k];
    eE[r] = s[r] * acc;
  }
}

// as end_derivs, with fs_r = r! s_r precomputed
template <class R>
__device__ __forceinline__ void end_derivs_f(const R (&ch)[NC], const R (&s)[NC], const R (&fs)[ND], R (&eS)[ND],
                                             R (&eE)[ND]) {
#pragma unroll
  for (int r = 0; r < ND; ++r) {
    eS[r] = fs[r] * ch[r];
    R acc = R(0);
#pragma unroll
    for (int k = r; k < NC; ++k) acc += R(falling(k, r)) * ch[k];
    eE[r] = s[r] * acc;
  }
}

// ch = G rhs, G packed symmetric 8x8
template <class R>
__device__ __forceinline__ void apply_g(const R (&G)[NG], const R (&rhs)[NC], R (&ch)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    R acc = R(0);
#pragma unroll
    for (int l = 0; l < NC; ++l) acc += G[gidx(k, l)] * rhs[l];
    ch[k] = acc;
  }
}

// normalised cost block  Qh_kl = F(k,4) F(l,4) / (k + l - 7)  for k, l >= 4, so that
// c^T Q(T) c = T^{-7} ch^T Qh ch  (Q of Sec. III-D.1)
__host__ __device__ constexpr double qhat(int k, int l) {
  return (k < PO || l < PO) ? 0.0
                            : double(falling(k, PO)) * double(falling(l, PO)) / double(k + l - 2 * PO + 1);
}

// projection onto the ball ||phi - o|| <= rad: the closed form of Eq. 14 with
// the centre shifted to o (o = 0 for the velocity-norm family)
__device__ __forceinline__ void project_ball(const float (&q)[3], const float (&o)[3], float rad,
                                             float (&phi)[3]) {
  float d0 = q[0] - o[0], d1 = q[1] - o[1], d2 = q[2] - o[2];
  float n2 = d0 * d0 + d1 * d1 + d2 * d2;
  float f = (n2 > rad * rad) ? rad * rsqrtf(n2) : 1.0f;
  phi[0] = o[0] + f * d0; phi[1] = o[1] + f * d1; phi[2] = o[2] + f * d2;
}

__device__ __forceinline__ void project_ball(const double (&q)[3], const double (&o)[3], double rad,
                                             double (&phi)[3]) {
  double d0 = q[0] - o[0], d1 = q[1] - o[1], d2 = q[2] - o[2];
  double n2 = d0 * d0 + d1 * d1 + d2 * d2;
  double f = (n2 > rad * rad) ? rad * rsqrt(n2) : 1.0;
  phi[0] = o[0] + f * d0; phi[1] = o[1] + f * d1; phi[2] = o[2] + f * d2;
}

}  // namespace top
