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

// ---- the same two maps through a Taylor shift (resident and cluster kernels) ----
// With F(k,r) = r! C(k,r) the end derivatives are eE_r = r! s_r b_r, where
// b_r = sum_{k>=r} C(k,r) ch_k are the coefficients of the same polynomial in
// powers of (t/T - 1); synthetic division (a Taylor shift by one) forms b_0..b_7
// with 28 additions.  The end-side part of the consensus right-hand side,
// sum_{r<=min(k,6)} F(k,r) s_r w_r, is the transposed shift applied to
// v_r = r! s_r w_r: the same 28 additions in reverse order.  Axes 0 and 1 run
// as one packed pair (two FP32 lanes per instruction), axis 2 alone.
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 mk2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mk2(double x, double y) { return make_double2(x, y); }
template <class R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// a_r <- sum_{k>=r} C(k,r) a_k
template <class V>
__device__ __forceinline__ void taylor_shift(V (&a)[NC]) {
#pragma unroll
  for (int i = 0; i < NC - 1; ++i)
#pragma unroll
    for (int j = NC - 2; j >= i; --j) a[j] = vadd(a[j], a[j + 1]);
}

// v_k <- sum_{r<=k} C(k,r) v_r  (the transpose of taylor_shift)
template <class V>
__device__ __forceinline__ void taylor_shift_t(V (&v)[NC]) {
#pragma unroll
  for (int i = NC - 2; i >= 0; --i)
#pragma unroll
    for (int j = i; j <= NC - 2; ++j) v[j + 1] = vadd(v[j + 1], v[j]);
}

// eS_r = fs_r ch_r and eE_r = fs_r b_r for the three axes (fs_r = r! s_r)
template <class R>
__device__ __forceinline__ void end_derivs_shift(const R (&ch)[AX][NC], const R (&fs)[ND], R (&eS)[AX][ND],
                                                 R (&eE)[AX][ND]) {
  using V = typename Vec2<R>::T;
  V p[NC];
  R q[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    p[k] = mk2(ch[0][k], ch[1][k]);
    q[k] = ch[2][k];
  }
  taylor_shift(p);
  taylor_shift(q);
#pragma unroll
  for (int r = 0; r < ND; ++r) {
    if (r == 0) {  // fs_0 = 1
#pragma unroll
      for (int a = 0; a < AX; ++a) eS[a][0] = ch[a][0];
      eE[0][0] = p[0].x;
      eE[1][0] = p[0].y;
      eE[2][0] = q[0];
      continue;
    }
    const V f2 = mk2(fs[r], fs[r]);
    const V s01 = vmul(f2, mk2(ch[0][r], ch[1][r]));
    const V e01 = vmul(f2, p[r]);
    eS[0][r] = s01.x;
    eS[1][r] = s01.y;
    eS[2][r] = fs[r] * ch[2][r];
    eE[0][r] = e01.x;
    eE[1][r] = e01.y;
    eE[2][r] = fs[r] * q[r];
  }
}

// ch = G rhs for the three axes; axes 0 and 1 as one packed pair, each entry of G
// applied to both lanes (the same sums in the same order as apply_g)
template <class R>
__device__ __forceinline__ void apply_g3(const R (&G)[NG], const R (&rhs)[AX][NC], R (&ch)[AX][NC]) {
  using V = typename Vec2<R>::T;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const R g0 = G[gidx(k, 0)];
    V acc = vmul(mk2(g0, g0), mk2(rhs[0][0], rhs[1][0]));
    R a2 = g0 * rhs[2][0];
#pragma unroll
    for (int l = 1; l < NC; ++l) {
      const R g = G[gidx(k, l)];
      acc = vfma(mk2(g, g), mk2(rhs[0][l], rhs[1][l]), acc);
      a2 += g * rhs[2][l];
    }
    ch[0][k] = acc.x;
    ch[1][k] = acc.y;
    ch[2][k] = a2;
  }
}

// rhs_k = rho (wSf_k + sum_{r<=min(k,6)} C(k,r) vE_r) for the three axes, with
// wSf_r = r! s_r (start-side target) and vE_r = r! s_r (end-side target)
template <class R>
__device__ __forceinline__ void consensus_rhs_shift(const R (&wSf)[AX][ND], const R (&vE)[AX][ND], R rho,
                                                    R (&rhs)[AX][NC]) {
  using V = typename Vec2<R>::T;
  V t[NC];
  R u[NC];
#pragma unroll
  for (int r = 0; r < ND; ++r) {
    t[r] = mk2(vE[0][r], vE[1][r]);
    u[r] = vE[2][r];
  }
  t[NC - 1] = mk2(R(0), R(0));
  u[NC - 1] = R(0);
  taylor_shift_t(t);
  taylor_shift_t(u);
  const V rr = mk2(rho, rho);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    if (k < ND) {
      t[k] = vadd(t[k], mk2(wSf[0][k], wSf[1][k]));
      u[k] += wSf[2][k];
    }
    t[k] = vmul(rr, t[k]);
    rhs[0][k] = t[k].x;
    rhs[1][k] = t[k].y;
    rhs[2][k] = rho * u[k];
  }
}

// The junction update of a free row (Eq. 18b-c in the targets p = z + u_R,
// m = z - u_L): u = (p - m)/2, p' = eE + u, m' = eS_next - u; two rows at once
// (axes 0 and 1), each result rounded exactly as the scalar form rounds it.
__device__ __forceinline__ void junction_pair(float ee0, float ee1, float en0, float en1, float &p0, float &p1,
                                              float &m0, float &m1) {
  const float2 u = __ffma2_rn(make_float2(-0.5f, -0.5f), make_float2(m0, m1),
                              __fmul2_rn(make_float2(0.5f, 0.5f), make_float2(p0, p1)));
  const float2 pn = __fadd2_rn(make_float2(ee0, ee1), u);
  const float2 mn = __ffma2_rn(make_float2(-1.0f, -1.0f), u, make_float2(en0, en1));
  p0 = pn.x; p1 = pn.y; m0 = mn.x; m1 = mn.y;
}
__device__ __forceinline__ void junction_pair(double ee0, double ee1, double en0, double en1, double &p0, double &p1,
                                              double &m0, double &m1) {
  const double u0 = 0.5 * (p0 - m0), u1 = 0.5 * (p1 - m1);
  p0 = ee0 + u0; p1 = ee1 + u1;
  m0 = en0 - u0; m1 = en1 - u1;
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
