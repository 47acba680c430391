// top_step.cuh -- the per-segment local step of one CADMM iteration, shared
// by the resident and the streaming kernels.
//
// Given the scaled consensus targets of both ends (wS_r = s_r E(z - u) at the
// start junction, wE_r likewise at the end), it forms the right-hand side of
// Eq. 18a in normalised coordinates, including the box slack terms (Eq. 18d-e,
// compressed state y) and the ball / velocity-norm projection terms (Eq.
// 18f-g, compressed state q), solves with the precomputed inverse G, then
// advances the constraint state with the new coefficients.  The constraint
// state lives wherever the caller keeps it (shared or global memory), one
// element every `stride` entries.
#pragma once

#include "top_internal.h"
#include "top_math.cuh"

namespace top {

template <class R>
__device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <class R>
__device__ __forceinline__ R rmax0(R x) { return x > R(0) ? x : R(0); }

// per-segment constants held in registers for the whole run
template <class R>
struct SegConst {
  R G[NG];      // (D K D)^{-1}, packed
  R s[NC];      // T^{-r}
  R vbox, vnorm, brad;
  R bo[3];
};

// sample tables: tab[j*8 + k] = k tau_j^{k-1} (velocity rows) or tau_j^k (position rows)
template <class R>
__device__ __forceinline__ void fill_sample_table(R *tab, int M, int order, int tid, int nthreads) {
  for (int q = tid; q < 8 * M; q += nthreads) {
    const int j = q / 8 + 1, k = q % 8;
    const double tau = double(j) / double(M);
    double t = 1.0;
    const int e = order == 0 ? k : k - 1;
    for (int x = 0; x < e; ++x) t *= tau;
    tab[q] = R(order == 0 ? t : (k == 0 ? 0.0 : double(k) * t));
  }
}

template <class R, int F>
__device__ __forceinline__ void local_step(const SegConst<R> &sc, const R (&wS)[AX][ND], const R (&wE)[AX][ND],
                                           R rho, bool first_iter, R *ybox, R *qball, R *qvn, int stride,
                                           const R *tabB, const R *tabQ, const R *tabV, int Mb, int Mq, int Mv,
                                           R (&ch)[AX][NC]) {
  constexpr bool BOX = (F & FAM_BOX) != 0;
  constexpr bool BALL = (F & FAM_BALL) != 0;
  constexpr bool VN = (F & FAM_VN) != 0;
  R rhs[AX][NC];
#pragma unroll
  for (int a = 0; a < AX; ++a) {
#pragma unroll
    for (int q = 0; q < NC; ++q) rhs[a][q] = R(0);
    consensus_rhs(wS[a], wE[a], rho, rhs[a]);
  }
  if (BOX) {
    for (int j = 0; j < Mb; ++j) {
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        const R yp = ybox[((j * 3 + a) * 2 + 0) * stride];
        const R ym = ybox[((j * 3 + a) * 2 + 1) * stride];
        const R coef = rho * sc.s[1] * (rabs(ym) - rabs(yp));
#pragma unroll
        for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tabB[j * 8 + q];
      }
    }
  }
  if (BALL && !first_iter) {
    for (int j = 0; j < Mq; ++j) {
      R qv[3], ph[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) qv[a] = qball[(j * 3 + a) * stride];
      project_ball(qv, sc.bo, sc.brad, ph);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        const R coef = rho * (R(2) * ph[a] - qv[a]);
#pragma unroll
        for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tabQ[j * 8 + q];
      }
    }
  }
  if (VN && !first_iter) {
    const R zero3[3] = {R(0), R(0), R(0)};
    for (int j = 0; j < Mv; ++j) {
      R qv[3], ph[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) qv[a] = qvn[(j * 3 + a) * stride];
      project_ball(qv, zero3, sc.vnorm, ph);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        const R coef = rho * sc.s[1] * (R(2) * ph[a] - qv[a]);
#pragma unroll
        for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tabV[j * 8 + q];
      }
    }
  }
#pragma unroll
  for (int a = 0; a < AX; ++a) apply_g(sc.G, rhs[a], ch[a]);
  // projections and their duals with the new coefficients (Eq. 18d-g)
  if (BOX) {
    for (int j = 0; j < Mb; ++j) {
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        R v = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) v += tabB[j * 8 + q] * ch[a][q];
        v *= sc.s[1];
        R *yp = &ybox[((j * 3 + a) * 2 + 0) * stride];
        R *ym = &ybox[((j * 3 + a) * 2 + 1) * stride];
        const R ypn = v - sc.vbox + rmax0(*yp);
        const R ymn = -v - sc.vbox + rmax0(*ym);
        *yp = ypn;
        *ym = ymn;
      }
    }
  }
  if (BALL) {
    for (int j = 0; j < Mq; ++j) {
      R qv[3], ph[3], pos[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        qv[a] = qball[(j * 3 + a) * stride];
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) acc += tabQ[j * 8 + q] * ch[a][q];
        pos[a] = acc;
      }
      project_ball(qv, sc.bo, sc.brad, ph);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R wprev = first_iter ? R(0) : qv[a] - ph[a];
        qball[(j * 3 + a) * stride] = pos[a] + wprev;
      }
    }
  }
  if (VN) {
    const R zero3[3] = {R(0), R(0), R(0)};
    for (int j = 0; j < Mv; ++j) {
      R qv[3], ph[3], vel[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        qv[a] = qvn[(j * 3 + a) * stride];
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) acc += tabV[j * 8 + q] * ch[a][q];
        vel[a] = acc * sc.s[1];
      }
      project_ball(qv, zero3, sc.vnorm, ph);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R wprev = first_iter ? R(0) : qv[a] - ph[a];
        qvn[(j * 3 + a) * stride] = vel[a] + wprev;
      }
    }
  }
}

// rho M^T (s .* dz) for one axis, mapped back to the paper's coefficients
// (multiplied by T^k), squared and summed: one segment's share of ||r_d||^2 (Eq. 20)
template <class R>
__device__ __forceinline__ double dual_residual_sq(const R (&dS)[ND], const R (&dE)[ND], R rho, const R (&Tk)[NC]) {
  R x[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) x[q] = R(0);
  consensus_rhs(dS, dE, rho, x);
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const double v = double(x[q]) * double(Tk[q]);
    acc += v * v;
  }
  return acc;
}

// per-segment cost c^T Q(T) c = T^{-7} ch^T Qh ch, in FP64
template <class R>
__device__ __forceinline__ double segment_cost(const R (&ch)[AX][NC], double t7) {
  double J = 0.0;
#pragma unroll
  for (int a = 0; a < AX; ++a)
    for (int k1 = PO; k1 < NC; ++k1) {
      double acc = 0.0;
      for (int k2 = PO; k2 < NC; ++k2) acc += qhat(k1, k2) * double(ch[a][k2]);
      J += double(ch[a][k1]) * acc;
    }
  return J * t7;
}

__device__ __forceinline__ bool finite_d(double x) { return x == x && x - x == 0.0; }

}  // namespace top
