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

// Coefficient output of a warp's 32 segments (one per lane) through a
// shared-memory tile: each lane has written its 24 values to row `lane` of
// `tile` (stride kOutRow doubles); the warp then stores them with consecutive
// lanes on consecutive words, so the segments of one trajectory (consecutive
// in g) go out as contiguous runs instead of 24 stores strided by a segment's
// 192 bytes.  That matters most when `out` is page-locked host memory written
// over the chip-to-host link.  Every lane of the warp calls it.
constexpr int kOutRow = 25;
__device__ __forceinline__ void store_rows_warp(double *out, const double *tile, int g, bool valid) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
#pragma unroll 4
  for (int t = 0; t < 24; ++t) {
    const int e = t * 32 + lane, s = e / 24, w = e - s * 24;
    const int gs = __shfl_sync(0xffffffffu, g, s);
    const int vs = __shfl_sync(0xffffffffu, valid ? 1 : 0, s);
    if (vs) out[(size_t)gs * 24 + w] = tile[s * kOutRow + w];
  }
  __syncwarp();
}

// One row of a sample table (8 values; rows start on 16-byte boundaries).
template <class R>
__device__ __forceinline__ void tab_row(const R *t, R (&v)[NC]) {
  if constexpr (sizeof(R) == 4) {
    const float4 a = reinterpret_cast<const float4 *>(t)[0], b = reinterpret_cast<const float4 *>(t)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int q = 0; q < NC / 2; ++q) {
      const double2 x = reinterpret_cast<const double2 *>(t)[q];
      v[2 * q] = x.x;
      v[2 * q + 1] = x.y;
    }
  }
}

// The right-hand side of Eq. 18a for the consensus rows and the box / ball /
// velocity-norm families (the first half of the local step).
// FS: the targets wS and wE both carry the factor r! (wS = r! s_r p, wE = r! s_r m)
// and the consensus rows go through the Taylor shift (consensus_rhs_shift)
// j0, js: the sample rows j = j0, j0 + js, ... (a segment's rows split over js
// lanes); cons: include the consensus rows (one lane of the js)
template <class R, int F, bool FS = false>
__device__ __forceinline__ void family_rhs(const SegConst<R> &sc, const R (&wS)[AX][ND], const R (&wE)[AX][ND],
                                           R rho, bool first_iter, const R *ybox, const R *qball, const R *qvn,
                                           int stride, const R *tabB, const R *tabQ, const R *tabV, int Mb, int Mq,
                                           int Mv, R (&rhs)[AX][NC], int j0 = 0, int js = 1, bool cons = true) {
  constexpr bool BOX = (F & FAM_BOX) != 0;
  constexpr bool BALL = (F & FAM_BALL) != 0;
  constexpr bool VN = (F & FAM_VN) != 0;
  if (!cons) {
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) rhs[a][q] = R(0);
  } else if (FS) {
    consensus_rhs_shift(wS, wE, rho, rhs);
  } else {
#pragma unroll
    for (int a = 0; a < AX; ++a) {
#pragma unroll
      for (int q = 0; q < NC; ++q) rhs[a][q] = R(0);
      consensus_rhs(wS[a], wE[a], rho, rhs[a]);
    }
  }
  if (BOX) {
    for (int j = j0; j < Mb; j += js) {
      R tb[NC];
      tab_row(tabB + j * 8, tb);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        const R yp = ybox[((j * 3 + a) * 2 + 0) * stride];
        const R ym = ybox[((j * 3 + a) * 2 + 1) * stride];
        const R coef = rho * sc.s[1] * (rabs(ym) - rabs(yp));
#pragma unroll
        for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tb[q];
      }
    }
  }
  if (BALL && !first_iter) {
    for (int j = j0; j < Mq; j += js) {
      R qv[3], ph[3], tq[NC];
      tab_row(tabQ + j * 8, tq);
#pragma unroll
      for (int a = 0; a < 3; ++a) qv[a] = qball[(j * 3 + a) * stride];
      project_ball(qv, sc.bo, sc.brad, ph);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        const R coef = rho * (R(2) * ph[a] - qv[a]);
#pragma unroll
        for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tq[q];
      }
    }
  }
  if (VN && !first_iter) {
    const R zero3[3] = {R(0), R(0), R(0)};
    for (int j = j0; j < Mv; j += js) {
      R qv[3], ph[3], tv[NC];
      tab_row(tabV + j * 8, tv);
#pragma unroll
      for (int a = 0; a < 3; ++a) qv[a] = qvn[(j * 3 + a) * stride];
      project_ball(qv, zero3, sc.vnorm, ph);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        const R coef = rho * sc.s[1] * (R(2) * ph[a] - qv[a]);
#pragma unroll
        for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tv[q];
      }
    }
  }
}

// Projections and their duals with the new coefficients (Eq. 18d-g) for the
// box / ball / velocity-norm families (the second half of the local step).
// (j0, js as in family_rhs: each lane updates the rows of its own samples)
template <class R, int F>
__device__ __forceinline__ void family_update(const SegConst<R> &sc, bool first_iter, R *ybox, R *qball, R *qvn,
                                              int stride, const R *tabB, const R *tabQ, const R *tabV, int Mb,
                                              int Mq, int Mv, const R (&ch)[AX][NC], int j0 = 0, int js = 1) {
  constexpr bool BOX = (F & FAM_BOX) != 0;
  constexpr bool BALL = (F & FAM_BALL) != 0;
  constexpr bool VN = (F & FAM_VN) != 0;
  if (BOX) {
    for (int j = j0; j < Mb; j += js) {
      R tb[NC];
      tab_row(tabB + j * 8, tb);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        R v = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) v += tb[q] * ch[a][q];
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
    for (int j = j0; j < Mq; j += js) {
      R qv[3], ph[3], pos[3], tq[NC];
      tab_row(tabQ + j * 8, tq);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        qv[a] = qball[(j * 3 + a) * stride];
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) acc += tq[q] * ch[a][q];
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
    for (int j = j0; j < Mv; j += js) {
      R qv[3], ph[3], vel[3], tv[NC];
      tab_row(tabV + j * 8, tv);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        qv[a] = qvn[(j * 3 + a) * stride];
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) acc += tv[q] * ch[a][q];
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

// The closed-form local step of Eq. 18a with the box / ball / velocity-norm
// families (Eq. 18d-g): right-hand side, ch = G rhs per axis, projections.
template <class R, int F, bool FS = false>
__device__ __forceinline__ void local_step(const SegConst<R> &sc, const R (&wS)[AX][ND], const R (&wE)[AX][ND],
                                           R rho, bool first_iter, R *ybox, R *qball, R *qvn, int stride,
                                           const R *tabB, const R *tabQ, const R *tabV, int Mb, int Mq, int Mv,
                                           R (&ch)[AX][NC]) {
  R rhs[AX][NC];
  family_rhs<R, F, FS>(sc, wS, wE, rho, first_iter, ybox, qball, qvn, stride, tabB, tabQ, tabV, Mb, Mq, Mv, rhs);
  if (FS) {
    apply_g3(sc.G, rhs, ch);
  } else {
#pragma unroll
    for (int a = 0; a < AX; ++a) apply_g(sc.G, rhs[a], ch[a]);
  }
  family_update<R, F>(sc, first_iter, ybox, qball, qvn, stride, tabB, tabQ, tabV, Mb, Mq, Mv, ch);
}

// ---- polytope family (FAM_POLY; streaming form) ----
// Data of segment g in the layout of PolyData: PN[(f * 3 + a) * S + g],
// PH[f * S + g], PU[(a * 3 + b) * S + g], PG[(b * 36 + q) * S + g]; the
// compressed slack / dual y of row (j, f) at ypoly[(j * F + f) * stride].

// rhs_a += rho sum_j tau_j^k sum_f n_f[a] (h_f - |y_jf|)   (A°^T (b - s - v), Eq. 18a)
template <class R>
__device__ __forceinline__ void poly_rhs(const R *PN, const R *PH, size_t S, size_t g, int F, int M, R rho,
                                         const R *ypoly, int stride, const R *tabP, R (&rhs)[AX][NC], int j0 = 0,
                                         int js = 1) {
  for (int j = j0; j < M; j += js) {
    R w[3] = {R(0), R(0), R(0)};
    for (int f = 0; f < F; ++f) {
      const R c = PH[(size_t)f * S + g] - rabs(ypoly[(j * F + f) * stride]);
#pragma unroll
      for (int a = 0; a < 3; ++a) w[a] += PN[(size_t)(f * 3 + a) * S + g] * c;
    }
    R tp[NC];
    tab_row(tabP + j * 8, tp);
#pragma unroll
    for (int a = 0; a < AX; ++a) {
      const R coef = rho * w[a];
#pragma unroll
      for (int q = 0; q < NC; ++q) rhs[a][q] += coef * tp[q];
    }
  }
}

// ch = U blockdiag(G_b) U^T rhs: rotate the axes into the eigenbasis of
// sum_f n_f n_f^T, one packed 8x8 inverse per rotated axis, rotate back
template <class R>
__device__ __forceinline__ void poly_solve(const R *PG, const R *PU, size_t S, size_t g, const R (&rhs)[AX][NC],
                                           R (&ch)[AX][NC]) {
  R U[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) U[a][b] = PU[(size_t)(a * 3 + b) * S + g];
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int q = 0; q < NC; ++q) ch[a][q] = R(0);
#pragma unroll 1
  for (int b = 0; b < 3; ++b) {
    R rt[NC], ct[NC], Gb[NG];
#pragma unroll
    for (int q = 0; q < NC; ++q) rt[q] = U[0][b] * rhs[0][q] + U[1][b] * rhs[1][q] + U[2][b] * rhs[2][q];
#pragma unroll
    for (int q = 0; q < NG; ++q) Gb[q] = PG[(size_t)(b * NG + q) * S + g];
    apply_g(Gb, rt, ct);
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) ch[a][q] += U[a][b] * ct[q];
  }
}

// y_jf <- n_f . p(t_j) - h_f + max(0, y_jf): the slack projection and dual
// update of Eq. 18d-e in the compressed form (s = max(0, -y), v = max(0, y))
template <class R>
__device__ __forceinline__ void poly_update(const R *PN, const R *PH, size_t S, size_t g, int F, int M, R *ypoly,
                                            int stride, const R *tabP, const R (&ch)[AX][NC], int j0 = 0,
                                            int js = 1) {
  for (int j = j0; j < M; j += js) {
    R pos[3], tp[NC];
    tab_row(tabP + j * 8, tp);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R acc = R(0);
#pragma unroll
      for (int q = 0; q < NC; ++q) acc += tp[q] * ch[a][q];
      pos[a] = acc;
    }
    for (int f = 0; f < F; ++f) {
      R v = R(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) v += PN[(size_t)(f * 3 + a) * S + g] * pos[a];
      R *y = &ypoly[(j * F + f) * stride];
      *y = v - PH[(size_t)f * S + g] + rmax0(*y);
    }
  }
}

// rho M^T (s .* dz) for one axis, mapped back to the paper's coefficients
// (multiplied by T^k), squared and summed: one segment's share of ||r_d||^2
// (Eq. 20), in the iteration's precision (FP64 arithmetic runs at 1/64 of the
// FP32 rate on this GPU, and the residual norms only steer the stopping test)
template <class R>
__device__ __forceinline__ R dual_residual_sq(const R (&dS)[ND], const R (&dE)[ND], R rho, const R (&Tk)[NC]) {
  R x[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) x[q] = R(0);
  consensus_rhs(dS, dE, rho, x);
  R acc = R(0);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const R v = x[q] * Tk[q];
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

// The next rho of residual balancing (Eq. 22), in FP64 on the FP64 residual norms.
__device__ __forceinline__ double next_rho(const DevProblem &p, double rho, double rp, double rd) {
  if (rp > p.rho_mu * rd) return rho * p.rho_incr;
  if (rd > p.rho_mu * rp) return rho / p.rho_decr;
  return rho;
}

// The local-matrix inverse for a new rho from the segment's adaptive-rho data
// (layout NE_* of top_internal.h): G = A0 / rho + sum_k y_k y_k^T / (lambda_k + rho).
// Every term is a positive multiple of a rank-one square, so the sum has no
// cancellation whatever rho is.  Written one entry at a time to global memory
// (Gw[q * S + g], the packed layout of the precompute): a dozen registers
// instead of 36 accumulators, for kernels that keep G in registers and
// reload it afterwards.
template <class R>
__device__ __forceinline__ void g_from_eig_store(const R *E, size_t S, size_t g, double rho, R *Gw) {
  const R ir = R(1.0 / rho);
  R w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = R(1.0 / (double(E[(size_t)(NE_L + k) * S + g]) + rho));
#pragma unroll 1
  for (int r = 0; r < NC; ++r) {
    R yr[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) yr[k] = w[k] * E[(size_t)(NE_Y + r * 4 + k) * S + g];
#pragma unroll 1
    for (int c = r; c < NC; ++c) {
      R v = (c < PO) ? E[(size_t)(NE_A0 + c * (c + 1) / 2 + r) * S + g] * ir : R(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) v += yr[k] * E[(size_t)(NE_Y + c * 4 + k) * S + g];
      Gw[(size_t)(r * NC - (r * (r - 1)) / 2 + (c - r)) * S + g] = v;
    }
  }
}

// q' = phi + f (q - phi), phi = the projection of q: the compressed ball /
// velocity-norm state with its scaled dual w = q - phi multiplied by f and
// the projection unchanged (the ray from phi through q keeps its projection).
template <class R>
__device__ __forceinline__ void rescale_projected(R *q, int stride, const R (&o)[3], R rad, R f) {
  R qv[3], ph[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) qv[a] = q[a * stride];
  project_ball(qv, o, rad, ph);
#pragma unroll
  for (int a = 0; a < 3; ++a) q[a * stride] = ph[a] + f * (qv[a] - ph[a]);
}

// ---------------------------------------------------------------------------
// Numerical local step for general convex constraints (Sec. III-C.3, Eq.
// 15-17): per segment, minimise
//   F(c) = c^T Qt c + rho/2 ||E(Mt c - z~ + u)||^2
//          + sum_j [rho/2 g_vj^2 + y_vj g_vj + rho/2 g_aj^2 + y_aj g_aj],
//   g = max(0, ||A c||^2 - g_max^2)^2   (velocity / acceleration norm at t_j)
// by L-BFGS in the normalised coordinates, with the exact inverse Hessian of
// the quadratic part (G, precomputed in FP64) as the initial inverse-Hessian
// approximation, starting from the minimiser of the quadratic part (which is
// the answer whenever no bound is violated there).  Then y += rho g (Eq. 17).
// ---------------------------------------------------------------------------
constexpr int LBFGS_MAX_MEM = 8;

template <class R>
__device__ __forceinline__ R num_F(const R (&ch)[AX][NC], const R (&w)[AX][2][ND], const SegConst<R> &sc, R rho,
                                   bool first, bool last, const R *yg, int stride, const R *tabV, const R *tabA,
                                   int Mg, R vmax, R amax, R (&gr)[AX][NC]) {
  R F = R(0);
  const R t7 = sc.s[7];
#pragma unroll
  for (int a = 0; a < AX; ++a) {
#pragma unroll
    for (int k = 0; k < NC; ++k) gr[a][k] = R(0);
#pragma unroll
    for (int k = PO; k < NC; ++k) {
      R acc = R(0);
#pragma unroll
      for (int l = PO; l < NC; ++l) acc += R(qhat(k, l)) * ch[a][l];
      F += t7 * ch[a][k] * acc;
      gr[a][k] = R(2) * t7 * acc;
    }
    R eS[ND], eE[ND], dS[ND], dE[ND];
    end_derivs(ch[a], sc.s, eS, eE);
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      const R a0 = (first && r >= PO) ? R(0) : eS[r] - w[a][0][r];
      const R a1 = (last && r >= PO) ? R(0) : eE[r] - w[a][1][r];
      F += R(0.5) * rho * (a0 * a0 + a1 * a1);
      dS[r] = sc.s[r] * a0;
      dE[r] = sc.s[r] * a1;
    }
    consensus_rhs(dS, dE, rho, gr[a]);
  }
  for (int j = 0; j < Mg; ++j) {
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const R *tab = kind ? tabA + j * 8 : tabV + j * 8;
      const R sc_t = kind ? sc.s[2] : sc.s[1];
      const R gmax = kind ? amax : vmax;
      R v[AX];
      R n2 = R(0);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < NC; ++k) acc += tab[k] * ch[a][k];
        v[a] = sc_t * acc;
        n2 += v[a] * v[a];
      }
      const R h = n2 - gmax * gmax;
      if (h > R(0)) {
        const R g = h * h;
        const R y = yg[(j * 2 + kind) * stride];
        F += R(0.5) * rho * g * g + y * g;
        const R coef = (rho * g + y) * R(4) * h * sc_t;
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int k = 0; k < NC; ++k) gr[a][k] += coef * v[a] * tab[k];
      }
    }
  }
  return F;
}

template <class R>
__device__ __forceinline__ R dot24(const R (&x)[AX][NC], const R (&y)[AX][NC]) {
  R acc = R(0);
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) acc += x[a][k] * y[a][k];
  return acc;
}

// returns the L-BFGS iteration count; ch receives the minimiser, y is advanced.
// DEFER: only the start and its bound check, -1 where a bound is violated (the
// caller hands the segment to the warp-cooperative solver); the L-BFGS code is
// then not compiled into the caller, which keeps its register count low.
template <class R, bool DEFER = false>
__device__ int numeric_step(const SegConst<R> &sc, const R (&w)[AX][2][ND], R rho, bool first, bool last, R *yg,
                            int stride, const R *tabV, const R *tabA, int Mg, R vmax, R amax, int mem, int max_it,
                            R tol, R (&ch)[AX][NC]) {
  // start: minimiser of the quadratic part (the closed-form step without constraint rows)
  R rhs[AX][NC];
#pragma unroll
  for (int a = 0; a < AX; ++a) {
    R oS[ND], oE[ND];
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      oS[r] = (first && r >= PO) ? R(0) : sc.s[r] * w[a][0][r];
      oE[r] = (last && r >= PO) ? R(0) : sc.s[r] * w[a][1][r];
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) rhs[a][q] = R(0);
    consensus_rhs(oS, oE, rho, rhs[a]);
    apply_g(sc.G, rhs[a], ch[a]);
  }
  // If no bound is violated at the minimiser of the quadratic part, every
  // penalty term and its gradient vanish there and F >= quadratic part >=
  // its minimum = F(start): the start is the exact minimiser (and y stays).
  {
    bool violated = false;
    for (int j = 0; j < Mg && !violated; ++j) {
#pragma unroll
      for (int kind = 0; kind < 2; ++kind) {
        const R *tab = kind ? tabA + j * 8 : tabV + j * 8;
        const R sc_t = kind ? sc.s[2] : sc.s[1];
        const R gmax = kind ? amax : vmax;
        R n2 = R(0);
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          R acc = R(0);
#pragma unroll
          for (int k = 0; k < NC; ++k) acc += tab[k] * ch[a][k];
          n2 += (sc_t * acc) * (sc_t * acc);
        }
        if (n2 > gmax * gmax) violated = true;
      }
    }
    if (!violated) return 0;
    if constexpr (DEFER) return -1;
  }
  if constexpr (DEFER) return -1;  // (not reached: keeps the L-BFGS code out of DEFER instances)
  R scale = dot24(rhs, ch);  // rhs^T G rhs: size of the linear term in the G metric
  if (!(scale > R(0))) scale = R(1);
  R g[AX][NC], gn[AX][NC], d[AX][NC], xn[AX][NC];
  R Fv = num_F(ch, w, sc, rho, first, last, yg, stride, tabV, tabA, Mg, vmax, amax, g);
  R Sh[LBFGS_MAX_MEM][AX][NC], Yh[LBFGS_MAX_MEM][AX][NC], rh[LBFGS_MAX_MEM], al[LBFGS_MAX_MEM];
  if (mem > LBFGS_MAX_MEM) mem = LBFGS_MAX_MEM;
  if (mem < 1) mem = 1;
  int npair = 0, head = 0, it = 0;
  for (it = 0; it < max_it; ++it) {
    // preconditioned gradient norm g^T G g
#pragma unroll
    for (int a = 0; a < AX; ++a) apply_g(sc.G, g[a], d[a]);
    const R gGg = dot24(g, d);
    if (!(gGg > tol * tol * scale)) break;
    // two-loop recursion with H0 = G
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int k = 0; k < NC; ++k) xn[a][k] = g[a][k];
    for (int q = 0; q < npair; ++q) {
      const int idx = (head - 1 - q + mem) % mem;
      al[q] = rh[idx] * dot24(Sh[idx], xn);
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int k = 0; k < NC; ++k) xn[a][k] -= al[q] * Yh[idx][a][k];
    }
#pragma unroll
    for (int a = 0; a < AX; ++a) apply_g(sc.G, xn[a], d[a]);
    for (int q = npair - 1; q >= 0; --q) {
      const int idx = (head - 1 - q + mem) % mem;
      const R be = rh[idx] * dot24(Yh[idx], d);
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int k = 0; k < NC; ++k) d[a][k] += (al[q] - be) * Sh[idx][a][k];
    }
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int k = 0; k < NC; ++k) d[a][k] = -d[a][k];
    R gd = dot24(g, d);
    if (!(gd < R(0))) {  // not a descent direction: restart from the preconditioned gradient
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        apply_g(sc.G, g[a], d[a]);
#pragma unroll
        for (int k = 0; k < NC; ++k) d[a][k] = -d[a][k];
      }
      gd = dot24(g, d);
      npair = 0;
    }
    // Armijo backtracking (c1 = 1e-4, halving)
    R step = R(1), Fn = Fv;
    bool ok = false;
    for (int bt = 0; bt < 30; ++bt) {
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int k = 0; k < NC; ++k) xn[a][k] = ch[a][k] + step * d[a][k];
      Fn = num_F(xn, w, sc, rho, first, last, yg, stride, tabV, tabA, Mg, vmax, amax, gn);
      if (Fn <= Fv + R(1e-4) * step * gd) { ok = true; break; }
      step *= R(0.5);
    }
    if (!ok) break;
    R sy = R(0);
    const int slot = head;
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        Sh[slot][a][k] = xn[a][k] - ch[a][k];
        Yh[slot][a][k] = gn[a][k] - g[a][k];
        sy += Sh[slot][a][k] * Yh[slot][a][k];
      }
    if (sy > R(0)) {
      rh[slot] = R(1) / sy;
      head = (head + 1) % mem;
      if (npair < mem) ++npair;
    }
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int k = 0; k < NC; ++k) { ch[a][k] = xn[a][k]; g[a][k] = gn[a][k]; }
    Fv = Fn;
  }
  // general-constraint duals (Eq. 17 dual update, y += rho g)
  for (int j = 0; j < Mg; ++j) {
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const R *tab = kind ? tabA + j * 8 : tabV + j * 8;
      const R sc_t = kind ? sc.s[2] : sc.s[1];
      const R gmax = kind ? amax : vmax;
      R n2 = R(0);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < NC; ++k) acc += tab[k] * ch[a][k];
        n2 += (sc_t * acc) * (sc_t * acc);
      }
      const R h = n2 - gmax * gmax;
      if (h > R(0)) yg[(j * 2 + kind) * stride] += rho * h * h;
    }
  }
  return it;
}

// ---- the numerical step with one warp per segment ----
// Lane a * 8 + k (a < 3) holds coefficient k of axis a of every vector of the
// solve; lanes 24..31 hold zeros.  Sums over lanes are xor butterflies, whose
// result is bit-identical in every lane, so every branch on a sum is uniform.
// Same algorithm as numeric_step (start at the minimiser of the quadratic
// part, L-BFGS with H0 = G, Armijo backtracking, then y += rho g).

template <class R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R>
__device__ __forceinline__ R wsum8(R v) {  // over the 8 lanes of an axis
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

__device__ __forceinline__ int fact_rt(int r) {
  int f = 1;
  for (int i = 2; i <= r; ++i) f *= i;
  return f;
}

__device__ __forceinline__ int falling_rt(int k, int r) {
  int f = 1;
  for (int i = 0; i < r; ++i) f *= (k - i);
  return f;
}

// y = G x for this lane's axis (Grow = row k of G)
template <class R>
__device__ __forceinline__ R wapply_g(const R (&Grow)[NC], R x) {
  const int base = (threadIdx.x & 31) & ~7;
  R y = R(0);
#pragma unroll
  for (int l = 0; l < NC; ++l) y += Grow[l] * __shfl_sync(0xffffffffu, x, base + l);
  return y;
}

// this lane's integer constants of the basis (k = lane & 7), formed once per segment
template <class R>
struct WLane {
  R q[NC];   // Qh[k][l] (zero unless k, l >= p)
  R fr[NC];  // F(m, k) = m! / (m - k)!  (zero for m < k)
  R fc[ND];  // F(k, r)                  (zero for r > k)
  R fk;      // k!
};

template <class R>
__device__ __forceinline__ void wlane_init(WLane<R> &L) {
  const int k = threadIdx.x & 7;
#pragma unroll
  for (int l = 0; l < NC; ++l) {
    L.q[l] = (k >= PO && l >= PO)
                 ? R(double(falling_rt(k, PO)) * double(falling_rt(l, PO)) / double(k + l - 2 * PO + 1))
                 : R(0);
    L.fr[l] = l >= k ? R(falling_rt(l, k)) : R(0);
  }
#pragma unroll
  for (int r = 0; r < ND; ++r) L.fc[r] = r <= k ? R(falling_rt(k, r)) : R(0);
  L.fk = R(fact_rt(k));
}

// the objective of the numerical local step and this lane's gradient entry.
// The general-bound terms take one (sample, kind) pair per lane: lanes 0-15
// the velocity rows of samples j0 .. j0+15, lanes 16-31 their acceleration
// rows; each lane reduces its row's gradient weight to three per-axis values
// in the warp's scratch wsc[3][32], from which lane (axis, coefficient) sums
// its gradient entry.
template <class R>
__device__ R wnum_F(R c, R w0, R w1, const WLane<R> &L, const R (&s)[NC], R rho, bool first, bool last,
                    const R *yg, int stride, const R *tabV, const R *tabA, int Mg, R vmax, R amax, R *wsc, R &gr) {
  const int lane = threadIdx.x & 31, k = lane & 7, base = lane & ~7;
  const bool live = lane < 24;
  R call[AX][NC];  // every coefficient of the segment in every lane
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int l = 0; l < NC; ++l) call[a][l] = __shfl_sync(0xffffffffu, c, a * NC + l);
  R cax[NC];  // this lane's axis
#pragma unroll
  for (int l = 0; l < NC; ++l) cax[l] = base == 0 ? call[0][l] : (base == 8 ? call[1][l] : call[2][l]);
  R Floc = R(0);
  gr = R(0);
  if (live) {  // cost c^T Q(T) c = T^-7 ch^T Qh ch (rows k >= p only)
    R acc = R(0);
#pragma unroll
    for (int l = 0; l < NC; ++l) acc += L.q[l] * cax[l];
    Floc += s[7] * c * acc;
    gr = R(2) * s[7] * acc;
  }
  R dS = R(0), dE = R(0);
  if (live && k < ND) {  // consensus rows, E-masked at the trajectory's ends
    R acc = R(0);
#pragma unroll
    for (int m = 0; m < NC; ++m) acc += L.fr[m] * cax[m];
    const R a0 = (first && k >= PO) ? R(0) : L.fk * s[k] * c - w0;
    const R a1 = (last && k >= PO) ? R(0) : s[k] * acc - w1;
    Floc += R(0.5) * rho * (a0 * a0 + a1 * a1);
    dS = s[k] * a0;
    dE = s[k] * a1;
  }
  {
    R acc = (live && k < ND) ? L.fk * dS : R(0);
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      const R dEr = __shfl_sync(0xffffffffu, dE, base + r);
      if (live) acc += L.fc[r] * dEr;
    }
    gr += rho * acc;
  }
  const int kind = lane >> 4;
  const R sc_t = kind ? s[2] : s[1];
  const R gmax = kind ? amax : vmax;
  for (int j0 = 0; j0 < Mg; j0 += 16) {
    const int jj = j0 + (lane & 15);
    const bool on = jj < Mg;
    const R *tab = (kind ? tabA : tabV) + jj * 8;
    R va[AX] = {R(0), R(0), R(0)};
    if (on) {
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const R tq = tab[q];
#pragma unroll
        for (int a = 0; a < AX; ++a) va[a] += tq * call[a][q];
      }
#pragma unroll
      for (int a = 0; a < AX; ++a) va[a] *= sc_t;
    }
    const R h = va[0] * va[0] + va[1] * va[1] + va[2] * va[2] - gmax * gmax;
    R wgt = R(0);
    if (on && h > R(0)) {
      const R g = h * h;
      const R y = yg[(jj * 2 + kind) * stride];
      Floc += R(0.5) * rho * g * g + y * g;
      wgt = (rho * g + y) * R(4) * h * sc_t;
    }
#pragma unroll
    for (int a = 0; a < AX; ++a) wsc[a * 32 + lane] = wgt * va[a];
    __syncwarp();
    if (live) {
      const int a = lane >> 3;
      R acc = R(0);
#pragma unroll
      for (int p = 0; p < 32; ++p) {
        const int jp = j0 + (p & 15);
        if (jp < Mg) acc += wsc[a * 32 + p] * ((p >> 4) ? tabA : tabV)[jp * 8 + k];
      }
      gr += acc;
    }
    __syncwarp();  // the scratch is rewritten by the next block of samples
  }
  return wsum(Floc);
}

template <class R>
__device__ __forceinline__ R wdot(R x, R y) { return wsum(x * y); }

// the numerical local step of one segment by the calling warp; writes the
// lane's coefficient to *c_out and returns the L-BFGS iteration count
template <class R>
__device__ int numeric_step_warp(const R (&Grow)[NC], const R (&s)[NC], R w0, R w1, R rho, bool first, bool last,
                                 R *yg, int stride, const R *tabV, const R *tabA, int Mg, R vmax, R amax, int mem,
                                 int max_it, R tol, R *wsc, R &c_out) {
  const int lane = threadIdx.x & 31, k = lane & 7, base = lane & ~7;
  const bool live = lane < 24;
  WLane<R> L;
  wlane_init(L);
  // start: minimiser of the quadratic part, rhs = rho Mh^T E w
  R oS = (live && k < ND && !(first && k >= PO)) ? s[k] * w0 : R(0);
  R oE = (live && k < ND && !(last && k >= PO)) ? s[k] * w1 : R(0);
  R rhs = (live && k < ND) ? L.fk * oS : R(0);
#pragma unroll
  for (int r = 0; r < ND; ++r) {
    const R oEr = __shfl_sync(0xffffffffu, oE, base + r);
    if (live) rhs += L.fc[r] * oEr;
  }
  rhs *= rho;
  R c = wapply_g(Grow, rhs);
  R scale = wdot(rhs, c);
  if (!(scale > R(0))) scale = R(1);
  R g;
  R Fv = wnum_F(c, w0, w1, L, s, rho, first, last, yg, stride, tabV, tabA, Mg, vmax, amax, wsc, g);
  R Sh[LBFGS_MAX_MEM], Yh[LBFGS_MAX_MEM], rh[LBFGS_MAX_MEM], al[LBFGS_MAX_MEM];  // [0] = newest pair
#pragma unroll
  for (int q = 0; q < LBFGS_MAX_MEM; ++q) { Sh[q] = Yh[q] = rh[q] = al[q] = R(0); }
  if (mem > LBFGS_MAX_MEM) mem = LBFGS_MAX_MEM;
  if (mem < 1) mem = 1;
  int npair = 0, it = 0;
  for (it = 0; it < max_it; ++it) {
    R d = wapply_g(Grow, g);
    if (!(wdot(g, d) > tol * tol * scale)) break;
    R xn = g;
#pragma unroll
    for (int q = 0; q < LBFGS_MAX_MEM; ++q)
      if (q < npair) {
        al[q] = rh[q] * wdot(Sh[q], xn);
        xn -= al[q] * Yh[q];
      }
    d = wapply_g(Grow, xn);
#pragma unroll
    for (int q = LBFGS_MAX_MEM - 1; q >= 0; --q)
      if (q < npair) {
        const R be = rh[q] * wdot(Yh[q], d);
        d += (al[q] - be) * Sh[q];
      }
    d = -d;
    R gd = wdot(g, d);
    if (!(gd < R(0))) {  // not a descent direction: restart from the preconditioned gradient
      d = -wapply_g(Grow, g);
      gd = wdot(g, d);
      npair = 0;
    }
    R step = R(1), Fn = Fv, gn = g, x = c;
    bool ok = false;
    for (int bt = 0; bt < 30; ++bt) {
      x = c + step * d;
      Fn = wnum_F(x, w0, w1, L, s, rho, first, last, yg, stride, tabV, tabA, Mg, vmax, amax, wsc, gn);
      if (Fn <= Fv + R(1e-4) * step * gd) { ok = true; break; }
      step *= R(0.5);
    }
    if (!ok) break;
    const R sn = x - c, yn = gn - g;
    const R sy = wdot(sn, yn);
    if (sy > R(0)) {
#pragma unroll
      for (int q = LBFGS_MAX_MEM - 1; q > 0; --q) { Sh[q] = Sh[q - 1]; Yh[q] = Yh[q - 1]; rh[q] = rh[q - 1]; }
      Sh[0] = sn;
      Yh[0] = yn;
      rh[0] = R(1) / sy;
      if (npair < mem) ++npair;
    }
    c = x;
    g = gn;
    Fv = Fn;
  }
  // general-constraint duals (Eq. 17 dual update, y += rho g)
  for (int j = 0; j < Mg; ++j) {
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const R *tab = kind ? tabA + j * 8 : tabV + j * 8;
      const R sc_t = kind ? s[2] : s[1];
      const R gmax = kind ? amax : vmax;
      const R va = sc_t * wsum8((live ? tab[k] : R(0)) * c);
      const R v0 = __shfl_sync(0xffffffffu, va, 0), v1 = __shfl_sync(0xffffffffu, va, 8),
              v2 = __shfl_sync(0xffffffffu, va, 16);
      const R h = v0 * v0 + v1 * v1 + v2 * v2 - gmax * gmax;
      if (h > R(0) && lane == 0) yg[(j * 2 + kind) * stride] += rho * h * h;
    }
  }
  c_out = c;
  return it;
}

// acceleration rows: tab[j*8 + k] = k (k-1) tau_j^{k-2}
template <class R>
__device__ __forceinline__ void fill_accel_table(R *tab, int M, int tid, int nthreads) {
  for (int q = tid; q < 8 * M; q += nthreads) {
    const int j = q / 8 + 1, k = q % 8;
    const double tau = double(j) / double(M);
    double t = 1.0;
    for (int x = 0; x < k - 2; ++x) t *= tau;
    tab[q] = R(k < 2 ? 0.0 : double(k) * double(k - 1) * t);
  }
}

}  // namespace top
