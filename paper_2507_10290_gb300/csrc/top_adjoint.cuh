// top_adjoint.cuh -- reverse-mode derivative of the cost after K closed-form
// CADMM iterations (no inequality rows) with respect to the waypoints and the
// durations.  The paper has no gradient; this differentiates its iteration
// (Eq. 18a-c) exactly as the forward kernels compute it.
//
// Forward map per iteration k (per segment i, per axis, normalised
// coordinates of top_math.cuh):
//   w   = E (z~ - u)                       targets at both ends (14 rows)
//   ch  = G(T) rho Mh^T (s .* w)           local solve, G = (D K D)^{-1}
//   e   = s .* (Mh ch)                     end derivatives
//   junction j (free rows):  z' = (eE_{j-1} + eS_j)/2, uL' = uL + eE - z', uR' = uR + eS - z'
//   pinned rows:             z' = P_j,                uL' = uL + eE - P,  uR' = uR + eS - P
//   trajectory ends (r<4):   u' = u + e - z_fixed
//   J = sum_i T_i^-7 ch^T Qh ch after the last local solve.
// Reverse step k (adjoint state xb = (zb, uLb, uRb) of x^{k+1}):
//   adj_junction: fold in the target adjoints of step k+1 (wb), then reverse
//                 the junction update: eb for both neighbours, zb -> 0 on free
//                 rows, pinned rows feed dP
//   adj_segment:  recompute ch from x^k (tape), reverse the local solve:
//                 chb = Mh^T (s .* eb) (+ the cost seed), rb = G chb,
//                 dT += -rb^T K'(T) ch + the s(T) terms, wb = s .* (rho Mh rb)
// The forward state x^k comes from checkpoints every `ckpt` iterations; each
// block is recomputed forward into a tape of `ckpt` states.
//
// With inequality rows (adj_segment_rows) the state also holds the box rows'
// compressed slack/dual y and the ball / velocity-norm projection states q
// (Eq. 18d-g, top_step.cuh), and the reverse local step adds:
//   box      y' = +-s_1 tB.ch - vmax + max(0, y);  rhs += rho s_1 (|y-| - |y+|) tB
//   ball     q' = tQ.ch + [k>0] (q - P(q));       rhs += [k>0] rho (2 P(q) - q) tQ
//   v-norm   q' = s_1 tV.ch + [k>0] (q - P(q));   rhs += [k>0] rho s_1 (2 P(q) - q) tV
// with P the projection onto the ball (Jacobian I inside, r/n (I - d d^T / n^2)
// outside, d = q - o, n = |d|), and the rows' share of K(T) = rho sum
// (2 s_1^2 tB tB^T + tQ tQ^T + s_1^2 tV tV^T) in dK/dT.  At a kink (y = 0,
// |q - o| = r exactly) the inactive branch is taken: max'(0) = 0, |.|'(0) = 0,
// P' = I.
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"
#include "top_step.cuh"

namespace top {

// fold the target adjoints of the following local step into junction jE (and jS for a first segment)
template <class R>
__device__ __forceinline__ void adj_fold(const AdjArgs &A, int b, int g, bool first, bool last) {
  const StreamArgs &F = A.f;
  R *zb = (R *)A.zb, *uLb = (R *)A.uLb, *uRb = (R *)A.uRb, *uR0b = (R *)A.uR0b;
  const R *wbS = (const R *)A.wbS, *wbE = (const R *)A.wbE;
  const int jE = g + b + 1;
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      const size_t row = (size_t)(a * ND + r) * F.Jn;
      const size_t sr = (size_t)(a * ND + r) * F.S;
      const R we = wbE[sr + g];
      if (!last) {
        const R ws = wbS[sr + g + 1];
        zb[row + jE] += we + ws;
        uLb[row + jE] -= we;
        uRb[row + jE] -= ws;
      } else if (r < PO) {
        uLb[row + jE] -= we;
      }
      if (first && r < PO) uR0b[(size_t)(a * PO + r) * F.p.B + b] -= wbS[sr + g];
    }
}

template <class R>
__global__ void __launch_bounds__(256) adj_junction(const AdjArgs A) {
  const StreamArgs &F = A.f;
  const bool pin = F.p.mode == 0;
  R *zb = (R *)A.zb, *uLb = (R *)A.uLb, *uRb = (R *)A.uRb, *uR0b = (R *)A.uR0b;
  R *eSb = (R *)A.eSb, *eEb = (R *)A.eEb;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < F.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(F, x, t, b, i, N, g)) continue;
    const bool first = i == 0, last = i == N - 1;
    const int jE = g + b + 1;
    adj_fold<R>(A, b, g, first, last);
    double pb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * F.Jn;
        const size_t sr = (size_t)(a * ND + r) * F.S;
        if (!last) {
          const R zz = zb[row + jE], ul = uLb[row + jE], ur = uRb[row + jE];
          if (pin && r == 0) {
            eEb[sr + g] = ul;
            eSb[sr + g + 1] = ur;
            pb[a] += double(zz) - double(ul) - double(ur);
          } else {
            const R zt = zz - ul - ur;
            eEb[sr + g] = ul + R(0.5) * zt;
            eSb[sr + g + 1] = ur + R(0.5) * zt;
          }
          zb[row + jE] = R(0);
        } else {
          eEb[sr + g] = r < PO ? uLb[row + jE] : R(0);
        }
        if (first) eSb[sr + g] = r < PO ? uR0b[(size_t)(a * PO + r) * F.p.B + b] : R(0);
      }
    if (pin && !last)
      for (int a = 0; a < 3; ++a) A.Pbar[(size_t)jE * 3 + a] += pb[a];
  }
}

template <class R>
__global__ void __launch_bounds__(256) adj_segment(const AdjArgs A, int seed) {
  const StreamArgs &F = A.f;
  const DevProblem &p = F.p;
  const bool pin = p.mode == 0;
  const R rho = R(p.rho);
  const R *tz = (const R *)A.tz, *tuL = (const R *)A.tuL, *tuRp = (const R *)A.tuRp, *tuR0 = (const R *)A.tuR0;
  const R *Gp = (const R *)F.G;
  const R *eSb = (const R *)A.eSb, *eEb = (const R *)A.eEb;
  R *wbS = (R *)A.wbS, *wbE = (R *)A.wbE;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < F.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(F, x, t, b, i, N, g)) continue;
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    R G[NG], s[NC];
#pragma unroll
    for (int q = 0; q < NG; ++q) G[q] = Gp[(size_t)q * F.S + g];
    const R T = R(p.durations[g]);
    inv_powers(T, s);
    const R iT = s[1];
    double tbar = 0.0;
#pragma unroll 1
    for (int a = 0; a < AX; ++a) {
      // ---- forward recompute from x^k ----
      R w[2][ND], om[2][ND];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * F.Jn;
        R us;
        if (first) us = (r < PO) ? tuR0[(size_t)(a * PO + r) * p.B + b] : R(0);
        else if (pin && r == 0) us = tuRp[(size_t)a * F.Jn + jS];
        else us = -tuL[row + jS];
        w[0][r] = (first && r >= PO) ? R(0) : tz[row + jS] - us;
        w[1][r] = (last && r >= PO) ? R(0) : tz[row + jE] - tuL[row + jE];
        om[0][r] = s[r] * w[0][r];
        om[1][r] = s[r] * w[1][r];
      }
      R rh[NC], ch[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) rh[q] = R(0);
      consensus_rhs(om[0], om[1], rho, rh);
      apply_g(G, rh, ch);
      // M ch rows (unscaled by s)
      R mcS[ND], mcE[ND];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        mcS[r] = R(fact(r)) * ch[r];
        R acc = R(0);
#pragma unroll
        for (int k = r; k < NC; ++k) acc += R(falling(k, r)) * ch[k];
        mcE[r] = acc;
      }
      // ---- reverse ----
      R eb[2][ND], seb[2][ND];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t sr = (size_t)(a * ND + r) * F.S;
        eb[0][r] = eSb[sr + g];
        eb[1][r] = eEb[sr + g];
        seb[0][r] = s[r] * eb[0][r];
        seb[1][r] = s[r] * eb[1][r];
        // s_r enters e_r = s_r (M ch)_r on both sides
        tbar += (double(eb[0][r]) * double(mcS[r]) + double(eb[1][r]) * double(mcE[r])) *
                (-double(r) * double(s[r]) / double(T));
      }
      R chb[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) chb[q] = R(0);
      consensus_rhs(seb[0], seb[1], R(1), chb);
      if (seed) {
        const double dj = A.dJ[b];
        const double t7 = double(s[7]);
        double qc[NC], cqc = 0.0;
        for (int k1 = 0; k1 < NC; ++k1) {
          double acc = 0.0;
          for (int k2 = 0; k2 < NC; ++k2) acc += qhat(k1, k2) * double(ch[k2]);
          qc[k1] = acc;
          cqc += double(ch[k1]) * acc;
        }
        for (int k1 = 0; k1 < NC; ++k1) chb[k1] += R(dj * 2.0 * t7 * qc[k1]);
        tbar += dj * (-7.0) * t7 / double(T) * cqc;
      }
      R rb[NC];
      apply_g(G, chb, rb);
      // dT from G(T): -rb^T K'(T) ch, K' = -14 T^-8 Qh + rho sum_rows E (-2 r s_r^2 / T) m m^T
      {
        double rqc = 0.0;
        for (int k1 = PO; k1 < NC; ++k1)
          for (int k2 = PO; k2 < NC; ++k2) rqc += double(rb[k1]) * qhat(k1, k2) * double(ch[k2]);
        double kp = -14.0 * double(s[7]) * double(iT) * rqc;
        for (int r = 1; r < ND; ++r) {
          const double c2 = -2.0 * double(r) * double(s[r]) * double(s[r]) * double(iT);
          if (!(first && r >= PO)) kp += double(rho) * c2 * (double(fact(r)) * double(rb[r])) * double(mcS[r]);
          if (!(last && r >= PO)) {
            double mr = 0.0;
            for (int k = r; k < NC; ++k) mr += double(falling(k, r)) * double(rb[k]);
            kp += double(rho) * c2 * mr * double(mcE[r]);
          }
        }
        tbar -= kp;
      }
      // omega_b = rho Mh rb; s enters omega = s .* w; wb = s .* omega_b (masked)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t sr = (size_t)(a * ND + r) * F.S;
        R obS = rho * R(fact(r)) * rb[r];
        R acc = R(0);
#pragma unroll
        for (int k = r; k < NC; ++k) acc += R(falling(k, r)) * rb[k];
        R obE = rho * acc;
        if (first && r >= PO) obS = R(0);
        if (last && r >= PO) obE = R(0);
        tbar += (double(obS) * double(w[0][r]) + double(obE) * double(w[1][r])) *
                (-double(r) * double(s[r]) / double(T));
        wbS[sr + g] = s[r] * obS;
        wbE[sr + g] = s[r] * obE;
      }
    }
    A.Tbar[g] += tbar;
  }
}

// the Jacobian of the projection onto ||x - o|| <= rad applied to g
// (symmetric; identity inside and on the boundary)
template <class R>
__device__ __forceinline__ void proj_jac(const R (&q)[3], const R (&o)[3], R rad, const R (&gv)[3], R (&out)[3]) {
  const R d0 = q[0] - o[0], d1 = q[1] - o[1], d2 = q[2] - o[2];
  const R n2 = d0 * d0 + d1 * d1 + d2 * d2;
  if (!(n2 > rad * rad)) {
    out[0] = gv[0]; out[1] = gv[1]; out[2] = gv[2];
    return;
  }
  const R n = sqrt(n2);
  const R f = rad / n;
  const R dg = (d0 * gv[0] + d1 * gv[1] + d2 * gv[2]) / n2;
  out[0] = f * (gv[0] - dg * d0);
  out[1] = f * (gv[1] - dg * d1);
  out[2] = f * (gv[2] - dg * d2);
}

// reverse of the local step with box / ball / velocity-norm rows (all three
// axes at once: the projections couple them); see the header for the maps
template <class R, int F>
__global__ void __launch_bounds__(256) adj_segment_rows(const AdjArgs A, int seed, int kiter) {
  constexpr bool BOX = (F & FAM_BOX) != 0, BALL = (F & FAM_BALL) != 0, VN = (F & FAM_VN) != 0;
  const StreamArgs &Fw = A.f;
  const DevProblem &p = Fw.p;
  extern __shared__ __align__(16) unsigned char smem[];
  const int Mb = BOX ? p.M_box : 0, Mq = BALL ? p.M_ball : 0, Mv = VN ? p.M_vn : 0;
  R *tabB = (R *)smem, *tabQ = tabB + 8 * Mb, *tabV = tabQ + 8 * Mq;
  if (BOX) fill_sample_table(tabB, Mb, 1, threadIdx.x, blockDim.x);
  if (BALL) fill_sample_table(tabQ, Mq, 0, threadIdx.x, blockDim.x);
  if (VN) fill_sample_table(tabV, Mv, 1, threadIdx.x, blockDim.x);
  __syncthreads();
  const bool pin = p.mode == 0;
  const bool later = kiter > 0;  // the projections' previous duals enter after the first iteration
  const R rho = R(p.rho);
  const size_t S = (size_t)Fw.S;
  const R *tz = (const R *)A.tz, *tuL = (const R *)A.tuL, *tuRp = (const R *)A.tuRp, *tuR0 = (const R *)A.tuR0;
  const R *tyb = (const R *)A.tyb, *tqb = (const R *)A.tqb, *tqv = (const R *)A.tqv;
  R *ybb = (R *)A.ybb, *qbb = (R *)A.qbb, *qvb = (R *)A.qvb;
  const R *Gp = (const R *)Fw.G;
  const R *eSb = (const R *)A.eSb, *eEb = (const R *)A.eEb;
  R *wbS = (R *)A.wbS, *wbE = (R *)A.wbE;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < Fw.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(Fw, x, t, b, i, N, g)) continue;
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    SegConst<R> sc;
#pragma unroll
    for (int q = 0; q < NG; ++q) sc.G[q] = Gp[(size_t)q * S + g];
    const R T = R(p.durations[g]);
    inv_powers(T, sc.s);
    const R iT = sc.s[1];
    const R ds1 = -sc.s[1] * iT;  // d s_1 / dT
    sc.vbox = BOX ? R(p.vbox[b]) : R(0);
    sc.vnorm = VN ? R(p.vnorm[b]) : R(0);
    sc.brad = BALL ? R(p.ball_r[g]) : R(0);
    for (int a = 0; a < 3; ++a) sc.bo[a] = BALL ? R(p.ball_c[(size_t)g * 3 + a]) : R(0);
    const R zero3[3] = {R(0), R(0), R(0)};
    double tbar = 0.0;
    // ---- forward recompute of the local step from x^k ----
    R w[AX][2][ND], wS[AX][ND], wE[AX][ND];
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * Fw.Jn;
        R us;
        if (first) us = (r < PO) ? tuR0[(size_t)(a * PO + r) * p.B + b] : R(0);
        else if (pin && r == 0) us = tuRp[(size_t)a * Fw.Jn + jS];
        else us = -tuL[row + jS];
        w[a][0][r] = (first && r >= PO) ? R(0) : tz[row + jS] - us;
        w[a][1][r] = (last && r >= PO) ? R(0) : tz[row + jE] - tuL[row + jE];
        wS[a][r] = sc.s[r] * w[a][0][r];
        wE[a][r] = sc.s[r] * w[a][1][r];
      }
    R rhs[AX][NC], ch[AX][NC];
    family_rhs<R, F>(sc, wS, wE, rho, !later, tyb + g, tqb + g, tqv + g, (int)S, tabB, tabQ, tabV, Mb, Mq, Mv, rhs);
#pragma unroll
    for (int a = 0; a < AX; ++a) apply_g(sc.G, rhs[a], ch[a]);
    // ---- reverse: end derivatives ----
    R chb[AX][NC];
    R mcS[AX][ND], mcE[AX][ND];
#pragma unroll
    for (int a = 0; a < AX; ++a) {
      R sbS[ND], sbE[ND];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        mcS[a][r] = R(fact(r)) * ch[a][r];
        R acc = R(0);
#pragma unroll
        for (int q = r; q < NC; ++q) acc += R(falling(q, r)) * ch[a][q];
        mcE[a][r] = acc;
        const size_t sr = (size_t)(a * ND + r) * S;
        const R e0 = eSb[sr + g], e1 = eEb[sr + g];
        tbar += double((e0 * mcS[a][r] + e1 * mcE[a][r]) * (-R(r) * sc.s[r] * iT));
        sbS[r] = sc.s[r] * e0;
        sbE[r] = sc.s[r] * e1;
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) chb[a][q] = R(0);
      consensus_rhs(sbS, sbE, R(1), chb[a]);
    }
    // ---- reverse: the rows' state updates (adjoints of x^{k+1} in ybb, qbb, qvb) ----
    if (BOX)
      for (int j = 0; j < Mb; ++j)
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          R tc = R(0);
#pragma unroll
          for (int q = 0; q < NC; ++q) tc += tabB[j * 8 + q] * ch[a][q];
          const size_t ip = (size_t)((j * 3 + a) * 2 + 0) * S + g, im = (size_t)((j * 3 + a) * 2 + 1) * S + g;
          const R bp = ybb[ip], bm = ybb[im];
          const R vb = bp - bm;  // adjoint of v = s_1 tB.ch
#pragma unroll
          for (int q = 0; q < NC; ++q) chb[a][q] += sc.s[1] * tabB[j * 8 + q] * vb;
          tbar += double(vb * ds1 * tc);
          ybb[ip] = tyb[ip] > R(0) ? bp : R(0);  // through max(0, y)
          ybb[im] = tyb[im] > R(0) ? bm : R(0);
        }
    if (BALL)
      for (int j = 0; j < Mq; ++j) {
        R qv[3], qb[3], jq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          qv[a] = tqb[(size_t)(j * 3 + a) * S + g];
          qb[a] = qbb[(size_t)(j * 3 + a) * S + g];
        }
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int q = 0; q < NC; ++q) chb[a][q] += tabQ[j * 8 + q] * qb[a];
        proj_jac(qv, sc.bo, sc.brad, qb, jq);
#pragma unroll
        for (int a = 0; a < 3; ++a) qbb[(size_t)(j * 3 + a) * S + g] = later ? qb[a] - jq[a] : R(0);
      }
    if (VN)
      for (int j = 0; j < Mv; ++j) {
        R qv[3], qb[3], jq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          qv[a] = tqv[(size_t)(j * 3 + a) * S + g];
          qb[a] = qvb[(size_t)(j * 3 + a) * S + g];
        }
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          R tc = R(0);
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            chb[a][q] += sc.s[1] * tabV[j * 8 + q] * qb[a];
            tc += tabV[j * 8 + q] * ch[a][q];
          }
          tbar += double(qb[a] * ds1 * tc);
        }
        proj_jac(qv, zero3, sc.vnorm, qb, jq);
#pragma unroll
        for (int a = 0; a < 3; ++a) qvb[(size_t)(j * 3 + a) * S + g] = later ? qb[a] - jq[a] : R(0);
      }
    if (seed) {  // the cost seed: J = T^-7 ch^T Qh ch after the last iteration
      const double dj = A.dJ[b];
      const double t7 = double(sc.s[7]);
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        double cqc = 0.0;
        for (int k1 = PO; k1 < NC; ++k1) {
          double acc = 0.0;
          for (int k2 = PO; k2 < NC; ++k2) acc += qhat(k1, k2) * double(ch[a][k2]);
          chb[a][k1] += R(dj * 2.0 * t7 * acc);
          cqc += double(ch[a][k1]) * acc;
        }
        tbar += dj * (-7.0) * t7 / double(T) * cqc;
      }
    }
    // ---- reverse: the local solve, G(T) = K(T)^-1 ----
    R rb[AX][NC];
#pragma unroll
    for (int a = 0; a < AX; ++a) apply_g(sc.G, chb[a], rb[a]);
    {
      double kp = 0.0;
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        double rqc = 0.0;
        for (int k1 = PO; k1 < NC; ++k1)
          for (int k2 = PO; k2 < NC; ++k2) rqc += double(rb[a][k1]) * qhat(k1, k2) * double(ch[a][k2]);
        kp += -14.0 * double(sc.s[7]) * double(iT) * rqc;
        for (int r = 1; r < ND; ++r) {
          const double c2 = -2.0 * double(r) * double(sc.s[r]) * double(sc.s[r]) * double(iT);
          if (!(first && r >= PO)) kp += double(rho) * c2 * (double(fact(r)) * double(rb[a][r])) * double(mcS[a][r]);
          if (!(last && r >= PO)) {
            double mr = 0.0;
            for (int q = r; q < NC; ++q) mr += double(falling(q, r)) * double(rb[a][q]);
            kp += double(rho) * c2 * mr * double(mcE[a][r]);
          }
        }
        // the rows' share of K: rho sum_j (2 s_1^2 tB tB^T + s_1^2 tV tV^T); d(s_1^2)/dT = -2 s_1^2 / T
        const double dss = -2.0 * double(sc.s[1]) * double(sc.s[1]) * double(iT);
        for (int j = 0; j < Mb; ++j) {
          double tr = 0.0, tc = 0.0;
          for (int q = 0; q < NC; ++q) { tr += double(tabB[j * 8 + q]) * double(rb[a][q]); tc += double(tabB[j * 8 + q]) * double(ch[a][q]); }
          kp += double(rho) * 2.0 * dss * tr * tc;
        }
        for (int j = 0; j < Mv; ++j) {
          double tr = 0.0, tc = 0.0;
          for (int q = 0; q < NC; ++q) { tr += double(tabV[j * 8 + q]) * double(rb[a][q]); tc += double(tabV[j * 8 + q]) * double(ch[a][q]); }
          kp += double(rho) * dss * tr * tc;
        }
      }
      tbar -= kp;
    }
    // ---- reverse: the right-hand side (targets and rows) ----
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t sr = (size_t)(a * ND + r) * S;
        R obS = rho * R(fact(r)) * rb[a][r];
        R acc = R(0);
#pragma unroll
        for (int q = r; q < NC; ++q) acc += R(falling(q, r)) * rb[a][q];
        R obE = rho * acc;
        if (first && r >= PO) obS = R(0);
        if (last && r >= PO) obE = R(0);
        tbar += double((obS * w[a][0][r] + obE * w[a][1][r]) * (-R(r) * sc.s[r] * iT));
        wbS[sr + g] = sc.s[r] * obS;
        wbE[sr + g] = sc.s[r] * obE;
      }
    if (BOX)
      for (int j = 0; j < Mb; ++j)
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          R gr = R(0);
#pragma unroll
          for (int q = 0; q < NC; ++q) gr += tabB[j * 8 + q] * rb[a][q];
          const size_t ip = (size_t)((j * 3 + a) * 2 + 0) * S + g, im = (size_t)((j * 3 + a) * 2 + 1) * S + g;
          const R yp = tyb[ip], ym = tyb[im];
          const R sp = yp > R(0) ? R(1) : (yp < R(0) ? R(-1) : R(0));
          const R sm = ym > R(0) ? R(1) : (ym < R(0) ? R(-1) : R(0));
          ybb[ip] -= rho * sc.s[1] * sp * gr;
          ybb[im] += rho * sc.s[1] * sm * gr;
          tbar += double(rho * (rabs(ym) - rabs(yp)) * ds1 * gr);
        }
    if (BALL && later)
      for (int j = 0; j < Mq; ++j) {
        R qv[3], h[3], jh[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          qv[a] = tqb[(size_t)(j * 3 + a) * S + g];
          R gr = R(0);
#pragma unroll
          for (int q = 0; q < NC; ++q) gr += tabQ[j * 8 + q] * rb[a][q];
          h[a] = rho * gr;
        }
        proj_jac(qv, sc.bo, sc.brad, h, jh);
#pragma unroll
        for (int a = 0; a < 3; ++a) qbb[(size_t)(j * 3 + a) * S + g] += R(2) * jh[a] - h[a];
      }
    if (VN && later)
      for (int j = 0; j < Mv; ++j) {
        R qv[3], ph[3], h[3], jh[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) qv[a] = tqv[(size_t)(j * 3 + a) * S + g];
        project_ball(qv, zero3, sc.vnorm, ph);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          R gr = R(0);
#pragma unroll
          for (int q = 0; q < NC; ++q) gr += tabV[j * 8 + q] * rb[a][q];
          h[a] = rho * sc.s[1] * gr;
          tbar += double(rho * ds1 * (R(2) * ph[a] - qv[a]) * gr);
        }
        proj_jac(qv, zero3, sc.vnorm, h, jh);
#pragma unroll
        for (int a = 0; a < 3; ++a) qvb[(size_t)(j * 3 + a) * S + g] += R(2) * jh[a] - h[a];
      }
    A.Tbar[g] += tbar;
  }
}

// after the last reverse step: fold the first local step's target adjoints,
// then the initial state (z^0 position rows = waypoints) feeds dP
template <class R>
__global__ void __launch_bounds__(256) adj_finish(const AdjArgs A, double *dwaypoints, double *ddurations) {
  const StreamArgs &F = A.f;
  R *zb = (R *)A.zb;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < F.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(F, x, t, b, i, N, g)) continue;
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    adj_fold<R>(A, b, g, first, last);
    for (int a = 0; a < 3; ++a) {
      double v = 0.0;
      if (!last) v = A.Pbar[(size_t)jE * 3 + a] + double(zb[(size_t)(a * ND) * F.Jn + jE]);
      dwaypoints[(size_t)jE * 3 + a] = v;
      if (first) dwaypoints[(size_t)jS * 3 + a] = 0.0;
    }
    ddurations[g] = A.Tbar[g];
  }
}

template <class R>
int run_adjoint_t(const StreamArgs &Fw, AdjArgs A, int fam, int ckpt, void *const *ck_base, void *const *tape_base,
                  const size_t *bytes, double *dwaypoints, double *ddurations, void *stream) {
  // ck_base[c*7 + q], tape_base[l*7 + q]: copies of (z, uL, uRp, uR0, ybox, qball, qvn) of bytes[q] bytes
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256;
  int blocks = (Fw.total + threads - 1) / threads;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  constexpr int NQ = 7;
  void *work[NQ] = {Fw.z, Fw.uL, Fw.uRp, Fw.uR0, Fw.ybox, Fw.qball, Fw.qvn};
  const DevProblem &p = Fw.p;
  const int Mb = (fam & FAM_BOX) ? p.M_box : 0, Mq = (fam & FAM_BALL) ? p.M_ball : 0,
            Mv = (fam & FAM_VN) ? p.M_vn : 0;
  const size_t tab_bytes = sizeof(R) * 8 * (size_t)(Mb + Mq + Mv);
  void (*init)(const StreamArgs) = nullptr;
  void (*local)(const StreamArgs, int) = nullptr;
  void (*seg_rows)(const AdjArgs, int, int) = nullptr;
  switch (fam) {
#define TOP_ADJ_CASE(FV) \
  case FV: init = stream_init<R, FV>; local = stream_local<R, FV>; seg_rows = adj_segment_rows<R, FV>; break;
    TOP_ADJ_CASE(0) TOP_ADJ_CASE(1) TOP_ADJ_CASE(2) TOP_ADJ_CASE(3)
    TOP_ADJ_CASE(4) TOP_ADJ_CASE(5) TOP_ADJ_CASE(6) TOP_ADJ_CASE(7)
#undef TOP_ADJ_CASE
    default: return (int)cudaErrorInvalidValue;
  }
  auto copy = [&](void *dst, const void *src, size_t n) -> int {
    if (n == 0) return 0;
    return (int)cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, st);
  };
  const int K = p.max_iters;
  init<<<blocks, threads, 0, st>>>(Fw);
  // forward with checkpoints of x^{c*ckpt}
  for (int k = 0; k < K; ++k) {
    if (k % ckpt == 0)
      for (int q = 0; q < NQ; ++q)
        if (copy(ck_base[(k / ckpt) * NQ + q], work[q], bytes[q])) return (int)cudaGetLastError();
    local<<<blocks, threads, tab_bytes, st>>>(Fw, k);
    stream_junction<R><<<blocks, threads, 0, st>>>(Fw, 0);
  }
  // reverse, block by block
  const int nblk = (K + ckpt - 1) / ckpt;
  for (int c = nblk - 1; c >= 0; --c) {
    const int k0 = c * ckpt, k1 = (k0 + ckpt < K) ? k0 + ckpt : K;
    for (int q = 0; q < NQ; ++q)
      if (copy(work[q], ck_base[c * NQ + q], bytes[q])) return (int)cudaGetLastError();
    for (int k = k0; k < k1; ++k) {
      for (int q = 0; q < NQ; ++q)
        if (copy(tape_base[(k - k0) * NQ + q], work[q], bytes[q])) return (int)cudaGetLastError();
      if (k + 1 < k1) {
        local<<<blocks, threads, tab_bytes, st>>>(Fw, k);
        stream_junction<R><<<blocks, threads, 0, st>>>(Fw, 0);
      }
    }
    for (int k = k1 - 1; k >= k0; --k) {
      void *const *tk = tape_base + (size_t)(k - k0) * NQ;
      A.tz = tk[0];
      A.tuL = tk[1];
      A.tuRp = tk[2];
      A.tuR0 = tk[3];
      A.tyb = tk[4];
      A.tqb = tk[5];
      A.tqv = tk[6];
      adj_junction<R><<<blocks, threads, 0, st>>>(A);
      if (fam == 0) adj_segment<R><<<blocks, threads, 0, st>>>(A, k == K - 1 ? 1 : 0);
      else seg_rows<<<blocks, threads, tab_bytes, st>>>(A, k == K - 1 ? 1 : 0, k);
    }
  }
  adj_finish<R><<<blocks, threads, 0, st>>>(A, dwaypoints, ddurations);
  return (int)cudaGetLastError();
}

}  // namespace top
