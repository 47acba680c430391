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
    stream_locate(F, x, t, b, i, N, g);
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
    stream_locate(F, x, t, b, i, N, g);
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

// after the last reverse step: fold the first local step's target adjoints,
// then the initial state (z^0 position rows = waypoints) feeds dP
template <class R>
__global__ void __launch_bounds__(256) adj_finish(const AdjArgs A, double *dwaypoints, double *ddurations) {
  const StreamArgs &F = A.f;
  R *zb = (R *)A.zb;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < F.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    stream_locate(F, x, t, b, i, N, g);
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
int run_adjoint_t(const StreamArgs &Fw, AdjArgs A, int ckpt, void *const *ck_base, void *const *tape_base,
                  const size_t *bytes, double *dwaypoints, double *ddurations, void *stream) {
  // ck_base[c*4 + q], tape_base[l*4 + q]: copies of (z, uL, uRp, uR0) arrays of `bytes[q]` bytes
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256;
  int blocks = (Fw.total + threads - 1) / threads;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  void *work[4] = {Fw.z, Fw.uL, Fw.uRp, Fw.uR0};
  const int K = Fw.p.max_iters;
  stream_init<R, 0><<<blocks, threads, 0, st>>>(Fw);
  // forward with checkpoints of x^{c*ckpt}
  for (int k = 0; k < K; ++k) {
    if (k % ckpt == 0)
      for (int q = 0; q < 4; ++q)
        if (cudaMemcpyAsync(ck_base[(k / ckpt) * 4 + q], work[q], bytes[q], cudaMemcpyDeviceToDevice, st))
          return (int)cudaGetLastError();
    stream_local<R, 0><<<blocks, threads, 0, st>>>(Fw, k);
    stream_junction<R><<<blocks, threads, 0, st>>>(Fw, 0);
  }
  // reverse, block by block
  const int nblk = (K + ckpt - 1) / ckpt;
  for (int c = nblk - 1; c >= 0; --c) {
    const int k0 = c * ckpt, k1 = (k0 + ckpt < K) ? k0 + ckpt : K;
    for (int q = 0; q < 4; ++q)
      if (cudaMemcpyAsync(work[q], ck_base[c * 4 + q], bytes[q], cudaMemcpyDeviceToDevice, st))
        return (int)cudaGetLastError();
    for (int k = k0; k < k1; ++k) {
      for (int q = 0; q < 4; ++q)
        if (cudaMemcpyAsync(tape_base[(k - k0) * 4 + q], work[q], bytes[q], cudaMemcpyDeviceToDevice, st))
          return (int)cudaGetLastError();
      if (k + 1 < k1) {
        stream_local<R, 0><<<blocks, threads, 0, st>>>(Fw, k);
        stream_junction<R><<<blocks, threads, 0, st>>>(Fw, 0);
      }
    }
    for (int k = k1 - 1; k >= k0; --k) {
      A.tz = tape_base[(k - k0) * 4 + 0];
      A.tuL = tape_base[(k - k0) * 4 + 1];
      A.tuRp = tape_base[(k - k0) * 4 + 2];
      A.tuR0 = tape_base[(k - k0) * 4 + 3];
      adj_junction<R><<<blocks, threads, 0, st>>>(A);
      adj_segment<R><<<blocks, threads, 0, st>>>(A, k == K - 1 ? 1 : 0);
    }
  }
  adj_finish<R><<<blocks, threads, 0, st>>>(A, dwaypoints, ddurations);
  return (int)cudaGetLastError();
}

}  // namespace top
