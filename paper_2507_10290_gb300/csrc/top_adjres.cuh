// top_adjres.cuh -- the resident adjoint of top_grad: one CTA per pack of
// whole trajectories runs the forward iterations, the checkpoints, the
// block-wise recomputation and the reverse sweep in a single launch, with the
// forward state and its adjoint in shared memory.  The paper has no gradient;
// this differentiates its closed-form iteration (Eq. 18a-c) without
// inequality rows, exactly as the resident kernel computes it.
//
// State (top_resident.cuh): per junction slot and row (axis a, order r) the
// consensus targets p (read by the right segment's local step) and m (read by
// the left segment's).  One iteration k:
//   local step   ch = G rho C(fs .* p_start, s .* m_end),  eS = fs .* ch,
//                eE = s .* (F ch)        (C, F the basis maps of top_math.cuh)
//   junction j   free rows:    p' = eE + (p - m)/2,  m' = eS_next - (p - m)/2
//                pinned rows:  p' = p + P - eS_next, m' = m + P - eE
//                end (r < 4):  m' = m + p - eE   (p holds the fixed end state)
//                start (r < 4): p' = p + m - eS  (m holds the fixed start state)
//   cost J = sum_i T_i^-7 ch_i^T Qh ch_i after the last local step.
// Reverse of iteration k, adjoint state (pb, mb) of x^{k+1} in, of x^k out:
//   A (slot owner): free rows   eEb = pb, eSb_next = mb, pb = -mb = (pb - mb)/2
//                   pinned rows eEb = -mb, eSb_next = -pb, Pbar += pb + mb
//                   end rows    eEb = -mb;  start rows  eSb = -pb
//   B (segment):   chb = C(fs .* eSb, s .* eEb) (+ 2 dJ T^-7 Qh ch at k = K-1),
//                  rb = G chb, pb[start] += rho fs .* rb, mb[end] += rho s .* (F rb),
//                  dJ/dT from s(T), G(T) = K(T)^-1 and the cost's T^-7.
// x^k comes from a tape in global memory, refilled block by block from
// checkpoints taken every `ckpt` iterations of the forward pass (the tape
// holds the slot state entering each iteration of the block).  At the end
// the initial state (position rows = waypoints) and the pinned rows give
// d/d(waypoints); the trajectory's first and last waypoints only enter
// through the boundary states and get zero.
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"
#include "top_step.cuh"

namespace top {

template <class R>
__device__ __forceinline__ void adjres_save(R *buf, size_t Jn, size_t jg, const R *p, const R *m) {
#pragma unroll
  for (int q = 0; q < NJ; ++q) {
    buf[(size_t)q * Jn + jg] = p[q];
    buf[(size_t)(NJ + q) * Jn + jg] = m[q];
  }
}

template <class R>
__device__ __forceinline__ void adjres_load(const R *buf, size_t Jn, size_t jg, R *p, R *m) {
#pragma unroll
  for (int q = 0; q < NJ; ++q) {
    p[q] = buf[(size_t)q * Jn + jg];
    m[q] = buf[(size_t)(NJ + q) * Jn + jg];
  }
}

template <class R>
__global__ void __launch_bounds__(256, 1) adjoint_resident_kernel(const AdjResArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevProblem &p = A.p;
  const Pack pk = A.packs[blockIdx.x];
  const int C = blockDim.x;
  const int l = threadIdx.x;
  const int ntp = A.ntp;
  const int J = C + ntp;
  const AdjResLayout L = adjres_layout(C, ntp, (int)sizeof(R));
  R *sp = (R *)(smem + L.p);
  R *sm = (R *)(smem + L.m);
  R *spb = (R *)(smem + L.pb);
  R *smb = (R *)(smem + L.mb);
  R *szP = (R *)(smem + L.zP);
  R *seS = (R *)(smem + L.eS);  // start derivatives (forward), their adjoints (reverse)
  int *soff = (int *)(smem + L.off);
  int *stid = (int *)(smem + L.tid);
  const R rho = R(p.rho);
  const int K = p.max_iters;
  const int ckpt = A.ckpt;
  const bool pin = (p.mode == 0);
  const size_t Jn = (size_t)A.Jn;
  R *ck = (R *)A.ck;
  R *tape = (R *)A.tape;
  const size_t state = (size_t)2 * NJ * Jn;  // one saved state: p and m of every slot

  // (the pack descriptor is block-uniform: a bad one ends the whole block)
  if (!TOP_IN_BOUNDS(p.err, pk.ntraj >= 1 && pk.ntraj <= ntp && pk.nseg >= 0 && pk.nseg <= C &&
                                pk.tlist >= 0 && pk.tlist + pk.ntraj <= p.B))
    return;
  for (int t = l; t < pk.ntraj; t += C) stid[t] = A.traj_list[pk.tlist + t];
  __syncthreads();
  if (l == 0) {
    int acc = 0;
    for (int t = 0; t < pk.ntraj; ++t) {
      soff[t] = acc;
      if (!TOP_IN_BOUNDS(p.err, stid[t] >= 0 && stid[t] < p.B)) { acc = -1; break; }
      acc += p.seg_offset[stid[t] + 1] - p.seg_offset[stid[t]];
    }
    soff[pk.ntraj] = acc;
  }
  for (int q = l; q < NJ * J; q += C) { sp[q] = R(0); sm[q] = R(0); spb[q] = R(0); smb[q] = R(0); }
  for (int q = l; q < 3 * J; q += C) szP[q] = R(0);
  __syncthreads();
  if (!TOP_IN_BOUNDS(p.err, soff[pk.ntraj] == pk.nseg)) return;

  const bool inside = l < pk.nseg;
  int tb = 0;
  if (inside) {
    int lo = 0, hi = pk.ntraj - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (soff[mid] <= l) lo = mid; else hi = mid - 1;
    }
    tb = lo;
  }
  const int i = l - soff[tb];
  const int Nb = soff[tb + 1] - soff[tb];
  const int b = stid[tb];
  const int g = p.seg_offset[b] + i;
  const bool valid = inside && TOP_IN_BOUNDS(p.err, i >= 0 && i < Nb && g >= 0 && g < p.S);
  const bool first = valid && i == 0;
  const bool last = valid && i == Nb - 1;
  const int jS = l + tb, jE = l + tb + 1;
  const size_t gS = (size_t)g + b, gE = (size_t)g + b + 1;  // global slot indices (the waypoint rows)
  R *pS = sp + jS * NJ, *mS = sm + jS * NJ, *pE = sp + jE * NJ, *mE = sm + jE * NJ;
  R *pbS = spb + jS * NJ, *mbS = smb + jS * NJ, *pbE = spb + jE * NJ, *mbE = smb + jE * NJ;
  const R *eSnext = seS + (l + 1) * NJ;

  R G[NG], s[NC], fs[ND];
  R Tq = R(1);
  if (valid) {
    const R *Gp = (const R *)A.G;
#pragma unroll
    for (int q = 0; q < NG; ++q) G[q] = Gp[(size_t)q * p.S + g];
    Tq = R(p.durations[g]);
    inv_powers(Tq, s);
  } else {
#pragma unroll
    for (int q = 0; q < NG; ++q) G[q] = R(0);
#pragma unroll
    for (int r = 0; r < NC; ++r) s[r] = R(r == 0);  // s_0 = 1 in every thread
  }
#pragma unroll
  for (int r = 0; r < ND; ++r) fs[r] = R(fact(r)) * s[r];
  // the local step's coefficients (Eq. 18a) from the start- and end-side targets of
  // the three axes (the resident kernel's maps: Taylor shift, packed pairs)
  auto local_coeffs = [&](const R *tS, size_t strS, const R *tE, size_t strE, R (&ch)[AX][NC]) {
    R wS[AX][ND], wE[AX][ND], rhs[AX][NC];
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        wS[a][r] = fs[r] * tS[(size_t)(a * ND + r) * strS];
        wE[a][r] = fs[r] * tE[(size_t)(a * ND + r) * strE];
      }
    consensus_rhs_shift(wS, wE, rho, rhs);
    apply_g3(G, rhs, ch);
  };

  // the initial state x^0 (Init of Algorithm 1), into the slots this thread owns
  auto init_state = [&]() {
    if (!valid) return;
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const int row = a * ND + r;
        if (!last) {
          const R P = (r == 0) ? R(p.waypoints[gE * 3 + a]) : R(0);
          pE[row] = P;
          mE[row] = P;
          if (r == 0) szP[jE * 3 + a] = P;
        } else {
          const R zN = (r < PO) ? R(p.end_state[((size_t)b * PO + r) * 3 + a]) : R(0);
          pE[row] = zN;
          mE[row] = zN;
        }
        if (first) {
          const R z0 = (r < PO) ? R(p.start_state[((size_t)b * PO + r) * 3 + a]) : R(0);
          pS[row] = z0;
          mS[row] = z0;
        }
      }
  };

  // one forward iteration (Eq. 18a-c); two barriers
  auto forward = [&]() {
    R eE[AX][ND], eSv[AX][ND];
    if (valid) {
      R ch[AX][NC];
      local_coeffs(pS, 1, mE, 1, ch);
      end_derivs_shift(ch, fs, eSv, eE);
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int r = 0; r < ND; ++r) seS[l * NJ + a * ND + r] = eSv[a][r];
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int r = 0; r < ND; ++r) {
          const int row = a * ND + r;
          if (!last) {
            const R ee = eE[a][r], en = eSnext[row];
            const R pv = pE[row], mv = mE[row];
            if (pin && r == 0) {
              const R P = szP[jE * 3 + a];
              mE[row] = mv + (P - ee);
              pE[row] = pv + (P - en);
            } else {
              const R uL = R(0.5) * (pv - mv);
              pE[row] = ee + uL;
              mE[row] = en - uL;
            }
          } else if (r < PO) {
            mE[row] += pE[row] - eE[a][r];
          }
          if (first && r < PO) pS[row] += mS[row] - eSv[a][r];
        }
    }
    __syncthreads();
  };

  auto save = [&](R *buf) {  // the slots this thread owns, into a saved state
    if (!valid) return;
    adjres_save(buf, Jn, gE, pE, mE);
    if (first) adjres_save(buf, Jn, gS, pS, mS);
  };

  // ---- forward pass with checkpoints of x^{c ckpt} ----
  const int nblk = (K + ckpt - 1) / ckpt;
  init_state();
  __syncthreads();
  for (int k = 0; k < (nblk - 1) * ckpt; ++k) {
    if (k % ckpt == 0) save(ck + (size_t)(k / ckpt) * state);
    forward();
  }
  if (nblk > 0) save(ck + (size_t)(nblk - 1) * state);

  // ---- reverse sweep, block by block ----
  double tbar = 0.0;          // dJ/dT of this segment
  double Pacc[3] = {0.0, 0.0, 0.0};  // dJ/dP of the junction this thread owns (pinned rows)
  for (int c = nblk - 1; c >= 0; --c) {
    const int k0 = c * ckpt, k1 = (k0 + ckpt < K) ? k0 + ckpt : K;
    __syncthreads();
    if (valid) {
      adjres_load(ck + (size_t)c * state, Jn, gE, pE, mE);
      if (first) adjres_load(ck + (size_t)c * state, Jn, gS, pS, mS);
    }
    __syncthreads();
    for (int k = k0; k < k1; ++k) {  // recompute the block into the tape
      save(tape + (size_t)(k - k0) * state);
      if (k + 1 < k1) forward();
    }
    __syncthreads();
    for (int k = k1 - 1; k >= k0; --k) {
      // ---- A. reverse of the junction update of iteration k (the slots this thread owns) ----
      R eEb[AX][ND];
      if (valid) {
        R *eSbn = seS + (l + 1) * NJ, *eSbo = seS + l * NJ;
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int r = 0; r < ND; ++r) {
            const int row = a * ND + r;
            const R pb = pbE[row], mb = mbE[row];
            if (!last) {
              if (pin && r == 0) {
                eEb[a][r] = -mb;
                eSbn[row] = -pb;
                Pacc[a] += double(pb) + double(mb);
              } else {
                const R h = R(0.5) * (pb - mb);
                eEb[a][r] = pb;
                eSbn[row] = mb;
                pbE[row] = h;
                mbE[row] = -h;
              }
            } else {
              eEb[a][r] = (r < PO) ? -mb : R(0);
              pbE[row] = R(0);
            }
            if (first) {
              eSbo[row] = (r < PO) ? -pbS[row] : R(0);
              mbS[row] = R(0);
            }
          }
      }
      __syncthreads();
      // ---- B. reverse of the local step of iteration k ----
      if (valid) {
        const R *tk = tape + (size_t)(k - k0) * state;
        const R *eSb = seS + l * NJ;
        R tb_k = R(0);  // this iteration's dJ/dT terms, in the iteration precision
        const R iT = s[1];
        // the iteration's coefficients, re-formed from the taped targets
        R ch[AX][NC];
        local_coeffs(tk + gS, Jn, tk + (size_t)NJ * Jn + gE, Jn, ch);
        // the adjoint of the end derivatives e = s .* (M ch) with respect to ch (the
        // transposed map takes r! s_r times the adjoints)
        R xS[AX][ND], xE[AX][ND];
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int r = 0; r < ND; ++r) {
            xS[a][r] = fs[r] * eSb[a * ND + r];
            xE[a][r] = fs[r] * eEb[a][r];
          }
        R chb[AX][NC];
        consensus_rhs_shift(xS, xE, R(1), chb);
        if (k == K - 1) {  // the cost seed: J = T^-7 ch^T Qh ch
          const double dj = A.dJ[b];
          const double t7 = double(s[7]);
#pragma unroll
          for (int a = 0; a < AX; ++a) {
            double cqc = 0.0;
#pragma unroll
            for (int k1q = PO; k1q < NC; ++k1q) {
              double acc = 0.0;
#pragma unroll
              for (int k2 = PO; k2 < NC; ++k2) acc += qhat(k1q, k2) * double(ch[a][k2]);
              chb[a][k1q] += R(dj * 2.0 * t7 * acc);
              cqc += double(ch[a][k1q]) * acc;
            }
            tbar += dj * (-7.0) * t7 / double(Tq) * cqc;
          }
        }
        R rb[AX][NC];
        apply_g3(G, chb, rb);
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          // M ch and M rb without the s_r factors: start rows r! x_r, end rows r! (x shifted by one)_r
          R mcE[NC], mrb[NC];
#pragma unroll
          for (int q = 0; q < NC; ++q) { mcE[q] = ch[a][q]; mrb[q] = rb[a][q]; }
          taylor_shift(mcE);
          taylor_shift(mrb);
          // e = s .* (M ch): the s_r(T) factors
#pragma unroll
          for (int r = 0; r < ND; ++r)
            tb_k += (eSb[a * ND + r] * (R(fact(r)) * ch[a][r]) + eEb[a][r] * (R(fact(r)) * mcE[r])) *
                    (-R(r) * s[r] * iT);
          // G(T) = K(T)^-1:  -rb^T K'(T) ch,  K' = -14 T^-8 Qh + rho sum_r (-2 r s_r^2 / T) (rows of M)
          R rqc = R(0);
#pragma unroll
          for (int k1q = PO; k1q < NC; ++k1q) {
            R acc = R(0);
#pragma unroll
            for (int k2 = PO; k2 < NC; ++k2) acc += R(qhat(k1q, k2)) * ch[a][k2];
            rqc += rb[a][k1q] * acc;
          }
          R kp = R(-14) * s[7] * iT * rqc;
#pragma unroll
          for (int r = 1; r < ND; ++r) {
            const R c2 = R(-2 * r) * s[r] * s[r] * iT;
            const R fr = R(fact(r));
            if (!(first && r >= PO)) kp += rho * c2 * (fr * rb[a][r]) * (fr * ch[a][r]);
            if (!(last && r >= PO)) kp += rho * c2 * (fr * mrb[r]) * (fr * mcE[r]);
          }
          tb_k -= kp;
          // the targets: w = s .* (rho M rb) (masked rows are constants)
#pragma unroll
          for (int r = 0; r < ND; ++r) {
            const R fr = R(fact(r));
            R obS = rho * fr * rb[a][r];
            R obE = rho * fr * mrb[r];
            if (first && r >= PO) obS = R(0);
            if (last && r >= PO) obE = R(0);
            const R w0 = tk[(size_t)(a * ND + r) * Jn + gS];       // p at the start slot
            const R w1 = tk[(size_t)(NJ + a * ND + r) * Jn + gE];  // m at the end slot
            tb_k += (obS * w0 + obE * w1) * (-R(r) * s[r] * iT);
            pbS[a * ND + r] += s[r] * obS;
            mbE[a * ND + r] += s[r] * obE;
          }
        }
        tbar += double(tb_k);
      }
      __syncthreads();
    }
  }

  // ---- outputs: dJ/dT, dJ/dP (initial position rows and pinned rows) ----
  if (valid) {
    A.dT[g] = tbar;
    if (!last)
#pragma unroll
      for (int a = 0; a < AX; ++a) A.dw[gE * 3 + a] = Pacc[a] + double(pbE[a * ND]) + double(mbE[a * ND]);
  }
}

template <class R>
int launch_adjres_t(const AdjResArgs &a, int nblocks, int C, size_t smem, void *stream) {
  auto kern = adjoint_resident_kernel<R>;
  cudaError_t e = func_attr_once((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<nblocks, C, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace top
