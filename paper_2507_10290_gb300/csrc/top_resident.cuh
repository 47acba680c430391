// top_resident.cuh -- the resident CADMM kernel: one CTA per pack of whole
// trajectories, one thread per segment, all iteration state in shared memory
// for the whole run (Algorithm 1 of the paper, Eq. 18a-g, 19-21).
//
// Per iteration and segment i (thread i of its pack):
//   1. local step (Eq. 18a, 18d-g): targets w = E (z - u) at both ends, the
//      shared local_step() solves with G and advances the constraint state
//   2. publish the start-end derivatives; barrier
//   3. junction i+1 (owned by thread i): consensus average (Eq. 18b, pinned
//      position rows kept at the waypoint), scaled duals (Eq. 18c), primal
//      residual contribution (Eq. 19); barrier
//   4. on check iterations: dual residual contribution (Eq. 20), per-
//      trajectory FP64 reductions in a fixed order, stopping test (Eq. 21)
// Junction state per slot: z[21], uL[21] (u of the left segment's end side),
// uRp[3] (u of the right segment's start side on pinned position rows); on
// free rows the right side's u equals -uL (the averaging keeps the pair
// summing to zero), and each trajectory's start junction keeps its own
// start-side u for orders 0..3 (uR0).
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"
#include "top_step.cuh"

namespace top {

template <class R, int F>
__global__ void __launch_bounds__(512, 1) resident_kernel(const ResidentArgs A) {
  constexpr bool BOX = (F & FAM_BOX) != 0;
  constexpr bool BALL = (F & FAM_BALL) != 0;
  constexpr bool VN = (F & FAM_VN) != 0;
  extern __shared__ __align__(16) unsigned char smem[];
  const DevProblem &p = A.p;
  const DevResult &res = A.r;
  const Pack pk = A.packs[blockIdx.x];
  const int C = blockDim.x;
  const int l = threadIdx.x;
  const int ntp = A.ntp;
  const int J = C + ntp;
  const int Mb = BOX ? p.M_box : 0, Mq = BALL ? p.M_ball : 0, Mv = VN ? p.M_vn : 0;
  const ResLayout L = res_layout(C, ntp, Mb, Mq, Mv, (int)sizeof(R));
  double *red_rp = (double *)(smem + L.red_rp);
  double *red_rd = (double *)(smem + L.red_rd);
  double *tr_rp = (double *)(smem + L.tr_rp);
  double *tr_rd = (double *)(smem + L.tr_rd);
  R *sz = (R *)(smem + L.z);
  R *suL = (R *)(smem + L.uL);
  R *suRp = (R *)(smem + L.uRp);
  R *seS = (R *)(smem + L.eS);
  R *sdz = (R *)(smem + L.dz);
  R *sybox = (R *)(smem + L.ybox);
  R *sqball = (R *)(smem + L.qball);
  R *sqvn = (R *)(smem + L.qvn);
  R *suR0 = (R *)(smem + L.uR0);
  R *tabB = (R *)(smem + L.tabB);
  R *tabQ = (R *)(smem + L.tabQ);
  R *tabV = (R *)(smem + L.tabV);
  int *soff = (int *)(smem + L.off);
  int *sdone = (int *)(smem + L.done);

  const R rho = R(p.rho);
  const int K = p.max_iters;
  const bool pin = (p.mode == 0);

  // ---- set-up: pack offsets, sample tables, zeroed state ----
  for (int t = l; t <= pk.ntraj; t += C) soff[t] = p.seg_offset[pk.traj0 + t] - pk.seg0;
  for (int t = l; t < ntp; t += C) { tr_rp[t] = 0.0; tr_rd[t] = 0.0; }
  for (int q = l; q < 12 * ntp; q += C) suR0[q] = R(0);
  for (int q = l; q < 21 * J; q += C) { sdz[q] = R(0); sz[q] = R(0); suL[q] = R(0); }
  for (int q = l; q < 3 * J; q += C) suRp[q] = R(0);
  if (BOX) for (int q = l; q < 6 * Mb * C; q += C) sybox[q] = R(0);
  if (BALL) for (int q = l; q < 3 * Mq * C; q += C) sqball[q] = R(0);
  if (VN) for (int q = l; q < 3 * Mv * C; q += C) sqvn[q] = R(0);
  if (BOX) fill_sample_table(tabB, Mb, 1, l, C);
  if (BALL) fill_sample_table(tabQ, Mq, 0, l, C);
  if (VN) fill_sample_table(tabV, Mv, 1, l, C);
  __syncthreads();
  for (int t = l; t < pk.ntraj; t += C) sdone[t] = (soff[t + 1] == soff[t]) ? 1 : 0;

  const bool valid = l < pk.nseg;
  int tb = 0;
  if (valid) {
    int lo = 0, hi = pk.ntraj - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (soff[mid] <= l) lo = mid; else hi = mid - 1;
    }
    tb = lo;
  }
  const int i = l - soff[tb];
  const int Nb = soff[tb + 1] - soff[tb];
  const bool first = valid && i == 0;
  const bool last = valid && i == Nb - 1;
  const int b = pk.traj0 + tb;
  const int g = pk.seg0 + l;
  const int jS = l + tb, jE = l + tb + 1;
  const int wrow0 = pk.seg0 + pk.traj0;

  SegConst<R> sc;
  R Tq = R(1);
  sc.vbox = sc.vnorm = sc.brad = R(0);
  sc.bo[0] = sc.bo[1] = sc.bo[2] = R(0);
  if (valid) {
    const R *Gp = (const R *)A.G;
#pragma unroll
    for (int q = 0; q < NG; ++q) sc.G[q] = Gp[(size_t)q * p.S + g];
    Tq = R(p.durations[g]);
    inv_powers(Tq, sc.s);
    if (BOX) sc.vbox = R(p.vbox[b]);
    if (VN) sc.vnorm = R(p.vnorm[b]);
    if (BALL) {
      sc.brad = R(p.ball_r[g]);
      for (int a = 0; a < 3; ++a) sc.bo[a] = R(p.ball_c[(size_t)g * 3 + a]);
    }
    // junction state (Init of Algorithm 1): positions from the path, other
    // orders zero, the trajectory's ends from the boundary states
    for (int a = 0; a < AX; ++a)
      for (int r = 0; r < ND; ++r) {
        R zv = R(0);
        if (!last) {
          if (r == 0) zv = R(p.waypoints[(size_t)(wrow0 + jE) * 3 + a]);
        } else if (r < PO) {
          zv = R(p.end_state[((size_t)b * PO + r) * 3 + a]);
        }
        sz[(a * ND + r) * J + jE] = zv;
        if (first) sz[(a * ND + r) * J + jS] = r < PO ? R(p.start_state[((size_t)b * PO + r) * 3 + a]) : R(0);
      }
  } else {
#pragma unroll
    for (int q = 0; q < NG; ++q) sc.G[q] = R(0);
#pragma unroll
    for (int r = 0; r < NC; ++r) sc.s[r] = R(0);
  }
  __syncthreads();

  R ch[AX][NC];
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) ch[a][k] = R(0);

  const int cev = p.check_every > 0 ? p.check_every : 1;
  const bool periodic = p.eps > 0.0 || res.history != nullptr;
  for (int k = 0; k < K; ++k) {
    const bool check = (k == K - 1) || (periodic && ((k + 1) % cev == 0));
    const bool act = valid && !sdone[tb];
    R eE[AX][ND];
    R eSv[AX][ND];
    if (act) {
      // ---- 1. local step (Eq. 18a, 18d-g) ----
      R wS[AX][ND], wE[AX][ND];
#pragma unroll
      for (int a = 0; a < AX; ++a) {
#pragma unroll
        for (int r = 0; r < ND; ++r) {
          const int row = (a * ND + r) * J;
          R us;
          if (first) us = (r < PO) ? suR0[(a * PO + r) * ntp + tb] : R(0);
          else if (pin && r == 0) us = suRp[a * J + jS];
          else us = -suL[row + jS];
          wS[a][r] = (first && r >= PO) ? R(0) : sc.s[r] * (sz[row + jS] - us);
          wE[a][r] = (last && r >= PO) ? R(0) : sc.s[r] * (sz[row + jE] - suL[row + jE]);
        }
      }
      local_step<R, F>(sc, wS, wE, rho, k == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV, Mb, Mq,
                       Mv, ch);
      // ---- 2. publish start derivatives ----
#pragma unroll
      for (int a = 0; a < AX; ++a) {
        end_derivs(ch[a], sc.s, eSv[a], eE[a]);
#pragma unroll
        for (int r = 0; r < ND; ++r) seS[(a * ND + r) * C + l] = eSv[a][r];
      }
    }
    __syncthreads();
    // ---- 3. junction update (Eq. 18b, 18c) and primal residual (Eq. 19) ----
    R rp2 = R(0);  // this segment's share of ||r_p||^2, only formed on check iterations
    if (act) {
#pragma unroll
      for (int a = 0; a < AX; ++a) {
#pragma unroll
        for (int r = 0; r < ND; ++r) {
          const int idx = (a * ND + r) * J + jE;
          if (!last) {
            const R en = seS[(a * ND + r) * C + l + 1];
            if (check) {
              const R gap = eE[a][r] - en;
              rp2 += gap * gap;
            }
            if (pin && r == 0) {
              const R P = sz[idx];
              suL[idx] += eE[a][r] - P;
              suRp[a * J + jE] += en - P;
              if (check) sdz[idx] = R(0);
            } else {
              const R zo = sz[idx];
              const R zn = R(0.5) * (eE[a][r] + en);
              suL[idx] += eE[a][r] - zn;
              sz[idx] = zn;
              if (check) sdz[idx] = zn - zo;
            }
          } else if (r < PO) {
            suL[idx] += eE[a][r] - sz[idx];
          }
          if (first && r < PO) suR0[(a * PO + r) * ntp + tb] += eSv[a][r] - sz[(a * ND + r) * J + jS];
        }
      }
    }
    __syncthreads();
    if (check) {
      // ---- 4. dual residual (Eq. 20), reductions, stopping rule (Eq. 21) ----
      double rd2 = 0.0;
      if (act) {
        R Tk[NC];
        Tk[0] = R(1);
#pragma unroll
        for (int q = 1; q < NC; ++q) Tk[q] = Tk[q - 1] * Tq;
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          R dS[ND], dE[ND];
#pragma unroll
          for (int r = 0; r < ND; ++r) {
            dS[r] = first ? R(0) : sc.s[r] * sdz[(a * ND + r) * J + jS];
            dE[r] = last ? R(0) : sc.s[r] * sdz[(a * ND + r) * J + jE];
          }
          rd2 += dual_residual_sq(dS, dE, rho, Tk);
        }
      }
      red_rp[l] = double(rp2);
      red_rd[l] = rd2;
      __syncthreads();
      const int warp = l >> 5, lane = l & 31, nw = C >> 5;
      for (int t = warp; t < pk.ntraj; t += nw) {
        if (sdone[t]) continue;
        double a1 = 0.0, a2 = 0.0;
        for (int x = soff[t] + lane; x < soff[t + 1]; x += 32) { a1 += red_rp[x]; a2 += red_rd[x]; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a1 += __shfl_xor_sync(0xffffffffu, a1, o);
          a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
          const double rp = sqrt(a1), rd = sqrt(a2);
          tr_rp[t] = rp;
          tr_rd[t] = rd;
          const int bb = pk.traj0 + t;
          if (res.history) {
            res.history[((size_t)k * p.B + bb) * 2 + 0] = rp;
            res.history[((size_t)k * p.B + bb) * 2 + 1] = rd;
          }
          const double tol = double(soff[t + 1] - soff[t]) * p.eps;
          int st = -1;
          if (!finite_d(rp) || !finite_d(rd)) st = 2;
          else if (p.eps > 0.0 && rp < tol && rd < tol) st = 0;
          if (st >= 0) {
            sdone[t] = 1;
            res.iters[bb] = k + 1;
            res.status[bb] = st;
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- outputs: coefficients in the paper's basis, FP64 cost per trajectory ----
  double Ji = 0.0;
  if (valid) {
    const double T = p.durations[g];
    double sd[NC];
    sd[0] = 1.0;
    for (int q = 1; q < NC; ++q) sd[q] = sd[q - 1] / T;
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) res.coeffs[((size_t)g * AX + a) * NC + q] = double(ch[a][q]) * sd[q];
    Ji = segment_cost(ch, sd[7]);
  }
  red_rp[l] = Ji;
  __syncthreads();
  {
    const int warp = l >> 5, lane = l & 31, nw = C >> 5;
    for (int t = warp; t < pk.ntraj; t += nw) {
      double a1 = 0.0;
      for (int x = soff[t] + lane; x < soff[t + 1]; x += 32) a1 += red_rp[x];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      if (lane == 0) {
        const int bb = pk.traj0 + t;
        res.cost[bb] = a1;
        res.r_primal[bb] = tr_rp[t];
        res.r_dual[bb] = tr_rd[t];
        const bool empty = soff[t + 1] == soff[t];
        if (empty) {
          res.iters[bb] = 0;
          res.status[bb] = 0;
        } else if (!sdone[t]) {
          res.iters[bb] = K;
          res.status[bb] = 1;
        }
      }
    }
  }
}

template <class R>
int launch_resident_t(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
#define TOP_RES_CASE(FV)                                                                               \
  case FV: {                                                                                           \
    auto kern = resident_kernel<R, FV>;                                                                \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return (int)e;                                                               \
    kern<<<nblocks, C, smem, st>>>(a);                                                                 \
    return (int)cudaGetLastError();                                                                    \
  }
  switch (fam) {
    TOP_RES_CASE(0)
    TOP_RES_CASE(1)
    TOP_RES_CASE(2)
    TOP_RES_CASE(3)
    TOP_RES_CASE(4)
    TOP_RES_CASE(5)
    TOP_RES_CASE(6)
    TOP_RES_CASE(7)
    default: return (int)cudaErrorInvalidValue;
  }
#undef TOP_RES_CASE
}

}  // namespace top
