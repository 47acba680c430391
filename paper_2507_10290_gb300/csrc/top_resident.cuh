// top_resident.cuh -- the resident CADMM kernel: one CTA per pack of whole
// trajectories, one thread per segment, all iteration state in shared memory
// for the whole run (Algorithm 1 of the paper, Eq. 18a-g, 19-21).
//
// Junction state.  For every junction slot and row (axis a, order r) the
// kernel keeps the two consensus targets the adjacent segments read in the
// local step of Eq. 18a, instead of z and u themselves:
//   p = z - u(start side of the right segment),  m = z - u(end side of the left segment).
// On free interior rows the two scaled duals sum to zero (the average of
// Eq. 18b makes the increments opposite), so with uL = u(end side):
//   p = z + uL,  m = z - uL,   z = (p + m)/2,  uL = (p - m)/2,
// and the updates of Eq. 18b-c become  p' = eE + uL,  m' = eS_next - uL.
// Rows whose z is fixed keep the fixed value in the slot no neighbour reads:
//   pinned interior positions (PIN mode): zP[slot][a] = waypoint;
//     m' = m + P - eE,  p' = p + P - eS_next
//   trajectory end (orders < p):   p = z_N (fixed),  m' = m + z_N - eE
//   trajectory start (orders < p): m = z_0 (fixed),  p' = p + z_0 - eS
//   orders >= p at the two ends: p = m = 0 (those consensus rows are dropped).
// The local step then reads p at its start slot and m at its end slot,
// 42 values, with every special case already encoded.
//
// Per iteration and segment i (thread i of its pack):
//   1. local step (Eq. 18a, 18d-g) from s_r p[start], s_r m[end]
//   2. publish the start derivatives; barrier
//   3. junction i+1 (owned by thread i): consensus update, primal-residual
//      share (Eq. 19) on check iterations; barrier
//   4. on check iterations: dual residual (Eq. 20), per-trajectory FP64
//      reductions of the segments' shares in a fixed order, stopping test
//      (Eq. 21), and with adaptive rho the update of Eq. 22; barrier
//   5. after a change of rho (adaptive rho only): the thread's own junction
//      targets, slack duals and projection states rescaled, its local inverse
//      rebuilt for the new rho; barrier
// Shared arrays are slot-major (21 values per slot): every access of a
// thread is a constant offset from one base, and consecutive threads are 21
// words apart (no bank conflicts).
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"
#include "top_step.cuh"
#include "top_tc.cuh"

namespace top {

// FP64 state needs twice the registers: 256 threads per CTA (255 registers each) in FP64
// TC: the G product of a warp whose 32 segments share one inverse runs on the
// tensor cores (top_tc.cuh); FP32, no inequality rows, fixed rho only.
// STALL: the stall rule (top_problem.stall_checks) is compiled in; a separate
// instance (top_resident_stall_*.cu), since even unused its code changes the
// code generation of the iteration loop (3 % on the 4096-trajectory batch).
template <class R, int F, bool ADAPT, bool TC = false, bool STALL = false>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512, 1) resident_kernel(const ResidentArgs A) {
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
  const ResLayout L = res_layout_resident(C, ntp, Mb, Mq, Mv, (int)sizeof(R), TC);
  double *red_rp = (double *)(smem + L.red_rp);  // FP64 cost shares (epilogue)
  R *sh_rp = (R *)(smem + L.red_rp);              // residual shares (check iterations)
  R *sh_rd = (R *)(smem + L.red_rd);
  double *tr_rp = (double *)(smem + L.tr_rp);
  double *tr_rd = (double *)(smem + L.tr_rd);
  R *sp = (R *)(smem + L.p);
  R *sm = (R *)(smem + L.m);
  R *szP = (R *)(smem + L.zP);
  R *seS = (R *)(smem + L.eS);
  R *sdz = (R *)(smem + L.dz);
  R *sybox = (R *)(smem + L.ybox);
  R *sqball = (R *)(smem + L.qball);
  R *sqvn = (R *)(smem + L.qvn);
  R *tabB = (R *)(smem + L.tabB);
  R *tabQ = (R *)(smem + L.tabQ);
  R *tabV = (R *)(smem + L.tabV);
  R *sch = (R *)(smem + L.ch);  // coefficients of the last check iteration (the output)
  // element q of segment l's coefficients in ch: [24][C], or [C][28] with TC
  auto chx = [C](int q, int seg) { return TC ? seg * kTcRow + q : q * C + seg; };
  int *soff = (int *)(smem + L.off);
  int *sdone = (int *)(smem + L.done);
  int *stid = (int *)(smem + L.tid);
  int *sflag = (int *)(smem + L.flag);
  int *sndone = (int *)(smem + L.ndone);  // trajectories of the pack that have stopped
  double *srho = (double *)(smem + L.rho);  // per-trajectory rho (Eq. 22)
  double *sfac = (double *)(smem + L.fac);  // rho_old / rho_new of the last update

  const R rho0 = R(p.rho);
  constexpr bool adapt = ADAPT;  // residual balancing of rho (Eq. 22); A.E is non-null
  const int K = p.max_iters;
  const bool pin = (p.mode == 0);

  // ---- set-up: the pack's trajectories, local offsets, tables, zeroed state ----
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
  for (int t = l; t < ntp; t += C) {
    tr_rp[t] = 0.0; tr_rd[t] = 0.0; srho[t] = p.rho; sfac[t] = 1.0;
  }
  if (l == 0) { *sflag = 0; *sndone = 0; }
  for (int q = l; q < NJ * J; q += C) { sdz[q] = R(0); sp[q] = R(0); }
  for (int q = l; q < NJ * ntp; q += C) sm[q] = R(0);
  for (int q = l; q < 24 * C; q += C) sch[q] = R(0);
  for (int q = l; q < 3 * J; q += C) szP[q] = R(0);
  if (BOX) for (int q = l; q < 6 * Mb * C; q += C) sybox[q] = R(0);
  if (BALL) for (int q = l; q < 3 * Mq * C; q += C) sqball[q] = R(0);
  if (VN) for (int q = l; q < 3 * Mv * C; q += C) sqvn[q] = R(0);
  if (BOX) fill_sample_table(tabB, Mb, 1, l, C);
  if (BALL) fill_sample_table(tabQ, Mq, 0, l, C);
  if (VN) fill_sample_table(tabV, Mv, 1, l, C);
  __syncthreads();
  // the trajectories' segments fill the pack exactly (else the whole block ends)
  if (!TOP_IN_BOUNDS(p.err, soff[pk.ntraj] == pk.nseg)) return;
  for (int t = l; t < pk.ntraj; t += C) {
    sdone[t] = (soff[t + 1] == soff[t]) ? 1 : 0;
    if (sdone[t]) atomicAdd(sndone, 1);
  }
  // stall-rule state of the pack's trajectories (global memory: read and written by the lane
  // that reduces the trajectory's residuals, on check iterations only)
  if (STALL && A.stall && p.stall > 0)
    for (int t = l; t < pk.ntraj; t += C) {
      double *sb = A.stall + 3 * (size_t)stid[t];
      sb[0] = sb[1] = 1e300;
      sb[2] = 0.0;
    }

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
  const int g = p.seg_offset[b] + i;        // global segment
  const bool valid = inside && TOP_IN_BOUNDS(p.err, i >= 0 && i < Nb && g >= 0 && g < p.S);
  const bool first = valid && i == 0;
  const bool last = valid && i == Nb - 1;
  const int jS = l + tb, jE = l + tb + 1;   // junction slots in shared memory
  R *pS = sp + jS * NJ, *mS = sm + tb * NJ;  // start slot (m only at a trajectory's start: [trajectory][21])
  R *pE = sp + jE * NJ;                      // end slot (owned by this thread)
  // m at the end slot is read and written by this thread alone (its local step
  // and its junction update): it lives in registers, not in shared memory
  R mE[NJ];
#pragma unroll
  for (int q = 0; q < NJ; ++q) mE[q] = R(0);
  const R *eSnext = seS + (l + 1) * NJ;

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
    // Init of Algorithm 1: z position rows from the path, other orders zero,
    // the trajectory's two ends from the boundary states, every u zero
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const int row = a * ND + r;
        if (!last) {
          const R P = (r == 0) ? R(p.waypoints[(size_t)(g + b + 1) * 3 + a]) : R(0);
          pE[row] = P;
          mE[row] = P;
          if (r == 0) szP[jE * 3 + a] = P;
        } else if (r < PO) {
          const R zN = R(p.end_state[((size_t)b * PO + r) * 3 + a]);
          pE[row] = zN;
          mE[row] = zN;
        }
        if (first && r < PO) {
          const R z0 = R(p.start_state[((size_t)b * PO + r) * 3 + a]);
          pS[row] = z0;
          mS[row] = z0;
        }
      }
    if (A.from.p) {  // resume (top_resume): the exported targets and row states replace Init
      const size_t oE = (size_t)(g + b + 1) * NJ, oS = (size_t)(g + b) * NJ;
#pragma unroll
      for (int q = 0; q < NJ; ++q) {
        pE[q] = R(A.from.p[oE + q]);
        mE[q] = R(A.from.m[oE + q]);
        if (first) {
          pS[q] = R(A.from.p[oS + q]);
          mS[q] = R(A.from.m[oS + q]);
        }
      }
      if (BOX) for (int q = 0; q < 6 * Mb; ++q) sybox[q * C + l] = R(A.from.ybox[(size_t)g * 6 * Mb + q]);
      if (BALL) for (int q = 0; q < 3 * Mq; ++q) sqball[q * C + l] = R(A.from.qball[(size_t)g * 3 * Mq + q]);
      if (VN) for (int q = 0; q < 3 * Mv; ++q) sqvn[q * C + l] = R(A.from.qvn[(size_t)g * 3 * Mv + q]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < NG; ++q) sc.G[q] = R(0);
#pragma unroll
    for (int r = 0; r < NC; ++r) sc.s[r] = R(r == 0);  // s_0 = 1 in every thread
  }
  __syncthreads();
  // tensor-core form: does this warp's every segment hold the same inverse?
  bool wtc = false;
  TcA tca{};
  if constexpr (TC) {
    bool same = valid;
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      const R g0 = __shfl_sync(0xffffffffu, sc.G[q], 0);
      same = same && (sc.G[q] == g0);
    }
    wtc = __all_sync(0xffffffffu, same);
    if (wtc) tca = tc_a_fragments((const float *)A.G + g, (size_t)p.S, l & 31);
  }
  R fs[ND];  // r! T^-r
#pragma unroll
  for (int r = 0; r < ND; ++r) fs[r] = R(fact(r)) * sc.s[r];


  const int cev = p.check_every > 0 ? p.check_every : 1;
  const bool periodic = p.eps > 0.0 || res.history != nullptr;
  R rho = rho0;  // this trajectory's rho (changes only with adaptive rho, step 5)
  const int k0 = (A.from.p && valid) ? A.from.iters[b] : 0;  // iterations run before a resume
  for (int k = 0; k < K; ++k) {
    const bool check = adapt || (k == K - 1) || (periodic && ((k + 1) % cev == 0));
    const bool act = valid && !sdone[tb];
    bool tcw = false;  // the whole warp takes the tensor-core product this iteration
    if constexpr (TC) tcw = wtc && __all_sync(0xffffffffu, act);
    R eE[AX][ND];
    R eSv[AX][ND];
    if (act) {
      R ch[AX][NC];
      // ---- 1. local step (Eq. 18a, 18d-g) ----
      R wS[AX][ND], wE[AX][ND];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        if (r == 0) {  // fs_0 = 1
#pragma unroll
          for (int a = 0; a < AX; ++a) {
            wS[a][0] = pS[a * ND];
            wE[a][0] = mE[a * ND];
          }
          continue;
        }
        using V = typename Vec2<R>::T;
        const V f2 = mk2(fs[r], fs[r]);
        const V s01 = vmul(f2, mk2(pS[r], pS[ND + r]));
        const V e01 = vmul(f2, mk2(mE[r], mE[ND + r]));
        wS[0][r] = s01.x;
        wS[1][r] = s01.y;
        wS[2][r] = fs[r] * pS[2 * ND + r];
        wE[0][r] = e01.x;
        wE[1][r] = e01.y;
        wE[2][r] = fs[r] * mE[2 * ND + r];
      }
      if constexpr (TC) {
        R rhs[AX][NC];
        family_rhs<R, F, true>(sc, wS, wE, rho, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV,
                               Mb, Mq, Mv, rhs);
        if (tcw) apply_g_mma(tca, rhs, ch, sch + (l & ~31) * kTcRow, l & 31);
        else apply_g3(sc.G, rhs, ch);
      } else {
        local_step<R, F, true>(sc, wS, wE, rho, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV, Mb,
                               Mq, Mv, ch);
      }
      // ---- 2. publish start derivatives ----
      end_derivs_shift(ch, fs, eSv, eE);
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int r = 0; r < ND; ++r) seS[l * NJ + a * ND + r] = eSv[a][r];
      // the start slot of a trajectory's first segment has no other reader: its
      // dual update (Eq. 18c against the fixed start state) needs no barrier
      if (first) {
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int r = 0; r < PO; ++r) {
            const int row = a * ND + r;
            pS[row] += mS[row] - eSv[a][r];
          }
      }
      // a check iteration may be a trajectory's last: keep its coefficients
      if (check) {
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int q = 0; q < NC; ++q) sch[chx(a * NC + q, l)] = ch[a][q];
      }
    }
    __syncthreads();
    // ---- 3. junction update (Eq. 18b, 18c) and primal residual (Eq. 19) ----
    R rp2 = R(0);  // this segment's share of ||r_p||^2, formed on check iterations only
    if (act) {
      if (!last) {
        if (check) {  // residual share and consensus change, from the values before the update
#pragma unroll
          for (int a = 0; a < AX; ++a) {
#pragma unroll
            for (int r = 0; r < ND; ++r) {
              const int row = a * ND + r;
              const R ee = eE[a][r], en = eSnext[row];
              const R gap = ee - en;
              rp2 += gap * gap;
              sdz[jE * NJ + row] = (pin && r == 0) ? R(0) : R(0.5) * ((ee + en) - (pE[row] + mE[row]));
            }
          }
        }
#pragma unroll
        for (int r = 0; r < ND; ++r) {
          if (pin && r == 0) {  // pinned position: z stays the waypoint
#pragma unroll
            for (int a = 0; a < AX; ++a) {
              const int row = a * ND;
              const R P = szP[jE * 3 + a];
              mE[row] = mE[row] + (P - eE[a][0]);
              pE[row] = pE[row] + (P - eSnext[row]);
            }
          } else {
            R p0 = pE[r], p1 = pE[ND + r];
            junction_pair(eE[0][r], eE[1][r], eSnext[r], eSnext[ND + r], p0, p1, mE[r], mE[ND + r]);
            pE[r] = p0;
            pE[ND + r] = p1;
            const int row = 2 * ND + r;
            const R u2 = R(0.5) * (pE[row] - mE[row]);
            pE[row] = eE[2][r] + u2;
            mE[row] = eSnext[row] - u2;
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int r = 0; r < PO; ++r) {
            const int row = a * ND + r;
            mE[row] += pE[row] - eE[a][r];
          }
      }
    }
    __syncthreads();
    if (check) {
      // ---- 4. dual residual (Eq. 20), reductions, stopping rule (Eq. 21), rho update (Eq. 22) ----
      if (adapt && l == 0) *sflag = 0;  // every reader of the last flag has passed a barrier since
      R rd2 = R(0);
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
            dS[r] = first ? R(0) : sc.s[r] * sdz[jS * NJ + a * ND + r];
            dE[r] = last ? R(0) : sc.s[r] * sdz[jE * NJ + a * ND + r];
          }
          rd2 += dual_residual_sq(dS, dE, rho, Tk);
        }
      }
      sh_rp[l] = rp2;
      sh_rd[l] = rd2;
      __syncthreads();
      const int warp = l >> 5, lane = l & 31, nw = C >> 5;
      for (int t = warp; t < pk.ntraj; t += nw) {
        if (sdone[t]) continue;
        // FP64 accumulation of the shares in a fixed order: lane-strided, then a butterfly
        double a1 = 0.0, a2 = 0.0;
        for (int x = soff[t] + lane; x < soff[t + 1]; x += 32) { a1 += double(sh_rp[x]); a2 += double(sh_rd[x]); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a1 += __shfl_xor_sync(0xffffffffu, a1, o);
          a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
          const double rp = sqrt(a1), rd = sqrt(a2);
          tr_rp[t] = rp;
          tr_rd[t] = rd;
          const int bb = stid[t];
          if (res.history) {
            res.history[((size_t)k * p.B + bb) * 2 + 0] = rp;
            res.history[((size_t)k * p.B + bb) * 2 + 1] = rd;
          }
          const double tol = double(soff[t + 1] - soff[t]) * p.eps;
          int st = -1;
          if (!finite_d(rp) || !finite_d(rd)) st = 2;
          else if (p.eps > 0.0 && rp < tol && rd < tol) st = 0;
          if (STALL && st < 0 && p.stall > 0 && p.eps > 0.0 && A.stall) {  // the stall rule (stall_checks)
            double *sb = A.stall + 3 * (size_t)bb;  // best ||r_p||, best ||r_d||, checks since
            const bool bp = rp < 0.99 * sb[0], bd = rd < 0.99 * sb[1];
            if (bp) sb[0] = rp;
            if (bd) sb[1] = rd;
            sb[2] = (bp || bd) ? 0.0 : sb[2] + 1.0;
            if (sb[2] >= double(p.stall)) st = 3;
          }
          if (st >= 0) {
            sdone[t] = 1;
            atomicAdd(sndone, 1);
            res.iters[bb] = k + 1;
            res.status[bb] = st;
          } else if (adapt) {
            const double ro = srho[t], rn = next_rho(p, ro, rp, rd);
            sfac[t] = ro / rn;
            if (rn != ro) {
              srho[t] = rn;
              *sflag = 1;
            }
          }
        }
      }
      __syncthreads();
      // every trajectory of the pack has stopped: the CTA leaves the loop and frees its SM
      if (*sndone >= pk.ntraj) break;
      // ---- 5. after a change of rho: keep the unscaled duals, new local inverse ----
      if (adapt && *sflag && k + 1 < K) {
        if (valid && !sdone[tb] && sfac[tb] != 1.0) {
          const R f = R(sfac[tb]);
#pragma unroll
          for (int a = 0; a < AX; ++a)
#pragma unroll
            for (int r = 0; r < ND; ++r) {
              const int row = a * ND + r;
              if (!last) {  // p = z + u_start-side, m = z - u_end-side, z fixed for pinned rows
                const R zc = (pin && r == 0) ? szP[jE * 3 + a] : R(0.5) * (pE[row] + mE[row]);
                pE[row] = zc + f * (pE[row] - zc);
                mE[row] = zc + f * (mE[row] - zc);
              } else if (r < PO) {  // p holds the fixed end value
                mE[row] = pE[row] + f * (mE[row] - pE[row]);
              }
              if (first && r < PO) pS[row] = mS[row] + f * (pS[row] - mS[row]);  // m holds the start value
            }
          if (BOX)
            for (int q = 0; q < 6 * Mb; ++q) {
              const R y = sybox[q * C + l];
              if (y > R(0)) sybox[q * C + l] = f * y;  // v = max(0, y) scales, s = max(0, -y) stays
            }
          if (BALL)
            for (int j = 0; j < Mq; ++j) rescale_projected(sqball + j * 3 * C + l, C, sc.bo, sc.brad, f);
          if (VN) {
            const R zero3[3] = {R(0), R(0), R(0)};
            for (int j = 0; j < Mv; ++j) rescale_projected(sqvn + j * 3 * C + l, C, zero3, sc.vnorm, f);
          }
          R *Gw = (R *)A.G;  // this segment's column of the precomputed inverses
          g_from_eig_store((const R *)A.E, (size_t)p.S, (size_t)g, srho[tb], Gw);
#pragma unroll
          for (int q = 0; q < NG; ++q) sc.G[q] = Gw[(size_t)q * p.S + g];
          rho = R(srho[tb]);
        }
        __syncthreads();
      }
    }
  }

  // ---- export of the state (top_resume) ----
  if (A.to.p && valid) {
    const size_t oE = (size_t)(g + b + 1) * NJ, oS = (size_t)(g + b) * NJ;
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      A.to.p[oE + q] = double(pE[q]);
      A.to.m[oE + q] = double(mE[q]);
      if (first) {
        A.to.p[oS + q] = double(pS[q]);
        A.to.m[oS + q] = double(mS[q]);
      }
    }
    if (BOX) for (int q = 0; q < 6 * Mb; ++q) A.to.ybox[(size_t)g * 6 * Mb + q] = double(sybox[q * C + l]);
    if (BALL) for (int q = 0; q < 3 * Mq; ++q) A.to.qball[(size_t)g * 3 * Mq + q] = double(sqball[q * C + l]);
    if (VN) for (int q = 0; q < 3 * Mv; ++q) A.to.qvn[(size_t)g * 3 * Mv + q] = double(sqvn[q * C + l]);
  }

  // ---- outputs: coefficients in the paper's basis, FP64 cost per trajectory ----
  __syncthreads();  // the junction state is dead: its memory holds the warps' output tiles
  double *tile = (double *)(smem + L.p) + (size_t)(l >> 5) * 32 * kOutRow;
  double Ji = 0.0;
  if (valid) {
    R ch[AX][NC];
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) ch[a][q] = sch[chx(a * NC + q, l)];
    // c_k = ch_k T^-k with the iteration's own powers s_k (one rounding in the
    // iteration precision; the FP64 pipe runs at 1/64 of the FP32 rate)
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) tile[(l & 31) * kOutRow + a * NC + q] = double(ch[a][q] * sc.s[q]);
    Ji = segment_cost(ch, double(sc.s[7]));
  }
  store_rows_warp(res.coeffs, tile, g, valid);
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
        const int bb = stid[t];
        res.cost[bb] = a1;
        res.r_primal[bb] = tr_rp[t];
        res.r_dual[bb] = tr_rd[t];
        if (res.rho) res.rho[bb] = srho[t];
        const bool empty = soff[t + 1] == soff[t];
        if (empty) {
          res.iters[bb] = 0;
          res.status[bb] = 0;
        } else if (!sdone[t]) {
          res.iters[bb] = K;
          res.status[bb] = 1;
        }
        if (A.to.p) A.to.iters[bb] = (A.from.p ? A.from.iters[bb] : 0) + res.iters[bb];
      }
    }
  }
}

template <class R>
int launch_resident_t(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool adapt = a.p.adaptive != 0 && a.E != nullptr;
  if (a.stall && a.p.stall > 0 && !adapt)  // the stall rule's instances (fixed rho)
    return sizeof(R) == 4 ? launch_resident_stall_f32(a, nblocks, C, smem, fam, stream)
                          : launch_resident_stall_f64(a, nblocks, C, smem, fam, stream);
  if constexpr (sizeof(R) == 4) {
    if (a.tc && fam == 0 && !adapt) {
      auto kern = resident_kernel<R, 0, false, true>;
      cudaError_t e = func_attr_once((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
      kern<<<nblocks, C, smem, st>>>(a);
      return (int)cudaGetLastError();
    }
  }
#define TOP_RES_CASE(FV)                                                                               \
  case FV: {                                                                                           \
    auto kern = adapt ? resident_kernel<R, FV, true> : resident_kernel<R, FV, false>;                  \
    cudaError_t e = func_attr_once((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
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

// the instances with the stall rule (fixed rho)
template <class R>
int launch_resident_stall_t(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
#define TOP_RES_STALL_CASE(FV)                                                                         \
  case FV: {                                                                                           \
    auto kern = resident_kernel<R, FV, false, false, true>;                                            \
    cudaError_t e = func_attr_once((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return (int)e;                                                               \
    kern<<<nblocks, C, smem, st>>>(a);                                                                 \
    return (int)cudaGetLastError();                                                                    \
  }
  switch (fam) {
    TOP_RES_STALL_CASE(0)
    TOP_RES_STALL_CASE(1)
    TOP_RES_STALL_CASE(2)
    TOP_RES_STALL_CASE(3)
    TOP_RES_STALL_CASE(4)
    TOP_RES_STALL_CASE(5)
    TOP_RES_STALL_CASE(6)
    TOP_RES_STALL_CASE(7)
    default: return (int)cudaErrorInvalidValue;
  }
#undef TOP_RES_STALL_CASE
}

}  // namespace top
