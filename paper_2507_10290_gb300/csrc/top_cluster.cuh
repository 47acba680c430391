// top_cluster.cuh -- the cluster-resident CADMM kernel: one thread-block
// cluster per trajectory that is longer than one CTA holds but not longer than
// a cluster of CTAs (Algorithm 1 of the paper, Eq. 18a-g, 19-21).
//
// CTA `rank` of the cluster owns segments rank*C .. rank*C + C - 1 of the
// trajectory, one thread per segment, with all iteration state in its shared
// memory in the layout of the resident kernel (top_resident.cuh: junction
// targets p, m per slot, thread l owns the junction at its segment's end).
// The only state that crosses CTAs is at the C-boundaries, read through
// distributed shared memory:
//   - thread 0 of rank r > 0 reads its start target p (and, on check
//     iterations, the change of z there) from slot C of rank r - 1, the
//     junction's owner;
//   - thread C - 1 of rank r reads the start derivatives of thread 0 of
//     rank r + 1 in the junction step.
// The CTA barriers of the resident kernel become cluster barriers.  On check
// iterations every CTA reduces its share of ||r_p||^2, ||r_d||^2 in a fixed
// order, rank 0 adds the shares in rank order, applies the stopping test
// (Eq. 21) and publishes the stop decision, which every CTA reads back.  All CTAs of
// a cluster run the same number of cluster barriers (no early exit), and the
// kernel ends with one, so no CTA leaves while another may still read its
// shared memory.  Polytope rows (fixed rho) use the rotated per-axis inverses
// and their slack state from global memory (L2-resident at these sizes).
// With adaptive rho, rank 0 also applies Eq. 22 and every CTA
// rescales its own state and local inverses after a change (step 5 of the
// resident kernel), followed by a cluster barrier.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"
#include "top_step.cuh"

namespace top {

namespace cg = cooperative_groups;

// the sum of a right-hand side over the LN lanes of a segment (xor butterfly:
// every lane gets the same sum, the additions being commutative)
template <int LN, class R>
__device__ __forceinline__ void lanes_allreduce(R (&rhs)[AX][NC], unsigned mask) {
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int o = 1; o < LN; o <<= 1) rhs[a][q] += __shfl_xor_sync(mask, rhs[a][q], o);
}

// LN lanes per segment (1, 2 or 4; LN > 1 for FP32 with sample rows and fixed
// rho): the sample rows of a segment's local step (box, ball, velocity-norm,
// polytope) are split over its LN consecutive lanes and their shares of the
// right-hand side summed across them, so every lane forms the same
// coefficients and updates the states of its own samples; lane 0 of the
// segment (`own`) does everything else.
template <class R, int F, bool ADAPT, int LN = 1>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512, 1) cluster_kernel(const ClusterArgs A) {
  static_assert(LN == 1 || ((LN == 2 || LN == 4) && !ADAPT && sizeof(R) == 4),
                "lanes per segment: FP32 and fixed rho only");
  constexpr bool BOX = (F & FAM_BOX) != 0;
  constexpr bool BALL = (F & FAM_BALL) != 0;
  constexpr bool VN = (F & FAM_VN) != 0;
  constexpr bool POLY = (F & FAM_POLY) != 0;
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int csz = (int)cl.num_blocks();
  const DevProblem &p = A.p;
  const DevResult &res = A.r;
  const int b = A.traj[blockIdx.x / csz];
  // (cluster-uniform checks: a bad trajectory ends every CTA of the cluster
  // before any of them touches another's shared memory)
  if (!TOP_IN_BOUNDS(p.err, b >= 0 && b < p.B)) return;
  const int g0 = p.seg_offset[b];
  const int Nb = p.seg_offset[b + 1] - g0;
  if (!TOP_IN_BOUNDS(p.err, Nb >= 0 && Nb <= csz * (int)blockDim.x && g0 >= 0 && g0 + Nb <= p.S)) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int C = nthr / LN;      // segments per CTA
  const int l = tid / LN;       // this thread's segment in the CTA
  const int sub = tid % LN;     // its lane within the segment
  const bool own = sub == 0;
  const int Mb = BOX ? p.M_box : 0, Mq = BALL ? p.M_ball : 0, Mv = VN ? p.M_vn : 0;
  const int Mp = POLY ? p.M_poly : 0, Fp = POLY ? p.F_poly : 0;
  const ResLayout L = res_layout(C, kClusterNtp, Mb, Mq, Mv, (int)sizeof(R), Mp);
  double *red = (double *)(smem + L.red_rp);   // [C] FP64 cost shares (epilogue)
  R *sh_rp = (R *)(smem + L.red_rp);           // [C] residual shares
  R *sh_rd = (R *)(smem + L.red_rd);
  double *part = (double *)(smem + L.tr_rp);   // [8]: shares ||r_p||^2, ||r_d||^2, rank 0's norms, cost share,
                                               //      rank 0's rho and rho_old / rho_new (Eq. 22)
  int *sdone = (int *)(smem + L.done);         // rank 0: the stop decision
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
  R *tabP = (R *)(smem + L.tabP);

  R rho = R(p.rho);  // the trajectory's rho (changes only with adaptive rho)
  const int K = p.max_iters;
  const bool pin = (p.mode == 0);
  const int i = rank * C + l;  // segment within the trajectory
  const bool valid = i < Nb;
  const bool first = valid && i == 0;
  const bool last = valid && i == Nb - 1;
  const int g = g0 + i;
  const int J = C + kClusterNtp;
  const int jS = l, jE = l + 1;

  // ---- set-up: zeroed state, tables ----
  for (int q = tid; q < NJ * J; q += nthr) { sdz[q] = R(0); sp[q] = R(0); sm[q] = R(0); }
  for (int q = tid; q < 3 * J; q += nthr) szP[q] = R(0);
  if (BOX) for (int q = tid; q < 6 * Mb * C; q += nthr) sybox[q] = R(0);
  if (BALL) for (int q = tid; q < 3 * Mq * C; q += nthr) sqball[q] = R(0);
  if (VN) for (int q = tid; q < 3 * Mv * C; q += nthr) sqvn[q] = R(0);
  if (BOX) fill_sample_table(tabB, Mb, 1, tid, nthr);
  if (BALL) fill_sample_table(tabQ, Mq, 0, tid, nthr);
  if (VN) fill_sample_table(tabV, Mv, 1, tid, nthr);
  if (POLY) fill_sample_table(tabP, Mp, 0, tid, nthr);
  if (tid == 0) {
    sdone[0] = 0;
    part[5] = p.rho;
    part[6] = 1.0;
  }
  __syncthreads();

  // targets at the start junction: local slot, or the owner's slot C in rank - 1
  const bool remote_start = (l == 0 && rank > 0);
  R *pS = remote_start ? cl.map_shared_rank(sp + C * NJ, rank - 1) : sp + jS * NJ;
  R *mS = sm + jS * NJ;  // read only by the trajectory's first segment (rank 0, local)
  const R *dzS = remote_start ? cl.map_shared_rank(sdz + C * NJ, rank - 1) : sdz + jS * NJ;
  R *pE = sp + jE * NJ, *mE = sm + jE * NJ;
  const bool remote_next = (l == C - 1 && rank + 1 < csz);
  const R *eSnext = remote_next ? cl.map_shared_rank(seS, rank + 1) : seS + (l + 1) * NJ;

  SegConst<R> sc;
  R Tq = R(1);
  sc.vbox = sc.vnorm = sc.brad = R(0);
  sc.bo[0] = sc.bo[1] = sc.bo[2] = R(0);
  R *ypoly = POLY ? (R *)A.ypoly + (valid ? g : 0) : nullptr;  // own column, stride S
  if (valid) {
    if (!POLY) {  // the polytope family keeps its per-axis inverses in A.poly
      const R *Gp = (const R *)A.G;
#pragma unroll
      for (int q = 0; q < NG; ++q) sc.G[q] = Gp[(size_t)q * p.S + g];
    } else {
#pragma unroll
      for (int q = 0; q < NG; ++q) sc.G[q] = R(0);
      if (own)
        for (int q = 0; q < Fp * Mp; ++q) ypoly[(size_t)q * p.S] = R(0);
    }
    Tq = R(p.durations[g]);
    inv_powers(Tq, sc.s);
    if (BOX) sc.vbox = R(p.vbox[b]);
    if (VN) sc.vnorm = R(p.vnorm[b]);
    if (BALL) {
      sc.brad = R(p.ball_r[g]);
      for (int a = 0; a < 3; ++a) sc.bo[a] = R(p.ball_c[(size_t)g * 3 + a]);
    }
    // Init of Algorithm 1 (the owner writes its end junction; the first
    // segment also its start junction)
    for (int a = 0; a < (own ? AX : 0); ++a)
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
    if (A.from.p && own) {  // resume (top_resume): the exported targets and row states replace Init
      const size_t oE = (size_t)(g + b + 1) * NJ, oS = (size_t)(g + b) * NJ;
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
  cl.sync();
  const int k0 = A.from.p ? A.from.iters[b] : 0;  // iterations run before a resume
  R fs[ND];  // r! T^-r
#pragma unroll
  for (int r = 0; r < ND; ++r) fs[r] = R(fact(r)) * sc.s[r];

  R ch[AX][NC];
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) ch[a][k] = R(0);

  const int cev = p.check_every > 0 ? p.check_every : 1;
  const bool periodic = p.eps > 0.0 || res.history != nullptr;
  int done = 0;     // the stop decision, identical in every CTA of the cluster
  double best_p = 1e300, best_d = 1e300;  // stall rule (rank 0, thread 0): best ||r_p||, ||r_d|| so far
  int stc = 0;                             // and the checks since either improved
  double rp_last = 0.0, rd_last = 0.0;
  const int warp = tid >> 5, lane = tid & 31;
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);  // lanes of valid segments (a prefix of the warp)
  (void)vmask;
  for (int k = 0; k < K; ++k) {
    const bool check = ADAPT || (k == K - 1) || (periodic && ((k + 1) % cev == 0));
    const bool act = valid && !done;
    R eE[AX][ND];
    R eSv[AX][ND];
    if (act) {
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
      if (POLY) {
        const R *PN = (const R *)A.poly.N, *PH = (const R *)A.poly.H;
        R rhs[AX][NC];
        family_rhs<R, F & 7, true>(sc, wS, wE, rho, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV,
                                   Mb, Mq, Mv, rhs, sub, LN, own);
        poly_rhs(PN, PH, (size_t)p.S, (size_t)g, Fp, Mp, rho, ypoly, p.S, tabP, rhs, sub, LN);
        if constexpr (LN > 1) lanes_allreduce<LN>(rhs, vmask);
        poly_solve((const R *)A.poly.G, (const R *)A.poly.U, (size_t)p.S, (size_t)g, rhs, ch);
        family_update<R, F & 7>(sc, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV, Mb, Mq, Mv, ch,
                                sub, LN);
        poly_update(PN, PH, (size_t)p.S, (size_t)g, Fp, Mp, ypoly, p.S, tabP, ch, sub, LN);
      } else if constexpr (LN > 1) {
        R rhs[AX][NC];
        family_rhs<R, F & 7, true>(sc, wS, wE, rho, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV,
                                   Mb, Mq, Mv, rhs, sub, LN, own);
        lanes_allreduce<LN>(rhs, vmask);
        apply_g3(sc.G, rhs, ch);
        family_update<R, F & 7>(sc, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV, Mb, Mq, Mv, ch,
                                sub, LN);
      } else {
        local_step<R, F, true>(sc, wS, wE, rho, k + k0 == 0, sybox + l, sqball + l, sqvn + l, C, tabB, tabQ, tabV, Mb,
                               Mq, Mv, ch);
      }
      // ---- 2. publish start derivatives ----
      if (own) {
        end_derivs_shift(ch, fs, eSv, eE);
#pragma unroll
        for (int a = 0; a < AX; ++a)
#pragma unroll
          for (int r = 0; r < ND; ++r) seS[l * NJ + a * ND + r] = eSv[a][r];
        // the trajectory's start slot has no other reader: its dual update (Eq. 18c
        // against the fixed start state) needs no barrier
        if (first) {
#pragma unroll
          for (int a = 0; a < AX; ++a)
#pragma unroll
            for (int r = 0; r < PO; ++r) {
              const int row = a * ND + r;
              pS[row] += mS[row] - eSv[a][r];
            }
        }
      }
    }
    cl.sync();
    // ---- 3. junction update (Eq. 18b, 18c) and primal residual (Eq. 19) ----
    R rp2 = R(0);
    if (act && own) {
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
            R p0 = pE[r], p1 = pE[ND + r], m0 = mE[r], m1 = mE[ND + r];
            junction_pair(eE[0][r], eE[1][r], eSnext[r], eSnext[ND + r], p0, p1, m0, m1);
            pE[r] = p0;
            pE[ND + r] = p1;
            mE[r] = m0;
            mE[ND + r] = m1;
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
    cl.sync();
    if (check) {
      // ---- 4. dual residual (Eq. 20), cluster reduction, stopping rule (Eq. 21) ----
      R rd2 = R(0);
      if (act && own) {
        R Tk[NC];
        Tk[0] = R(1);
#pragma unroll
        for (int q = 1; q < NC; ++q) Tk[q] = Tk[q - 1] * Tq;
#pragma unroll
        for (int a = 0; a < AX; ++a) {
          R dS[ND], dE[ND];
#pragma unroll
          for (int r = 0; r < ND; ++r) {
            dS[r] = first ? R(0) : sc.s[r] * dzS[a * ND + r];
            dE[r] = last ? R(0) : sc.s[r] * sdz[jE * NJ + a * ND + r];
          }
          rd2 += dual_residual_sq(dS, dE, rho, Tk);
        }
      }
      if (own) {
        sh_rp[l] = rp2;
        sh_rd[l] = rd2;
      }
      __syncthreads();
      if (warp == 0) {  // this CTA's shares, accumulated in FP64 in a fixed order
        double a1 = 0.0, a2 = 0.0;
        for (int x = lane; x < C; x += 32) { a1 += double(sh_rp[x]); a2 += double(sh_rd[x]); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a1 += __shfl_xor_sync(0xffffffffu, a1, o);
          a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) { part[0] = a1; part[1] = a2; }
      }
      cl.sync();
      if (rank == 0 && tid == 0 && !done) {  // shares in rank order, the stop decision
        double s1 = 0.0, s2 = 0.0;
        for (int q = 0; q < csz; ++q) {
          const double *pq = cl.map_shared_rank(part, q);
          s1 += pq[0];
          s2 += pq[1];
        }
        const double rp = sqrt(s1), rd = sqrt(s2);
        part[2] = rp;
        part[3] = rd;
        if (res.history) {
          res.history[((size_t)k * p.B + b) * 2 + 0] = rp;
          res.history[((size_t)k * p.B + b) * 2 + 1] = rd;
        }
        const double tol = double(Nb) * p.eps;
        int st = -1;
        if (!finite_d(rp) || !finite_d(rd)) st = 2;
        else if (p.eps > 0.0 && rp < tol && rd < tol) st = 0;
        if (st < 0 && p.stall > 0 && p.eps > 0.0) {  // the stall rule (top_problem.stall_checks)
          const bool bp = rp < 0.99 * best_p, bd = rd < 0.99 * best_d;
          if (bp) best_p = rp;
          if (bd) best_d = rd;
          if (bp || bd) stc = 0;
          else if (++stc >= p.stall) st = 3;
        }
        part[6] = 1.0;
        if (st >= 0) {
          sdone[0] = 1;
          res.iters[b] = k + 1;
          res.status[b] = st;
        } else if (ADAPT) {  // UpdateRho (Eq. 22)
          const double ro = part[5], rn = next_rho(p, ro, rp, rd);
          part[5] = rn;
          part[6] = ro / rn;
        }
      }
      cl.sync();
      const int *vd = cl.map_shared_rank(sdone, 0);
      done = vd[0];
      double fac = 1.0, rho_new = 0.0;
      if (ADAPT) {
        const double *p0 = cl.map_shared_rank(part, 0);
        fac = p0[6];
        rho_new = p0[5];
      }
      if (rank == 0) { rp_last = part[2]; rd_last = part[3]; }
      cl.sync();  // the decision is read everywhere before rank 0 may write the next shares
      if (done) break;  // the same decision in every CTA: a uniform exit from the loop
      // ---- 5. after a change of rho (adaptive rho): keep the unscaled duals, new local inverse ----
      if (ADAPT && fac != 1.0 && k + 1 < K) {  // the same fac in every CTA
        if (valid) {
          const R f = R(fac);
#pragma unroll
          for (int a = 0; a < AX; ++a)
#pragma unroll
            for (int r = 0; r < ND; ++r) {
              const int row = a * ND + r;
              if (!last) {
                const R zc = (pin && r == 0) ? szP[jE * 3 + a] : R(0.5) * (pE[row] + mE[row]);
                pE[row] = zc + f * (pE[row] - zc);
                mE[row] = zc + f * (mE[row] - zc);
              } else if (r < PO) {
                mE[row] = pE[row] + f * (mE[row] - pE[row]);
              }
              if (first && r < PO) pS[row] = mS[row] + f * (pS[row] - mS[row]);
            }
          if (BOX)
            for (int q = 0; q < 6 * Mb; ++q) {
              const R y = sybox[q * C + l];
              if (y > R(0)) sybox[q * C + l] = f * y;
            }
          if (BALL)
            for (int j = 0; j < Mq; ++j) rescale_projected(sqball + j * 3 * C + l, C, sc.bo, sc.brad, f);
          if (VN) {
            const R zero3[3] = {R(0), R(0), R(0)};
            for (int j = 0; j < Mv; ++j) rescale_projected(sqvn + j * 3 * C + l, C, zero3, sc.vnorm, f);
          }
          R *Gw = (R *)A.G;
          g_from_eig_store((const R *)A.E, (size_t)p.S, (size_t)g, rho_new, Gw);
#pragma unroll
          for (int q = 0; q < NG; ++q) sc.G[q] = Gw[(size_t)q * p.S + g];
          rho = R(rho_new);
        }
        cl.sync();  // the owners' rescaled targets before any start-side read
      }
    }
  }

  // ---- export of the state (top_resume) ----
  if (A.to.p && valid && own) {
    const size_t oE = (size_t)(g + b + 1) * NJ, oS = (size_t)(g + b) * NJ;
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

  // ---- outputs: coefficients in the paper's basis, FP64 cost (cluster sum in rank order) ----
  double Ji = 0.0;
  if (valid && own) {
    // c_k = ch_k T^-k with the iteration's own powers s_k
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) res.coeffs[((size_t)g * AX + a) * NC + q] = double(ch[a][q] * sc.s[q]);
    Ji = segment_cost(ch, double(sc.s[7]));
  }
  if (own) red[l] = Ji;
  __syncthreads();
  if (warp == 0) {
    double a1 = 0.0;
    for (int x = lane; x < C; x += 32) a1 += red[x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    if (lane == 0) part[4] = a1;
  }
  cl.sync();
  if (rank == 0 && tid == 0) {
    double J = 0.0;
    for (int q = 0; q < csz; ++q) J += cl.map_shared_rank(part, q)[4];
    res.cost[b] = J;
    if (res.rho) res.rho[b] = part[5];
    res.r_primal[b] = rp_last;
    res.r_dual[b] = rd_last;
    if (!done) {
      res.iters[b] = K;
      res.status[b] = 1;
    }
    if (A.to.p) A.to.iters[b] = k0 + res.iters[b];
  }
  cl.sync();  // no CTA leaves while rank 0 reads its shared memory
}

}  // namespace top

namespace top {

template <class R, bool ADAPT>
__host__ void *cluster_kernel_for_t(int fam) {
  switch (fam) {
    case 0: return (void *)cluster_kernel<R, 0, ADAPT>;
    case 1: return (void *)cluster_kernel<R, 1, ADAPT>;
    case 2: return (void *)cluster_kernel<R, 2, ADAPT>;
    case 3: return (void *)cluster_kernel<R, 3, ADAPT>;
    case 4: return (void *)cluster_kernel<R, 4, ADAPT>;
    case 5: return (void *)cluster_kernel<R, 5, ADAPT>;
    case 6: return (void *)cluster_kernel<R, 6, ADAPT>;
    case 7: return (void *)cluster_kernel<R, 7, ADAPT>;
    case 16: return (void *)cluster_kernel<R, 16, false>;
    case 17: return (void *)cluster_kernel<R, 17, false>;
    case 18: return (void *)cluster_kernel<R, 18, false>;
    case 19: return (void *)cluster_kernel<R, 19, false>;
    case 20: return (void *)cluster_kernel<R, 20, false>;
    case 21: return (void *)cluster_kernel<R, 21, false>;
    case 22: return (void *)cluster_kernel<R, 22, false>;
    case 23: return (void *)cluster_kernel<R, 23, false>;
    default: return nullptr;
  }
}

// ln lanes per segment (ln > 1: FP32, fixed rho, families with sample rows; top_cluster_l*_f32.cu)
template <class R>
__host__ void *cluster_kernel_for(int fam, bool adapt, int ln) {
  if (ln > 1) return (sizeof(R) == 4 && !adapt) ? cluster_lanes_kernel_f32(fam, ln) : nullptr;
  return adapt ? cluster_kernel_for_t<R, true>(fam) : cluster_kernel_for_t<R, false>(fam);
}

template <class R>
__host__ int cluster_max_size_t(int C, int ln, size_t smem, int fam) {
  void *kern = cluster_kernel_for<R>(fam, false, ln);
  if (!kern) return 0;
  if (func_attr_once(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      func_attr_once(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int csz = 16; csz >= 1; csz >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csz);
    cfg.blockDim = dim3(C * ln);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csz;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) return csz;
    cudaGetLastError();
  }
  return 0;
}

template <class R>
__host__ int launch_cluster_t(const ClusterArgs &a, int nclusters, int csz, int C, int ln, size_t smem, int fam,
                              void *stream) {
  void *kern = cluster_kernel_for<R>(fam, a.p.adaptive != 0 && a.E != nullptr, ln);
  if (!kern || nclusters <= 0) return kern ? 0 : (int)cudaErrorInvalidValue;
  cudaError_t e = func_attr_once(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = func_attr_once(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return (int)e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * csz);
  cfg.blockDim = dim3(C * ln);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csz;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void *args[] = {(void *)&a};
  e = cudaLaunchKernelExC(&cfg, kern, args);
  return (int)e;
}

}  // namespace top
