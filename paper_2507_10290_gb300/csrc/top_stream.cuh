// top_stream.cuh -- the streaming CADMM form for trajectories longer than one
// CTA's shared memory holds: all iteration state in global memory, one launch
// per phase of each iteration (Algorithm 1, Eq. 18a-g, 19-21):
//   stream_local     every segment: local step + projections (shared
//                    local_step; polytope rows through the rotated per-axis
//                    inverses), end derivatives to global memory
//   stream_junction  every segment's end junction: consensus average, scaled
//                    duals, primal-residual share, consensus change
//   stream_reduce    on check iterations: dual-residual shares, then blocks of
//                    kReduceChunk segments sum the shares in a fixed order and
//                    the last block of each trajectory adds the chunk sums,
//                    records the history and applies the stopping rule
//   stream_output    coefficients in the paper's basis and per-trajectory cost
// Segments are addressed through a compact index x over the long
// trajectories (lt_prefix[t] .. lt_prefix[t+1]-1 belong to trajectory lt_b[t]);
// junction state is indexed like the waypoints (segment g of trajectory b ends
// at junction g + b + 1).
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"
#include "top_math.cuh"
#include "top_step.cuh"

namespace top {

// false (checked build only) when the derived indices leave their arrays: the
// caller then skips the segment
__device__ __forceinline__ bool stream_locate(const StreamArgs &A, int x, int &t, int &b, int &i, int &N, int &g) {
  if (A.seg_t) {  // one load instead of a search over the trajectories
    t = A.seg_t[x];
    if (!TOP_IN_BOUNDS(A.p.err, t >= 0 && t < A.nl)) return false;
  } else {
    int lo = 0, hi = A.nl - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (A.lt_prefix[mid] <= x) lo = mid; else hi = mid - 1;
    }
    t = lo;
  }
  b = A.lt_b[t];
  if (!TOP_IN_BOUNDS(A.p.err, b >= 0 && b < A.p.B)) return false;
  i = x - A.lt_prefix[t];
  N = A.lt_prefix[t + 1] - A.lt_prefix[t];
  g = A.p.seg_offset[b] + i;
  return TOP_IN_BOUNDS(A.p.err, i >= 0 && i < N && g >= 0 && g < A.S && g + b + 1 < A.Jn);
}

// the streaming trajectory of every compact index: block t fills trajectory t's range
// (a template like the other kernels, so each precision's translation unit has its own instance)
template <class R>
__global__ void __launch_bounds__(256) stream_map(const StreamArgs A) {
  for (int t = blockIdx.x; t < A.nl; t += gridDim.x) {
    const int x0 = A.lt_prefix[t], x1 = A.lt_prefix[t + 1];
    if (!TOP_IN_BOUNDS(A.p.err, x0 >= 0 && x0 <= x1 && x1 <= A.total)) continue;
    for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) A.seg_t[x] = t;
  }
}

template <class R, int F>
__global__ void stream_init(const StreamArgs A) {
  constexpr bool BOX = (F & FAM_BOX) != 0, BALL = (F & FAM_BALL) != 0, VN = (F & FAM_VN) != 0;
  const DevProblem &p = A.p;
  R *z = (R *)A.z, *uL = (R *)A.uL, *uRp = (R *)A.uRp, *dz = (R *)A.dz, *uR0 = (R *)A.uR0;
  R *ch = (R *)A.ch, *ybox = (R *)A.ybox, *qball = (R *)A.qball, *qvn = (R *)A.qvn;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < A.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    for (int a = 0; a < AX; ++a)
      for (int r = 0; r < ND; ++r) {
        R zv = R(0);
        if (!last) {
          if (r == 0) zv = R(p.waypoints[(size_t)jE * 3 + a]);
        } else if (r < PO) {
          zv = R(p.end_state[((size_t)b * PO + r) * 3 + a]);
        }
        const size_t row = (size_t)(a * ND + r) * A.Jn;
        const R zs = r < PO ? R(p.start_state[((size_t)b * PO + r) * 3 + a]) : R(0);
        z[row + jE] = zv;
        uL[row + jE] = R(0);
        dz[row + jE] = R(0);
        if (first) {
          z[row + jS] = zs;
          uL[row + jS] = R(0);
          dz[row + jS] = R(0);
        }
        if (A.zB) {  // both halves: the rows no junction update writes stay valid in either
          ((R *)A.zB)[row + jE] = zv;
          ((R *)A.uLB)[row + jE] = R(0);
          if (first) {
            ((R *)A.zB)[row + jS] = zs;
            ((R *)A.uLB)[row + jS] = R(0);
          }
        }
      }
    for (int a = 0; a < 3; ++a) {
      uRp[(size_t)a * A.Jn + jE] = R(0);
      if (first) uRp[(size_t)a * A.Jn + jS] = R(0);
      if (A.uRpB) {
        ((R *)A.uRpB)[(size_t)a * A.Jn + jE] = R(0);
        if (first) ((R *)A.uRpB)[(size_t)a * A.Jn + jS] = R(0);
      }
    }
    if (first)
      for (int q = 0; q < 12; ++q) uR0[(size_t)q * p.B + b] = R(0);
    for (int q = 0; q < 24; ++q) ch[(size_t)q * A.S + g] = R(0);
    if (BOX) for (int q = 0; q < 6 * p.M_box; ++q) ybox[(size_t)q * A.S + g] = R(0);
    if (BALL) for (int q = 0; q < 3 * p.M_ball; ++q) qball[(size_t)q * A.S + g] = R(0);
    if (VN) for (int q = 0; q < 3 * p.M_vn; ++q) qvn[(size_t)q * A.S + g] = R(0);
    if (F & FAM_POLY)
      for (int q = 0; q < p.F_poly * p.M_poly; ++q) ((R *)A.ypoly)[(size_t)q * A.S + g] = R(0);
    if (F & FAM_GEN) {
      for (int q = 0; q < 2 * p.M_gen; ++q) ((R *)A.ygen)[(size_t)q * A.S + g] = R(0);
      if (A.inner_iters) A.inner_iters[g] = 0;
    }
    if (x == 0 && A.nwork) A.nwork[0] = A.nwork[1] = 0;  // both work-list counts start at zero
    if (first) {
      A.done[t] = 0;
      if (A.kcount) A.kcount[t] = 0;
      if (A.ticket) A.ticket[t] = 0;
      A.tr_rp[t] = 0.0;
      A.tr_rd[t] = 0.0;
      A.rho_t[t] = p.rho;
      A.fac_t[t] = 1.0;
    }
  }
}

// The fused form's first half: the previous iteration's junction update
// (Eq. 18b-c, the arithmetic of stream_junction) at both ends of segment g,
// from the previous end values eSp, eEp and the junction state z, uL, uRp,
// giving the local step's targets w = z - u at both ends.  The segment owns
// its end junction and stores that junction's new state in zn, uLn, uRpn (and
// the first segment its trajectory's start duals uR0, in place); its start
// junction belongs to the previous segment, whose update it repeats in
// registers with the same operands, so both see the same values.
template <class R>
__device__ __forceinline__ void fused_junctions(const StreamArgs &A, bool first, bool last, bool pin, int b, int g,
                                                int jS, int jE, R (&w)[AX][2][ND]) {
  const DevProblem &p = A.p;
  const R *z = (const R *)A.z, *uL = (const R *)A.uL, *uRp = (const R *)A.uRp;
  const R *eSp = (const R *)A.eSp, *eEp = (const R *)A.eEp;
  R *zn = (R *)A.zn, *uLn = (R *)A.uLn, *uRpn = (R *)A.uRpn, *uR0 = (R *)A.uR0;
#pragma unroll
  for (int a = 0; a < AX; ++a) {
    R em[ND], es[ND], ee[ND], en[ND], zS[ND], uS[ND], zE[ND], uE[ND];
    R upS = R(0), upE = R(0);
#pragma unroll
    for (int r = 0; r < ND; ++r) {  // every load of the axis first
      const size_t row = (size_t)(a * ND + r) * A.Jn, er = (size_t)(a * ND + r) * A.S;
      em[r] = first ? R(0) : eEp[er + g - 1];
      es[r] = eSp[er + g];
      ee[r] = eEp[er + g];
      en[r] = last ? R(0) : eSp[er + g + 1];
      zS[r] = (!first || r < PO) ? z[row + jS] : R(0);
      uS[r] = first ? (r < PO ? uR0[(size_t)(a * PO + r) * p.B + b] : R(0)) : uL[row + jS];
      zE[r] = (!last || r < PO) ? z[row + jE] : R(0);
      uE[r] = (!last || r < PO) ? uL[row + jE] : R(0);
    }
    if (pin && !first) upS = uRp[(size_t)a * A.Jn + jS];
    if (pin && !last) upE = uRp[(size_t)a * A.Jn + jE];
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      const size_t row = (size_t)(a * ND + r) * A.Jn;
      // end junction (owned): stream_junction's update, stored
      if (!last) {
        if (pin && r == 0) {
          const R P = zE[r];
          const R ul = uE[r] + (ee[r] - P);
          uLn[row + jE] = ul;
          uRpn[(size_t)a * A.Jn + jE] = upE + (en[r] - P);
          w[a][1][r] = P - ul;
        } else {
          const R zm = R(0.5) * (ee[r] + en[r]);
          const R ul = uE[r] + (ee[r] - zm);
          uLn[row + jE] = ul;
          zn[row + jE] = zm;
          w[a][1][r] = zm - ul;
        }
      } else if (r < PO) {
        const R ul = uE[r] + (ee[r] - zE[r]);
        uLn[row + jE] = ul;
        w[a][1][r] = zE[r] - ul;
      } else {
        w[a][1][r] = R(0);
      }
      // start junction: the trajectory's start (its duals uR0 kept in place) or the previous segment's end
      if (first) {
        if (r < PO) {
          const R u0 = uS[r] + (es[r] - zS[r]);
          uR0[(size_t)(a * PO + r) * p.B + b] = u0;
          w[a][0][r] = zS[r] - u0;
        } else {
          w[a][0][r] = R(0);
        }
      } else if (pin && r == 0) {
        const R P = zS[r];
        w[a][0][r] = P - (upS + (es[r] - P));
      } else {
        const R zm = R(0.5) * (em[r] + es[r]);
        const R ul = uS[r] + (em[r] - zm);
        w[a][0][r] = zm - (-ul);
      }
    }
  }
}

// F may carry kDeferNumeric with FAM_GEN: the numerical step's segments whose
// bound is violated go to the work list of stream_numeric_warp (the warp form);
// with kFused the step begins with the previous iteration's junction update
// (fused_junctions) instead of reading the state that stream_junction wrote
constexpr int kDeferNumeric = 32;
constexpr int kFused = 64;
template <class R, int F>
__global__ void __launch_bounds__(256, ((F & kFused) && sizeof(R) == 4 && (!(F & FAM_GEN) || (F & kDeferNumeric))) ? 2 : 1)
stream_local(const StreamArgs A, int k) {
  constexpr bool BOX = (F & FAM_BOX) != 0, BALL = (F & FAM_BALL) != 0, VN = (F & FAM_VN) != 0;
  constexpr bool DEFER = (F & kDeferNumeric) != 0, FUSED = (F & kFused) != 0;
  const DevProblem &p = A.p;
  extern __shared__ __align__(16) unsigned char smem[];
  const int Mb = BOX ? p.M_box : 0, Mq = BALL ? p.M_ball : 0, Mv = VN ? p.M_vn : 0;
  R *tabB = (R *)smem, *tabQ = tabB + 8 * Mb, *tabV = tabQ + 8 * Mq;
  if (BOX) fill_sample_table(tabB, Mb, 1, threadIdx.x, blockDim.x);
  if (BALL) fill_sample_table(tabQ, Mq, 0, threadIdx.x, blockDim.x);
  if (VN) fill_sample_table(tabV, Mv, 1, threadIdx.x, blockDim.x);
  constexpr bool GEN = (F & FAM_GEN) != 0;
  const int Mg = GEN ? p.M_gen : 0;
  R *tabGV = tabV + 8 * Mv, *tabGA = tabGV + 8 * Mg;
  if (GEN) {
    fill_sample_table(tabGV, Mg, 1, threadIdx.x, blockDim.x);
    fill_accel_table(tabGA, Mg, threadIdx.x, blockDim.x);
  }
  constexpr bool POLY = (F & FAM_POLY) != 0;
  const int Mp = POLY ? p.M_poly : 0, Fp = POLY ? p.F_poly : 0;
  R *tabP = tabGA + 8 * Mg;
  if (POLY) fill_sample_table(tabP, Mp, 0, threadIdx.x, blockDim.x);
  __syncthreads();
  const R *z = (const R *)A.z, *uL = (const R *)A.uL, *uRp = (const R *)A.uRp, *uR0 = (const R *)A.uR0;
  const R *Gp = (const R *)A.G;
  R *eS = (R *)A.eS, *eE = (R *)A.eE, *chg = (R *)A.ch;
  const bool pin = p.mode == 0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < A.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    if (A.done[t]) continue;
    const R rho = R(A.rho_t[t]);
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    SegConst<R> sc;
    if (!POLY) {  // the polytope family keeps its per-axis inverses in A.poly
#pragma unroll
      for (int q = 0; q < NG; ++q) sc.G[q] = Gp[(size_t)q * A.S + g];
    }
    inv_powers(R(p.durations[g]), sc.s);
    sc.vbox = BOX ? R(p.vbox[b]) : R(0);
    sc.vnorm = VN ? R(p.vnorm[b]) : R(0);
    sc.brad = BALL ? R(p.ball_r[g]) : R(0);
    for (int a = 0; a < 3; ++a) sc.bo[a] = BALL ? R(p.ball_c[(size_t)g * 3 + a]) : R(0);
    R w[AX][2][ND];  // E (z~ - u) at both ends, unscaled
    if (FUSED) {
      fused_junctions<R>(A, first, last, pin, b, g, jS, jE, w);
    } else {
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int r = 0; r < ND; ++r) {
          const size_t row = (size_t)(a * ND + r) * A.Jn;
          R us;
          if (first) us = (r < PO) ? uR0[(size_t)(a * PO + r) * p.B + b] : R(0);
          else if (pin && r == 0) us = uRp[(size_t)a * A.Jn + jS];
          else us = -uL[row + jS];
          w[a][0][r] = (first && r >= PO) ? R(0) : z[row + jS] - us;
          w[a][1][r] = (last && r >= PO) ? R(0) : z[row + jE] - uL[row + jE];
        }
    }
    R ch[AX][NC];
    if (GEN) {
      const int its = numeric_step<R, DEFER>(sc, w, rho, first, last, (R *)A.ygen + g, A.S, tabGV, tabGA, Mg,
                                             R(p.gen_vmax[b]), R(p.gen_amax[b]), p.lbfgs_mem, p.lbfgs_max_iters,
                                             R(p.lbfgs_tol), ch);
      if (its < 0) {  // a violated bound: one warp per such segment solves it (stream_numeric_warp)
        A.work[atomicAdd(A.nwork, 1)] = x;
        continue;
      }
      if (A.inner_iters) A.inner_iters[g] += its;
    } else {
      R wS[AX][ND], wE[AX][ND];
#pragma unroll
      for (int a = 0; a < AX; ++a)
#pragma unroll
        for (int r = 0; r < ND; ++r) {
          wS[a][r] = sc.s[r] * w[a][0][r];
          wE[a][r] = sc.s[r] * w[a][1][r];
        }
      if (POLY) {
        const R *PN = (const R *)A.poly.N, *PH = (const R *)A.poly.H;
        R rhs[AX][NC];
        family_rhs<R, F & 7>(sc, wS, wE, rho, k == 0, (R *)A.ybox + g, (R *)A.qball + g, (R *)A.qvn + g, A.S,
                             tabB, tabQ, tabV, Mb, Mq, Mv, rhs);
        poly_rhs(PN, PH, (size_t)A.S, (size_t)g, Fp, Mp, rho, (const R *)A.ypoly + g, A.S, tabP, rhs);
        poly_solve((const R *)A.poly.G, (const R *)A.poly.U, (size_t)A.S, (size_t)g, rhs, ch);
        family_update<R, F & 7>(sc, k == 0, (R *)A.ybox + g, (R *)A.qball + g, (R *)A.qvn + g, A.S, tabB, tabQ,
                                tabV, Mb, Mq, Mv, ch);
        poly_update(PN, PH, (size_t)A.S, (size_t)g, Fp, Mp, (R *)A.ypoly + g, A.S, tabP, ch);
      } else {
        local_step<R, F & 7>(sc, wS, wE, rho, k == 0, (R *)A.ybox + g, (R *)A.qball + g, (R *)A.qvn + g, A.S,
                             tabB, tabQ, tabV, Mb, Mq, Mv, ch);
      }
    }
#pragma unroll
    for (int a = 0; a < AX; ++a) {
      R s7[ND], e7[ND];
      end_derivs(ch[a], sc.s, s7, e7);
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        eS[(size_t)(a * ND + r) * A.S + g] = s7[r];
        eE[(size_t)(a * ND + r) * A.S + g] = e7[r];
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) chg[(size_t)(a * NC + q) * A.S + g] = ch[a][q];
    }
  }
}

// The numerical step for the segments stream_local deferred (a bound violated
// at the minimiser of the quadratic part): one warp per segment, lanes over
// (axis, coefficient); writes the coefficients, the end derivatives, the duals y
// and the L-BFGS iteration count.  The order of the work list does not matter:
// each segment's result depends only on its own data.
template <class R>
__global__ void __launch_bounds__(256) stream_numeric_warp(const StreamArgs A) {
  const DevProblem &p = A.p;
  extern __shared__ __align__(16) unsigned char smem[];
  const int Mg = p.M_gen;
  R *tabGV = (R *)smem, *tabGA = tabGV + 8 * Mg;
  R *wsc = tabGA + 8 * Mg + (threadIdx.x >> 5) * 96;  // this warp's [3][32] gradient scratch
  // fused iterations: the next iteration's local step appends to the other count, which nothing reads now
  if (A.nwork_next && blockIdx.x == 0 && threadIdx.x == 0) *A.nwork_next = 0;
  const int n = *A.nwork;
  if (blockIdx.x * (blockDim.x >> 5) >= n) return;  // no listed segment for this block (uniform in the block)
  fill_sample_table(tabGV, Mg, 1, threadIdx.x, blockDim.x);
  fill_accel_table(tabGA, Mg, threadIdx.x, blockDim.x);
  __syncthreads();
  const R *z = (const R *)A.z, *uL = (const R *)A.uL, *uRp = (const R *)A.uRp, *uR0 = (const R *)A.uR0;
  const R *Gp = (const R *)A.G;
  R *eS = (R *)A.eS, *eE = (R *)A.eE, *chg = (R *)A.ch;
  const bool pin = p.mode == 0;
  const int lane = threadIdx.x & 31, k = lane & 7, a = lane >> 3;
  const bool live = lane < 24;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < n; item += nwarps) {
    const int x = A.work[item];
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    const R rho = R(A.rho_t[t]);
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    R s[NC];
    inv_powers(R(p.durations[g]), s);
    R Grow[NC];
#pragma unroll
    for (int l = 0; l < NC; ++l) Grow[l] = live ? Gp[(size_t)gidx(k, l) * A.S + g] : R(0);
    R w0 = R(0), w1 = R(0);  // E (z~ - u) at the two ends, row (a, k)
    if (live && k < ND) {
      const int r = k;
      const size_t row = (size_t)(a * ND + r) * A.Jn;
      R us;
      if (first) us = (r < PO) ? uR0[(size_t)(a * PO + r) * p.B + b] : R(0);
      else if (pin && r == 0) us = uRp[(size_t)a * A.Jn + jS];
      else us = -uL[row + jS];
      w0 = (first && r >= PO) ? R(0) : z[row + jS] - us;
      w1 = (last && r >= PO) ? R(0) : z[row + jE] - uL[row + jE];
    }
    R c;
    const int its = numeric_step_warp<R>(Grow, s, w0, w1, rho, first, last, (R *)A.ygen + g, A.S, tabGV, tabGA,
                                         Mg, R(p.gen_vmax[b]), R(p.gen_amax[b]), p.lbfgs_mem, p.lbfgs_max_iters,
                                         R(p.lbfgs_tol), wsc, c);
    // outputs: coefficients, end derivatives (rows of M(T) c, Sec. III-D.1)
    const int base = lane & ~7;
    R cax[NC];
#pragma unroll
    for (int l = 0; l < NC; ++l) cax[l] = __shfl_sync(0xffffffffu, c, base + l);
    if (live) {
      chg[(size_t)(a * NC + k) * A.S + g] = c;
      if (k < ND) {
        R acc = R(0);
        for (int m = k; m < NC; ++m) acc += R(falling_rt(m, k)) * cax[m];
        eS[(size_t)(a * ND + k) * A.S + g] = R(fact_rt(k)) * s[k] * c;
        eE[(size_t)(a * ND + k) * A.S + g] = s[k] * acc;
      }
    }
    if (lane == 0 && A.inner_iters) A.inner_iters[g] += its;
  }
}

// Every junction value one axis needs is loaded before any of that axis's
// updates is stored, so the loads of an axis are in flight together (a store
// to z, uL or uRp would otherwise order the next row's loads behind it).
template <class R>
__global__ void __launch_bounds__(256) stream_junction(const StreamArgs A, int check) {
  const DevProblem &p = A.p;
  R *z = (R *)A.z, *uL = (R *)A.uL, *uRp = (R *)A.uRp, *dz = (R *)A.dz, *uR0 = (R *)A.uR0;
  const R *eS = (const R *)A.eS, *eE = (const R *)A.eE;
  const bool pin = p.mode == 0;
  // stream_numeric_warp of this iteration has read its work list: the next local step starts a new one
  if (A.nwork && blockIdx.x == 0 && threadIdx.x == 0) *A.nwork = 0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < A.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    if (A.done[t]) continue;
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    R rp2 = R(0);
#pragma unroll
    for (int a = 0; a < AX; ++a) {
      R ee[ND], en[ND], zE[ND], uE[ND], es[PO], zS[PO], u0[PO];
      R up = R(0);
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * A.Jn;
        ee[r] = eE[(size_t)(a * ND + r) * A.S + g];
        en[r] = last ? R(0) : eS[(size_t)(a * ND + r) * A.S + g + 1];
        zE[r] = (!last || r < PO) ? z[row + jE] : R(0);
        uE[r] = (!last || r < PO) ? uL[row + jE] : R(0);
        if (r < PO) {
          es[r] = first ? eS[(size_t)(a * ND + r) * A.S + g] : R(0);
          zS[r] = first ? z[row + jS] : R(0);
          u0[r] = first ? uR0[(size_t)(a * PO + r) * p.B + b] : R(0);
        }
      }
      if (pin && !last) up = uRp[(size_t)a * A.Jn + jE];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * A.Jn;
        if (!last) {
          if (check) {
            const R gap = ee[r] - en[r];
            rp2 += gap * gap;
          }
          if (pin && r == 0) {
            const R P = zE[r];
            uL[row + jE] = uE[r] + (ee[r] - P);
            uRp[(size_t)a * A.Jn + jE] = up + (en[r] - P);
            if (check) dz[row + jE] = R(0);
          } else {
            const R zn = R(0.5) * (ee[r] + en[r]);
            uL[row + jE] = uE[r] + (ee[r] - zn);
            z[row + jE] = zn;
            if (check) dz[row + jE] = zn - zE[r];
          }
        } else if (r < PO) {
          uL[row + jE] = uE[r] + (ee[r] - zE[r]);
        }
        if (first && r < PO) uR0[(size_t)(a * PO + r) * p.B + b] = u0[r] + (es[r] - zS[r]);
      }
    }
    if (check) A.rp2[x] = double(rp2);
  }
}

template <class R>
__global__ void __launch_bounds__(256) stream_dual(const StreamArgs A) {
  const DevProblem &p = A.p;
  const R *dz = (const R *)A.dz;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < A.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    if (A.done[t]) continue;
    const R rho = R(A.rho_t[t]);
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    R s[NC], Tk[NC];
    const R T = R(p.durations[g]);
    inv_powers(T, s);
    Tk[0] = R(1);
#pragma unroll
    for (int q = 1; q < NC; ++q) Tk[q] = Tk[q - 1] * T;
    R rd2 = R(0);
#pragma unroll
    for (int a = 0; a < AX; ++a) {
      R dS[ND], dE[ND];
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * A.Jn;
        dS[r] = first ? R(0) : s[r] * dz[row + jS];
        dE[r] = last ? R(0) : s[r] * dz[row + jE];
      }
      rd2 += dual_residual_sq(dS, dE, rho, Tk);
    }
    A.rd2[x] = double(rd2);
  }
}

// The residual sums of Eq. 19-20 for the streaming trajectories, in FP64 and
// in a fixed order.  Block (t, c) sums chunk c (kReduceChunk segments) of
// trajectory t and stores the two chunk sums; the block that completes the
// trajectory's last chunk (an atomic ticket, no waiting) adds the chunk sums in
// chunk order, records the history and applies the stopping rule (Eq. 21).
// k >= 0: the iteration; k < 0: a periodic evaluation, the n-th of which (kept
// per trajectory in kcount) falls on iteration (n + 1) cev - 1, so the same
// launch serves every iteration of a recorded graph.
template <class R>
__global__ void __launch_bounds__(256) stream_reduce(const StreamArgs A, int k) {
  __shared__ double s1[256], s2[256];
  __shared__ int closing;
  const int t = blockIdx.x, c = blockIdx.y;
  if (t >= A.nl || A.done[t]) return;
  const int b = A.lt_b[t];
  const int x0 = A.lt_prefix[t], x1 = A.lt_prefix[t + 1];
  if (!TOP_IN_BOUNDS(A.p.err, b >= 0 && b < A.p.B && x0 >= 0 && x0 <= x1 && x1 <= A.total)) return;
  const int nch = max(1, (x1 - x0 + kReduceChunk - 1) / kReduceChunk);
  if (c >= nch) return;
  if (!TOP_IN_BOUNDS(A.p.err, nch <= A.nchunk)) return;
  const int c0 = x0 + c * kReduceChunk, c1 = min(x1, c0 + kReduceChunk);
  double a1 = 0.0, a2 = 0.0;
  for (int x = c0 + threadIdx.x; x < c1; x += blockDim.x) { a1 += A.rp2[x]; a2 += A.rd2[x]; }
  s1[threadIdx.x] = a1;
  s2[threadIdx.x] = a2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *pt = A.part + ((size_t)t * A.nchunk + c) * 2;
    pt[0] = s1[0];
    pt[1] = s2[0];
    __threadfence();  // the chunk sums are visible before the ticket is taken
    closing = atomicAdd(&A.ticket[t], 1) == nch - 1;
  }
  __syncthreads();
  if (!closing || threadIdx.x != 0) return;
  __threadfence();
  A.ticket[t] = 0;  // for the next evaluation
  const volatile double *pt = A.part + (size_t)t * A.nchunk * 2;
  double q1 = 0.0, q2 = 0.0;
  for (int q = 0; q < nch; ++q) { q1 += pt[2 * q]; q2 += pt[2 * q + 1]; }
  if (k < 0) {
    k = (A.kcount[t] + 1) * A.cev - 1;
    A.kcount[t] += 1;
  }
  const double rp = sqrt(q1), rd = sqrt(q2);
  A.tr_rp[t] = rp;
  A.tr_rd[t] = rd;
  if (A.r.history) {
    A.r.history[((size_t)k * A.p.B + b) * 2 + 0] = rp;
    A.r.history[((size_t)k * A.p.B + b) * 2 + 1] = rd;
  }
  const double tol = double(x1 - x0) * A.p.eps;
  int st = -1;
  if (!finite_d(rp) || !finite_d(rd)) st = 2;
  else if (A.p.eps > 0.0 && rp < tol && rd < tol) st = 0;
  if (st >= 0) {
    A.done[t] = 1;
    A.r.iters[b] = k + 1;
    A.r.status[b] = st;
  } else if (A.p.adaptive && A.E) {  // UpdateRho (Eq. 22)
    const double ro = A.rho_t[t], rn = next_rho(A.p, ro, rp, rd);
    A.fac_t[t] = ro / rn;
    A.rho_t[t] = rn;
  }
}

// after a change of rho (adaptive rho): every scaled dual times rho_old / rho_new
// (the unscaled duals are kept) and the segment's local inverse for the new rho
template <class R, int F>
__global__ void __launch_bounds__(256) stream_rescale(const StreamArgs A) {
  constexpr bool BOX = (F & FAM_BOX) != 0, BALL = (F & FAM_BALL) != 0, VN = (F & FAM_VN) != 0;
  const DevProblem &p = A.p;
  R *uL = (R *)A.uL, *uRp = (R *)A.uRp, *uR0 = (R *)A.uR0, *Gw = (R *)A.G;
  const bool pin = p.mode == 0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < A.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    if (A.done[t] || A.fac_t[t] == 1.0) continue;
    const R f = R(A.fac_t[t]);
    const bool first = i == 0, last = i == N - 1;
    const int jS = g + b, jE = g + b + 1;
    (void)jS;
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int r = 0; r < ND; ++r) {
        const size_t row = (size_t)(a * ND + r) * A.Jn;
        if (!last || r < PO) uL[row + jE] *= f;
        if (!last && pin && r == 0) uRp[(size_t)a * A.Jn + jE] *= f;
        if (first && r < PO) uR0[(size_t)(a * PO + r) * p.B + b] *= f;
      }
    if (BOX) {
      R *yb = (R *)A.ybox;
      for (int q = 0; q < 6 * p.M_box; ++q) {
        const R y = yb[(size_t)q * A.S + g];
        if (y > R(0)) yb[(size_t)q * A.S + g] = f * y;
      }
    }
    if (BALL) {
      const R o[3] = {R(p.ball_c[(size_t)g * 3]), R(p.ball_c[(size_t)g * 3 + 1]), R(p.ball_c[(size_t)g * 3 + 2])};
      for (int j = 0; j < p.M_ball; ++j)
        rescale_projected((R *)A.qball + (size_t)j * 3 * A.S + g, A.S, o, R(p.ball_r[g]), f);
    }
    if (VN) {
      const R zero3[3] = {R(0), R(0), R(0)};
      for (int j = 0; j < p.M_vn; ++j)
        rescale_projected((R *)A.qvn + (size_t)j * 3 * A.S + g, A.S, zero3, R(p.vnorm[b]), f);
    }
    g_from_eig_store((const R *)A.E, (size_t)A.S, (size_t)g, A.rho_t[t], Gw);
  }
}

template <class R>
__global__ void __launch_bounds__(256) stream_output(const StreamArgs A) {
  const DevProblem &p = A.p;
  const R *chg = (const R *)A.ch;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < A.total; x += gridDim.x * blockDim.x) {
    int t, b, i, N, g;
    if (!stream_locate(A, x, t, b, i, N, g)) continue;
    const double T = p.durations[g];
    double sd[NC];
    sd[0] = 1.0;
    for (int q = 1; q < NC; ++q) sd[q] = sd[q - 1] / T;
    R ch[AX][NC];
#pragma unroll
    for (int a = 0; a < AX; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        ch[a][q] = chg[(size_t)(a * NC + q) * A.S + g];
        A.r.coeffs[((size_t)g * AX + a) * NC + q] = double(ch[a][q]) * sd[q];
      }
    A.rp2[x] = segment_cost(ch, sd[7]);
  }
}

// per streaming trajectory: the cost (Eq. 4) summed like the residuals of
// stream_reduce (chunk sums, then the closing block in chunk order), the last
// residuals and the iteration count of a trajectory that did not stop
template <class R>
__global__ void __launch_bounds__(256) stream_finish(const StreamArgs A, int K) {
  __shared__ double s1[256];
  __shared__ int closing;
  const int t = blockIdx.x, c = blockIdx.y;
  if (t >= A.nl) return;
  const int b = A.lt_b[t];
  const int x0 = A.lt_prefix[t], x1 = A.lt_prefix[t + 1];
  if (!TOP_IN_BOUNDS(A.p.err, b >= 0 && b < A.p.B && x0 >= 0 && x0 <= x1 && x1 <= A.total)) return;
  const int nch = max(1, (x1 - x0 + kReduceChunk - 1) / kReduceChunk);
  if (c >= nch) return;
  if (!TOP_IN_BOUNDS(A.p.err, nch <= A.nchunk)) return;
  const int c0 = x0 + c * kReduceChunk, c1 = min(x1, c0 + kReduceChunk);
  double a1 = 0.0;
  for (int x = c0 + threadIdx.x; x < c1; x += blockDim.x) a1 += A.rp2[x];
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s1[threadIdx.x] += s1[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    A.part[((size_t)t * A.nchunk + c) * 2] = s1[0];
    __threadfence();
    closing = atomicAdd(&A.ticket[t], 1) == nch - 1;
  }
  __syncthreads();
  if (!closing || threadIdx.x != 0) return;
  __threadfence();
  A.ticket[t] = 0;
  const volatile double *pt = A.part + (size_t)t * A.nchunk * 2;
  double cost = 0.0;
  for (int q = 0; q < nch; ++q) cost += pt[2 * q];
  A.r.cost[b] = cost;
  A.r.r_primal[b] = A.tr_rp[t];
  A.r.r_dual[b] = A.tr_rd[t];
  if (A.r.rho) A.r.rho[b] = A.rho_t[t];
  if (!A.done[t]) {
    A.r.iters[b] = K;
    A.r.status[b] = 1;
  }
}

template <class R>
int run_stream_t(const StreamArgs &A, int fam, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (A.total == 0) return 0;
  const int threads = 256;
  int blocks = (A.total + threads - 1) / threads;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  const DevProblem &p = A.p;
  const int Mb = (fam & FAM_BOX) ? p.M_box : 0, Mq = (fam & FAM_BALL) ? p.M_ball : 0,
            Mv = (fam & FAM_VN) ? p.M_vn : 0;
  const int Mg = (fam & FAM_GEN) ? p.M_gen : 0;
  const int Mp = (fam & FAM_POLY) ? p.M_poly : 0;
  const size_t tab_bytes = sizeof(R) * 8 * (size_t)(Mb + Mq + Mv + 2 * Mg + Mp);
  void (*init)(const StreamArgs) = nullptr;
  void (*local)(const StreamArgs, int) = nullptr;
  void (*fused)(const StreamArgs, int) = nullptr;
  void (*rescale)(const StreamArgs) = nullptr;
  switch (fam) {
#define TOP_ST_CASE(FV)                                                                               \
  case FV:                                                                                            \
    init = stream_init<R, FV>; local = stream_local<R, FV>; fused = stream_local<R, FV | kFused>;     \
    rescale = stream_rescale<R, FV>;                                                                  \
    break;
    TOP_ST_CASE(0) TOP_ST_CASE(1) TOP_ST_CASE(2) TOP_ST_CASE(3)
    TOP_ST_CASE(4) TOP_ST_CASE(5) TOP_ST_CASE(6) TOP_ST_CASE(7) TOP_ST_CASE(8)
    TOP_ST_CASE(16) TOP_ST_CASE(17) TOP_ST_CASE(18) TOP_ST_CASE(19)
    TOP_ST_CASE(20) TOP_ST_CASE(21) TOP_ST_CASE(22) TOP_ST_CASE(23)
#undef TOP_ST_CASE
    default: return (int)cudaErrorInvalidValue;
  }
  if (fam == FAM_GEN && A.nwork) {  // the warp form
    local = stream_local<R, FAM_GEN | kDeferNumeric>;
    fused = stream_local<R, FAM_GEN | kDeferNumeric | kFused>;
  }
  long long nl = 1;  // kernel launches, for the handle's count
  if (A.seg_t) {
    stream_map<R><<<A.nl < 65535 ? A.nl : 65535, 256, 0, st>>>(A);
    nl += 1;
  }
  init<<<blocks, threads, 0, st>>>(A);
  const int K = p.max_iters;
  const bool adapt = p.adaptive && A.E;
  const int cev = adapt ? 1 : (p.check_every > 0 ? p.check_every : 1);
  const bool periodic = adapt || p.eps > 0.0 || A.r.history;
  StreamArgs Ak = A;
  Ak.cev = cev;
  // one iteration; `first` selects the Init-dependent local step, the
  // final iteration's evaluation names its k unless it is a periodic one
  const bool gen = (fam & FAM_GEN) != 0 && A.nwork;
  // the warp form's grid: as many blocks as are resident at once (8 warps each,
  // the warps stride over the work list); the blocks past the list's length
  // leave at once, so an iteration without violated bounds costs one short launch
  const size_t wsmem = sizeof(R) * (16 * (size_t)p.M_gen + 8 * 96);
  int wocc = 0;
  if (gen && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wocc, stream_numeric_warp<R>, 256, wsmem) != cudaSuccess)
    cudaGetLastError();
  int wblocks = sm_count() * (wocc > 0 ? wocc : 1);
  if (wblocks > (A.total + 7) / 8) wblocks = (A.total + 7) / 8;
  // Fused iterations: the junction update of an iteration without a residual
  // evaluation is applied at the start of the next iteration's local step
  // (stream_local<..., kFused>), which reads the junction state from one half
  // (ze) and the end values from one half (ee) and writes the other halves;
  // the numerical step's work list alternates between two counts (wc), the
  // one not in use cleared by stream_numeric_warp for the next iteration.
  const bool fuse = A.zB && A.uLB && A.uRpB && A.eSB && A.eEB;
  void *const Zh[2][3] = {{A.z, A.uL, A.uRp}, {A.zB, A.uLB, A.uRpB}};
  void *const Eh[2][2] = {{A.eS, A.eE}, {A.eSB, A.eEB}};
  int ze = 0, ee = 0, wc = 0;
  auto halves = [&](int zh, int eh) {
    StreamArgs a = Ak;
    a.z = Zh[zh][0]; a.uL = Zh[zh][1]; a.uRp = Zh[zh][2];
    a.eS = Eh[eh][0]; a.eE = Eh[eh][1];
    if (fuse && gen) { a.nwork = A.nwork + wc; a.nwork_next = A.nwork + (wc ^ 1); }
    return a;
  };
  auto iteration = [&](cudaStream_t s, int k, bool first) {
    const bool per = periodic && ((k + 1) % cev == 0);
    const bool check = per || (k == K - 1);
    // the previous iteration's junction update is pending unless that iteration evaluated residuals
    const bool pending = fuse && !first && !(periodic && k % cev == 0);
    const int eo = fuse ? (ee ^ 1) : 0;
    if (pending) {
      StreamArgs a = halves(ze, eo);
      a.zn = Zh[ze ^ 1][0]; a.uLn = Zh[ze ^ 1][1]; a.uRpn = Zh[ze ^ 1][2];
      a.eSp = Eh[ee][0]; a.eEp = Eh[ee][1];
      fused<<<blocks, threads, tab_bytes, s>>>(a, 1);
      ze ^= 1;
    } else {
      local<<<blocks, threads, tab_bytes, s>>>(halves(ze, eo), first ? 0 : 1);
    }
    ee = eo;
    const StreamArgs cur = halves(ze, ee);
    if (gen) stream_numeric_warp<R><<<wblocks, 256, wsmem, s>>>(cur);
    nl += gen ? 2 : 1;
    if (check || !fuse) {
      stream_junction<R><<<blocks, threads, 0, s>>>(cur, check ? 1 : 0);
      nl += 1;
    }
    if (check) {
      stream_dual<R><<<blocks, threads, 0, s>>>(cur);
      stream_reduce<R><<<dim3(Ak.nl, Ak.nchunk), 256, 0, s>>>(cur, per ? -1 : k);
      nl += 2;
    }
    if (adapt && k + 1 < K) {
      rescale<<<blocks, threads, 0, s>>>(cur);
      nl += 1;
    }
    if (fuse && gen) wc ^= 1;
  };
  int k = 0;
  if (K > 0) iteration(st, k++, true);
  // iterations 1 .. K-2 in blocks of G recorded once into a CUDA graph: the
  // launches of a block depend on the iteration only through the pattern of
  // evaluations, which repeats with period cev (G is a multiple of cev and
  // every block starts at k = 1 mod cev); with fused iterations G is a
  // multiple of 2 cev, so a block switches every half an even number of
  // times and each replay starts from the halves it was recorded with
  const int G = fuse ? 2 * cev * ((16 + cev - 1) / cev) : cev * ((32 + cev - 1) / cev);
  const int ze0 = ze, ee0 = ee, wc0 = wc;
  const int nblk = K >= 2 ? (K - 2) / G : 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (nblk >= 2 && A.kcount && cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const long long before = nl;
    if (ok) {
      for (int j = 0; j < G; ++j) iteration(cs, 1 + j, false);
      ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && graph != nullptr;
    }
    const long long per_replay = nl - before;  // recorded, not launched
    nl = before;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    bool launched = true;
    if (ok) {
      for (int q = 0; launched && q < nblk; ++q) {
        launched = cudaGraphLaunch(exec, st) == cudaSuccess;
        if (launched) nl += per_replay;
      }
      k = 1 + nblk * G;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    ze = ze0; ee = ee0; wc = wc0;  // recording switched them an even number of times, or stopped part-way
    if (!ok) cudaGetLastError();  // no graph: the direct launches below do every iteration
    if (!launched) return (int)cudaErrorLaunchFailure;  // a partly run graph cannot be resumed
  }
  for (; k < K; ++k) iteration(st, k, false);
  stream_output<R><<<blocks, threads, 0, st>>>(A);
  stream_finish<R><<<dim3(A.nl, A.nchunk), 256, 0, st>>>(A, K);
  if (A.launches) *A.launches += nl + 2;
  return (int)cudaGetLastError();
}

}  // namespace top
