// top_internal.h -- argument blocks shared by the host driver and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

namespace top {

enum Family : int { FAM_BOX = 1, FAM_BALL = 2, FAM_VN = 4, FAM_GEN = 8, FAM_POLY = 16 };

// A pack is a set of whole trajectories processed by one CTA of the
// resident kernel (all of its state stays in shared memory for every
// iteration); its trajectories are traj_list[tlist .. tlist+ntraj-1].
struct Pack {
  int tlist;  // first entry in the trajectory list
  int nseg;   // segments in the pack (<= CTA capacity)
  int ntraj;  // trajectories in the pack
  int pad;
};

// Problem data, all device pointers (FP64, the ABI layout).
struct DevProblem {
  int B, S;
  const int32_t *seg_offset;
  const double *waypoints, *durations, *start_state, *end_state;
  int mode;       // 0 pin, 1 free
  int inner;      // 0 closed form, 1 numeric
  double rho, eps;
  int max_iters, check_every;
  int M_box;  const double *vbox;
  int M_ball; const double *ball_c, *ball_r;
  int M_vn;   const double *vnorm;
  int M_gen;  const double *gen_vmax, *gen_amax;
  int lbfgs_mem, lbfgs_max_iters;
  double lbfgs_tol;
  int adaptive;   // residual balancing of rho (Eq. 22)
  double rho_mu, rho_incr, rho_decr;
  int M_poly, F_poly; const double *poly_n, *poly_h;  // polytope corridors
  int *err;       // error word: 1 invalid input, 2 not positive definite, 4 bounds (checked build)
  int stall;      // stall rule: checks in which neither residual fell 1 % below its best before TOP_STALLED (0 = off)
};

// Bounds checks of the checked build (TOP_CHECKED, libtop_checked.so): every
// kernel checks the index bases it derives (pack, trajectory, segment, slot)
// against the sizes of the arrays they address; every other access is a
// compile-time-bounded offset from one of them.  A failed check sets bit 4 of
// the error word and the thread skips its accesses (the host then returns
// TOP_E_BOUNDS).  In the regular build the checks compile to nothing.
#ifdef TOP_CHECKED
__device__ __forceinline__ bool top_in_bounds(int *err, bool ok) {
  if (!ok && err) atomicOr(err, 4);
  return ok;
}
#define TOP_IN_BOUNDS(err, cond) top_in_bounds((err), (cond))
#else
#define TOP_IN_BOUNDS(err, cond) true
#endif

struct DevResult {
  double *coeffs, *cost, *r_primal, *r_dual, *history;
  int32_t *iters, *status;
  double *rho;          // [B] final rho, or null
};

// Per-segment data that rebuilds the local-matrix inverse for any rho
// (adaptive rho): K(rho) = 2 T^-7 Qh + rho H in the normalised basis, and
//   G(rho) = K(rho)^{-1} = A0 / rho + sum_{k<4} y_k y_k^T / (lambda_k + rho)
// with A0 supported on the top-left 4x4 block (packed lower, 10 values),
// Y = [y_0 .. y_3] (8 x 4, row-major) and lambda_k >= 0.  Layout [NE][S].
constexpr int NE_A0 = 0, NE_Y = 10, NE_L = 42, NE = 46;

// Per-segment data of the polytope family, element type = iteration type,
// layout [rows][S]: with N3 = sum_f n_f n_f^T = U diag(nu) U^T, the local
// matrix is block diagonal in the rotated axes c~_b = sum_a U[a][b] c_a:
//   PG: [3 * 36]  packed inverses of K8 + rho nu_b B_pos, one per rotated axis b
//   PU: [9]       U[a][b] at row a * 3 + b
//   PN: [3 F]     normals, row f * 3 + a;   PH: [F] offsets
struct PolyData {
  void *G, *U, *N, *H;
};

// Iteration state in the ABI's layout (top_state of top.h), device pointers:
// p, m [S+B][3][7] consensus targets at every junction (start side, end side),
// ybox [S][6 M_box], qball [S][M_ball][3], qvn [S][M_vn][3], iters [B].
// p == nullptr: no state (Init of Algorithm 1 / no export).
struct StateView {
  double *p, *m, *ybox, *qball, *qvn;
  int32_t *iters;
};

struct ResidentArgs {
  DevProblem p;
  DevResult r;
  StateView from, to;   // resume from / export to (top_resume), or null views
  const void *G;        // [36][S] packed (D K D)^{-1}, element type = iteration type
  const void *E;        // [NE][S] adaptive-rho data (same type), or null
  const Pack *packs;
  const int *traj_list; // trajectory ids, grouped by pack
  int ntp;              // trajectory slots per pack (shared-memory sizing)
  int tc;               // 1: the G product of warps that share one inverse on the tensor cores
  double *stall;        // [B][3] stall-rule state (best ||r_p||, best ||r_d||, checks since), or null
};

// Cluster-resident form (top_cluster.cuh): one trajectory per thread-block
// cluster, CTA rank r owning segments r*C .. r*C + C - 1.
struct ClusterArgs {
  DevProblem p;
  DevResult r;
  StateView from, to;   // resume from / export to (top_resume), or null views
  const void *G;        // [36][S], element type = iteration type (rewritten on a change of rho)
  const void *E;        // [NE][S] adaptive-rho data, or null
  const int *traj;      // [nclusters] trajectory ids
  PolyData poly;        // polytope family (FAM_POLY), else null pointers
  void *ypoly;          // [F_poly M_poly][S] compressed slack / dual of the polytope rows
};
constexpr int kClusterNtp = 8;  // res_layout's trajectory slots for the cluster form (room for its shares)

// Shared-memory layout of the resident kernel; the same function sizes the
// launch on the host and carves the buffer on the device.
struct ResLayout {
  size_t red_rp, red_rd, tr_rp, tr_rd;           // double arrays
  size_t p, m, zP, eS, dz, ybox, qball, qvn, tabB, tabQ, tabV, tabP, ch;  // element arrays
  size_t off, done, tid, flag, ndone;            // int arrays (ndone: trajectories of the pack stopped)
  size_t rho, fac;                               // double arrays (per trajectory)
  size_t total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// mreg (the resident kernel): the end-side targets of a segment's end slot
// live in its thread's registers, so m holds only the start slots of the
// pack's trajectories ([trajectory][21]); the coefficients of check
// iterations are kept in ch ([24][C]) for the output; with tc (the tensor-core
// form of the G product) ch is [C][28], one row per segment, and doubles as
// the warps' operand scratch.
__host__ __device__ inline ResLayout res_layout(int C, int ntp, int Mb, int Mq, int Mv, int rb, int Mp = 0,
                                                bool mreg = false, bool tc = false) {
  ResLayout L{};
  const size_t J = size_t(C) + size_t(ntp);
  size_t o = 0;
  L.red_rp = o; o += sizeof(double) * C;
  L.red_rd = o; o += sizeof(double) * C;
  L.tr_rp = o;  o += sizeof(double) * ntp;
  L.tr_rd = o;  o += sizeof(double) * ntp;
  o = align_up(o, 16);
  L.p = o;      o += size_t(rb) * 21 * J;  // [slot][21] start-side targets
  L.m = o;      o += size_t(rb) * 21 * (mreg ? size_t(ntp) : J);  // [slot][21] end-side targets
  L.zP = o;     o += size_t(rb) * 3 * J;   // [slot][3] pinned positions
  L.eS = o;     o += size_t(rb) * 21 * C;  // [segment][21] published start derivatives
  L.dz = o;     o += size_t(rb) * 21 * J;  // [slot][21] consensus change (check iterations)
  L.ybox = o;   o += size_t(rb) * 6 * Mb * C;
  L.qball = o;  o += size_t(rb) * 3 * Mq * C;
  L.qvn = o;    o += size_t(rb) * 3 * Mv * C;
  o = align_up(o, 16);  // table rows are read as 16-byte vectors
  L.tabB = o;   o += size_t(rb) * 8 * Mb;
  L.tabQ = o;   o += size_t(rb) * 8 * Mq;
  L.tabV = o;   o += size_t(rb) * 8 * Mv;
  L.tabP = o;   o += size_t(rb) * 8 * Mp;  // polytope sample rows (cluster form)
  L.ch = o;     o += mreg ? size_t(rb) * (tc ? 28 : 24) * C : 0;
  o = align_up(o, 16);
  L.off = o;    o += sizeof(int) * (ntp + 1);
  L.done = o;   o += sizeof(int) * ntp;
  L.tid = o;    o += sizeof(int) * ntp;
  L.flag = o;   o += sizeof(int);
  L.ndone = o;  o += sizeof(int);
  o = align_up(o, 8);
  L.rho = o;    o += sizeof(double) * ntp;
  L.fac = o;    o += sizeof(double) * ntp;
  L.total = align_up(o, 16);
  return L;
}

// the layout of the resident kernel (top_resident.cuh); at 512 FP32 segments
// with 128 trajectory slots and no sample rows it takes 231,952 of the
// 232,448 bytes a CTA may opt in to (tests/test_parity_gpu.py checks it fits)
__host__ __device__ inline ResLayout res_layout_resident(int C, int ntp, int Mb, int Mq, int Mv, int rb,
                                                         bool tc = false) {
  return res_layout(C, ntp, Mb, Mq, Mv, rb, 0, true, tc);
}

// segments per block of the streaming residual sums (stream_reduce)
constexpr int kReduceChunk = 2048;

// Streaming form (trajectories longer than a resident CTA): state in global
// memory.  Compact segment index x over the streaming trajectories:
// lt_prefix[t] .. lt_prefix[t+1]-1 belong to trajectory lt_b[t].
struct StreamArgs {
  DevProblem p;
  DevResult r;
  const void *G;           // [36][S] (rewritten on a change of rho)
  const void *E;           // [NE][S] adaptive-rho data, or null
  PolyData poly;           // polytope family (FAM_POLY), else null pointers
  const int *lt_b;         // [nl]
  const int *lt_prefix;    // [nl+1]
  int *seg_t;              // [total] streaming trajectory of each compact index, filled by stream_map (or null:
                           // the kernels search lt_prefix)
  int nl, total;           // trajectories, segments in the streaming set
  int S, Jn;               // global segments, global junctions (S + B)
  // state, element type = iteration type; junction arrays indexed like the waypoints
  void *z, *uL, *dz;       // [21][Jn]
  void *uRp;               // [3][Jn]
  void *uR0;               // [12][B]
  void *eS, *eE;           // [21][S]
  void *ch;                // [24][S]
  void *ybox, *qball, *qvn;  // [6 M_box][S], [3 M_ball][S], [3 M_vn][S]
  void *ygen;              // [2 M_gen][S] numerical-step duals (velocity, acceleration)
  void *ypoly;             // [F_poly M_poly][S] compressed slack / dual of the polytope rows, row j * F + f
  int *inner_iters;        // [S] L-BFGS iterations summed over the run (numerical step), or null
  double *rp2, *rd2;       // [total]
  int *done;               // [nl]
  double *tr_rp, *tr_rd;   // [nl]
  double *rho_t, *fac_t;   // [nl] current rho, rescale factor of the last update
  int *kcount;             // [nl] periodic residual evaluations so far (or null)
  int cev;                 // iterations between periodic evaluations
  int *nwork, *work;       // numerical step: count and compact indices of segments with a violated bound
  // fused iterations (top_config.stream_form): the second halves of the junction state z, uL, uRp and of
  // the end values eS, eE (null: one launch per phase); a fused local step reads the previous iteration's
  // end values from eSp, eEp and the junction state from z, uL, uRp, and writes the state after the
  // previous iteration's junction update to zn, uLn, uRpn
  void *zB, *uLB, *uRpB, *eSB, *eEB;
  void *zn, *uLn, *uRpn;
  const void *eSp, *eEp;
  int *nwork_next;         // fused iterations: the next iteration's work-list count, cleared by stream_numeric_warp
  double *part;            // [nl][nchunk][2] residual sums per chunk of kReduceChunk segments (or null)
  int *ticket;             // [nl] chunks of the current evaluation summed so far (or null)
  int nchunk;              // chunks of the longest streaming trajectory
  long long *launches;     // host counter of kernel launches (or null); never read on the device
};

// A kernel attribute set once per (device, kernel, value): cudaFuncSetAttribute
// is not a stream operation, so launches that only repeat known settings stay
// free of it (and can be recorded in a CUDA graph).
inline cudaError_t func_attr_once(const void *kern, cudaFuncAttribute attr, int value) {
  static std::mutex mu;
  static const void *keys[512];
  static int devs[512], attrs[512], vals[512];
  static int n = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  int slot = -1;
  for (int i = 0; i < n; ++i)
    if (keys[i] == kern && devs[i] == dev && attrs[i] == (int)attr) {
      if (vals[i] >= value) return cudaSuccess;
      slot = i;
    }
  const cudaError_t e = cudaFuncSetAttribute(kern, attr, value);
  if (e != cudaSuccess) return e;
  if (slot < 0 && n < 512) slot = n++;
  if (slot >= 0) { keys[slot] = kern; devs[slot] = dev; attrs[slot] = (int)attr; vals[slot] = value; }
  return cudaSuccess;
}

// Streaming multiprocessors of the current device (grid-stride kernels cap
// their grids at a multiple of it); queried once per device.
inline int sm_count() {
  static int counts[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 128;  // any count > 0 is correct
  if (counts[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 128;
    counts[dev] = n;
  }
  return counts[dev];
}

// launchers (defined in the .cu files)
// copy (optional, [2S + 1] ints of workspace): reuse the inverse of the first
// interior segment for interior segments of the same duration
int launch_kinv(const DevProblem &p, double rho, void *G32, void *G64, int *err_flag, void *stream,
                int *copy = nullptr);
int launch_keig(const DevProblem &p, void *E32, void *E64, int *err_flag, void *stream);
int launch_kinv_poly(const DevProblem &p, double rho, bool fp64, const PolyData &out, int *err_flag, void *stream);
int launch_fill(double *x, int n, double v, void *stream);
int launch_sample(const int32_t *off, const double *T, int B, int M, int order, const double *coeffs,
                  double *tstart, double *ttot, double *out, void *stream);
int launch_time_step(double *T, const double *dT, int S, double kT, double lr, void *stream);
int launch_resident_f32(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream);
int launch_resident_f64(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream);
int launch_resident_stall_f32(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream);
int launch_resident_stall_f64(const ResidentArgs &a, int nblocks, int C, size_t smem, int fam, void *stream);
// C segments per CTA, ln lanes per segment (blockDim = C * ln; ln > 1: FP32, fixed rho, families 1-7)
int launch_cluster_f32(const ClusterArgs &a, int nclusters, int csz, int C, int ln, size_t smem, int fam,
                       void *stream);
int launch_cluster_f64(const ClusterArgs &a, int nclusters, int csz, int C, int ln, size_t smem, int fam,
                       void *stream);
void *cluster_lanes_kernel_f32(int fam, int ln);
void *cluster_lanes2_kernel_f32(int fam);
void *cluster_lanes4_kernel_f32(int fam);
// largest cluster size (power of two <= 16) whose CTAs of C threads and `smem`
// bytes can be co-scheduled, 0 if none
int cluster_max_size(int C, int ln, size_t smem, int fam, bool fp64);
int cluster_max_size_f32(int C, int ln, size_t smem, int fam);
int cluster_max_size_f64(int C, int ln, size_t smem, int fam);
int launch_stream_f32(const StreamArgs &a, int fam, void *stream);
int launch_stream_f64(const StreamArgs &a, int fam, void *stream);
// Adjoint of the unrolled iteration (top_grad)
struct AdjArgs {
  StreamArgs f;              // forward views (segment list, problem, G)
  const void *tz, *tuL, *tuRp, *tuR0;  // x^k from the tape
  const void *tyb, *tqb, *tqv;         // x^k from the tape: box / ball / velocity-norm states ([rows][S])
  void *ybb, *qbb, *qvb;               // their adjoints ([rows][S])
  void *zb, *uLb, *uRb;      // [21][Jn] adjoint of the junction state
  void *uR0b;                // [12][B]
  void *eSb, *eEb;           // [21][S] adjoint of the end derivatives
  void *wbS, *wbE;           // [21][S] adjoint of the targets
  double *Tbar;              // [S]
  double *Pbar;              // [Jn][3]
  const double *dJ;          // [B]
};
// Resident adjoint (top_adjres.cuh): packs of whole trajectories, fixed rho,
// closed-form step without inequality rows.
struct AdjResArgs {
  DevProblem p;
  const void *G;          // [36][S] packed local inverses (iteration type)
  const Pack *packs;
  const int *traj_list;
  int ntp;                // trajectory slots per pack
  int ckpt;               // checkpoint interval in iterations
  int Jn;                 // global junction slots, S + B
  void *ck;               // [ceil(K / ckpt)][2][21][Jn] checkpoints of the slot state (p, m)
  void *tape;             // [ckpt][2][21][Jn] the slot state entering each iteration of a block
  const double *dJ;       // [B] cost seeds
  double *dw;             // [Jn][3] dJ/d(waypoints) (interior junctions written, others left)
  double *dT;             // [S] dJ/d(durations)
};
struct AdjResLayout {
  size_t p, m, pb, mb, zP, eS, off, tid, total;
};
__host__ __device__ inline AdjResLayout adjres_layout(int C, int ntp, int rb) {
  AdjResLayout L{};
  const size_t J = size_t(C) + size_t(ntp);
  size_t o = 0;
  L.p = o;   o += size_t(rb) * 21 * J;   // [slot][21] forward targets p, m and their adjoints
  L.m = o;   o += size_t(rb) * 21 * J;
  L.pb = o;  o += size_t(rb) * 21 * J;
  L.mb = o;  o += size_t(rb) * 21 * J;
  L.zP = o;  o += size_t(rb) * 3 * J;
  L.eS = o;  o += size_t(rb) * 21 * size_t(C);
  o = align_up(o, 16);
  L.off = o; o += sizeof(int) * (ntp + 1);
  L.tid = o; o += sizeof(int) * ntp;
  L.total = align_up(o, 16);
  return L;
}
int launch_adjres_f32(const AdjResArgs &a, int nblocks, int C, size_t smem, void *stream);
int launch_adjres_f64(const AdjResArgs &a, int nblocks, int C, size_t smem, void *stream);
// the streaming adjoint; fam: FAM_BOX / FAM_BALL / FAM_VN bits (closed-form step);
// ck[c * 7 + q], tape[l * 7 + q]: copies of the arrays (z, uL, uRp, uR0, ybox,
// qball, qvn) of bytes[q] bytes (0 for an absent family)
int launch_adjoint_f32(const StreamArgs &f, const AdjArgs &a, int fam, int ckpt, void *const *ck, void *const *tape,
                       const size_t *bytes, double *dw, double *dT, void *stream);
int launch_adjoint_f64(const StreamArgs &f, const AdjArgs &a, int fam, int ckpt, void *const *ck, void *const *tape,
                       const size_t *bytes, double *dw, double *dT, void *stream);

}  // namespace top
