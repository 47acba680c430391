// top_api.cu -- host driver behind the C ABI of include/top.h: argument
// validation, workspace ownership, batch planning (packing trajectories into
// resident CTAs, routing long ones to the streaming kernels) and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/top.h"
#include "top_internal.h"
#include "top_math.cuh"

using namespace top;

namespace {
// NVTX range for profilers (header-only NVTX; a no-op unless a tool is attached)
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

struct top_handle {
  top_config cfg{};
  long long launches = 0;  // kernels launched by top_solve (top_launch_count)
  int device = 0;
  int sm_count = 0;
  int smem_optin = 0;
  int last_cuda = 0;
  // device workspace
  void *G = nullptr;          // [36][max_segments] of the iteration type
  void *E = nullptr;          // [NE][S] adaptive-rho data (allocated on first use)
  size_t E_bytes = 0;
  void *P = nullptr;          // polytope family data (PolyData), allocated on first use
  size_t P_bytes = 0;
  unsigned char *d_pstage = nullptr;  // staging of host polytope arrays
  size_t pstage_bytes = 0;
  unsigned char *d_aux = nullptr;     // top_sample / top_time_alloc workspace (grow-only)
  size_t aux_bytes = 0;
  int *d_copy = nullptr;              // [2 max_segments + 1]: shared-duration reuse map and inversion list
  void *d_ypoly = nullptr;            // polytope slack state of the cluster form (grow-only)
  size_t ypoly_bytes = 0;
  // the cluster-resident launches run on a side stream, concurrently with the
  // resident packs (they share only the precompute, which both wait for)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  Pack *d_packs = nullptr;    // [max_segments]
  int *d_err = nullptr;       // error flag of the precompute kernel
  double *d_stall = nullptr;  // [max_batch][3] stall-rule state of the resident kernel
  // staging for TOP_MEM_HOST problems
  unsigned char *d_stage = nullptr;
  size_t stage_bytes = 0;
  // pinned host memory
  int32_t *h_off = nullptr;   // [max_batch + 1]
  Pack *h_packs = nullptr;    // [max_segments]
  int *h_lt = nullptr;        // [2 * max_batch + 1] streaming trajectory list and prefix
  // resident plan (packs + trajectory list), reused while the batch layout repeats
  int *h_tlist = nullptr;     // [max_batch]
  int *d_tlist = nullptr;     // [max_batch]
  int32_t *plan_off = nullptr;  // [max_batch + 1] layout the plan was made for
  bool plan_valid = false;
  int plan_B = -1, plan_cap = -1, plan_npack = 0, plan_max_nseg = 0, plan_max_ntraj = 0;
  bool plan_has_long = false;
  int *h_err = nullptr;
  // streaming-form workspace (allocated on first use)
  unsigned char *d_stream = nullptr;
  size_t stream_bytes = 0;
  // kernel timing (top_set_profiling)
  bool profiling = false;
  cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool ran[4] = {false, false, false, false};
  // cluster-resident form: trajectory lists (pinned host, device) and the cached
  // largest co-schedulable cluster size for (C, family, precision)
  int *h_ctraj = nullptr, *d_ctraj = nullptr;  // [max_batch]
  int csz_key_C[4] = {-1, -1, -1, -1}, csz_key_fam[4] = {-1, -1, -1, -1}, csz_val[4] = {0, 0, 0, 0};  // per lanes group
  size_t csz_key_smem[4] = {0, 0, 0, 0};
  // top_resume with host memory: device copies of the states (grow-only)
  unsigned char *d_ws = nullptr;
  size_t ws_bytes = 0;
  // capture-safe mode (top_set_layout): host copy of the batch layout
  int layout_B = 0;
  int32_t *layout_off = nullptr;  // [max_batch + 1]
};

namespace {

int cuda_fail(top_handle *h, cudaError_t e) {
  if (h) h->last_cuda = (int)e;
  return TOP_E_CUDA;
}

#define TOP_CUDA(h, expr)                              \
  do {                                                 \
    cudaError_t e__ = (expr);                          \
    if (e__ != cudaSuccess) return cuda_fail(h, e__);  \
  } while (0)

size_t rbytes(const top_handle *h) { return h->cfg.precision == TOP_FP64 ? 8 : 4; }

// grow-only device buffer; cudaSuccess or the allocation's error (sticky errors cleared)
cudaError_t grow(void **ptr, size_t *cap, size_t want) {
  if (want <= *cap) return cudaSuccess;
  cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return e;
  }
  *cap = want;
  return cudaSuccess;
}

int families(const top_problem *pb) {
  int f = 0;
  if (pb->inner == TOP_CLOSED_FORM) {
    if (pb->M_box > 0) f |= FAM_BOX;
    if (pb->M_ball > 0) f |= FAM_BALL;
    if (pb->M_vn > 0) f |= FAM_VN;
    if (pb->M_poly > 0) f |= FAM_POLY;
  } else if (pb->M_gen > 0) {
    f |= FAM_GEN;
  }
  return f;
}

// largest resident capacity (threads = segments per CTA, multiple of 32, <= 512)
// whose shared-memory layout fits the device's opt-in limit
// threads per CTA of the resident and cluster kernels: 512, or 256 with FP64 state
int max_cta_threads(const top_handle *h) { return h->cfg.precision == TOP_FP64 ? 256 : 512; }

int resident_capacity(const top_handle *h, const top_problem *pb) {
  const int fam = families(pb);
  const int Mb = (fam & FAM_BOX) ? pb->M_box : 0;
  const int Mq = (fam & FAM_BALL) ? pb->M_ball : 0;
  const int Mv = (fam & FAM_VN) ? pb->M_vn : 0;
  const int tmax = max_cta_threads(h);
  int cap = h->cfg.segs_per_cta > 0 ? std::min(tmax, h->cfg.segs_per_cta / 32 * 32) : tmax;
  for (int C = cap; C >= 32; C -= 32) {
    ResLayout L = res_layout_resident(C, C / 4, Mb, Mq, Mv, (int)rbytes(h));
    if (L.total <= (size_t)h->smem_optin) return C;
  }
  return 0;
}

// per-CTA capacity of the cluster-resident form (one trajectory per cluster)
int cluster_capacity(const top_handle *h, const top_problem *pb) {
  const int fam = families(pb);
  const int Mb = (fam & FAM_BOX) ? pb->M_box : 0;
  const int Mq = (fam & FAM_BALL) ? pb->M_ball : 0;
  const int Mv = (fam & FAM_VN) ? pb->M_vn : 0;
  const int tmax = max_cta_threads(h);
  int cap = h->cfg.segs_per_cta > 0 ? std::min(tmax, h->cfg.segs_per_cta / 32 * 32) : tmax;
  const int Mp = (fam & FAM_POLY) ? pb->M_poly : 0;
  for (int C = cap; C >= 32; C -= 32) {
    ResLayout L = res_layout(C, kClusterNtp, Mb, Mq, Mv, (int)rbytes(h), Mp);
    if (L.total <= (size_t)h->smem_optin) return C;
  }
  return 0;
}

// Best-fit-decreasing packing of the trajectories that fit one resident CTA
// (N_b <= cap) into packs of at most `cap` segments and `ntp_cap`
// trajectories.  Trajectories longer than `cap` are left for the streaming
// form (has_long).  Writes packs[] and the trajectory list grouped by pack.
void plan_packs(const int32_t *off, int B, int cap, int ntp_cap, Pack *packs, int *tlist, int &npack,
                int &max_nseg, int &max_ntraj, bool &has_long) {
  npack = max_nseg = max_ntraj = 0;
  has_long = false;
  if (cap <= 0) {
    for (int b = 0; b < B; ++b)
      if (off[b + 1] > off[b]) has_long = true;
    // empty trajectories need no kernel: their outputs are zeroed by the caller
    return;
  }
  // counting sort by length, longest first
  std::vector<int> cnt(cap + 2, 0), order;
  order.reserve(B);
  for (int b = 0; b < B; ++b) {
    const int nb = off[b + 1] - off[b];
    if (nb > cap) { has_long = true; continue; }
    ++cnt[nb];
  }
  std::vector<int> start(cap + 2, 0);
  for (int n = cap; n >= 0; --n) start[n] = (n == cap ? 0 : start[n + 1] + cnt[n + 1]);
  int packable = 0;
  for (int n = 0; n <= cap; ++n) packable += cnt[n];
  order.assign(packable, 0);
  for (int b = 0; b < B; ++b) {
    const int nb = off[b + 1] - off[b];
    if (nb <= cap) order[start[nb]++] = b;
  }
  // bins indexed by remaining room; a bitset of non-empty room buckets
  std::vector<int> room, ntraj, nseg, bin_of(B, -1);
  std::vector<std::vector<int>> bucket(cap + 1);
  const int words = cap / 64 + 1;
  std::vector<uint64_t> live(words, 0);
  auto push = [&](int r, int bin) {
    bucket[r].push_back(bin);
    live[r >> 6] |= (1ull << (r & 63));
  };
  auto find_at_least = [&](int n) -> int {
    for (int w = n >> 6; w < words; ++w) {
      uint64_t m = live[w];
      if (w == (n >> 6)) m &= ~0ull << (n & 63);
      if (m) return (w << 6) + __builtin_ctzll(m);
    }
    return -1;
  };
  for (int b : order) {
    const int nb = off[b + 1] - off[b];
    int r = find_at_least(nb);
    int bin;
    if (r >= 0 && r <= cap) {
      bin = bucket[r].back();
      bucket[r].pop_back();
      if (bucket[r].empty()) live[r >> 6] &= ~(1ull << (r & 63));
    } else {
      bin = (int)room.size();
      room.push_back(cap);
      ntraj.push_back(0);
      nseg.push_back(0);
    }
    room[bin] -= nb;
    nseg[bin] += nb;
    ntraj[bin] += 1;
    bin_of[b] = bin;
    if (ntraj[bin] < ntp_cap) push(room[bin], bin);
  }
  npack = (int)room.size();
  // trajectory list grouped by pack (ascending trajectory id inside a pack)
  std::vector<int> pos(npack + 1, 0);
  for (int q = 0; q < npack; ++q) pos[q + 1] = pos[q] + ntraj[q];
  for (int q = 0; q < npack; ++q) {
    packs[q] = Pack{pos[q], nseg[q], ntraj[q], 0};
    max_nseg = std::max(max_nseg, nseg[q]);
    max_ntraj = std::max(max_ntraj, ntraj[q]);
  }
  for (int b = 0; b < B; ++b)
    if (bin_of[b] >= 0) tlist[pos[bin_of[b]]++] = b;
}

struct StagePlan {
  size_t off_seg, off_wp, off_T, off_s0, off_s1, off_vbox, off_bc, off_br, off_vn, off_gv, off_ga;
  size_t off_coef, off_cost, off_rp, off_rd, off_it, off_st, off_rho, total;
};

StagePlan stage_plan(int Bmax, int Smax) {
  StagePlan P{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
  P.off_seg = take(sizeof(int32_t) * (Bmax + 1));
  P.off_wp = take(sizeof(double) * 3 * (size_t)(Smax + Bmax));
  P.off_T = take(sizeof(double) * Smax);
  P.off_s0 = take(sizeof(double) * 12 * (size_t)Bmax);
  P.off_s1 = take(sizeof(double) * 12 * (size_t)Bmax);
  P.off_vbox = take(sizeof(double) * Bmax);
  P.off_bc = take(sizeof(double) * 3 * (size_t)Smax);
  P.off_br = take(sizeof(double) * Smax);
  P.off_vn = take(sizeof(double) * Bmax);
  P.off_gv = take(sizeof(double) * Bmax);
  P.off_ga = take(sizeof(double) * Bmax);
  P.off_coef = take(sizeof(double) * 24 * (size_t)Smax);
  P.off_cost = take(sizeof(double) * Bmax);
  P.off_rp = take(sizeof(double) * Bmax);
  P.off_rd = take(sizeof(double) * Bmax);
  P.off_it = take(sizeof(int32_t) * Bmax);
  P.off_st = take(sizeof(int32_t) * Bmax);
  P.off_rho = take(sizeof(double) * Bmax);
  P.total = o;
  return P;
}

int validate(const top_handle *h, const top_problem *pb, const top_result *res) {
  if (!h || !pb || !res) return TOP_E_INVAL;
  if (pb->B < 0 || pb->B > h->cfg.max_batch) return pb->B < 0 ? TOP_E_INVAL : TOP_E_NOMEM;
  if (pb->memory != TOP_MEM_DEVICE && pb->memory != TOP_MEM_HOST) return TOP_E_INVAL;
  if (pb->mode != TOP_PIN && pb->mode != TOP_FREE) return TOP_E_INVAL;
  if (pb->inner != TOP_CLOSED_FORM && pb->inner != TOP_NUMERIC) return TOP_E_INVAL;
  if (!(pb->rho > 0.0) || !(pb->rho < 1e300)) return TOP_E_INVAL;
  if (!(pb->eps >= 0.0)) return TOP_E_INVAL;
  if (pb->max_iters < 0 || pb->check_every < 0 || pb->stall_checks < 0) return TOP_E_INVAL;
  if (pb->M_box < 0 || pb->M_ball < 0 || pb->M_vn < 0 || pb->M_gen < 0) return TOP_E_INVAL;
  const int mmax = std::max(std::max(pb->M_box, pb->M_ball), std::max(pb->M_vn, pb->M_gen));
  if (mmax > h->cfg.max_samples) return TOP_E_NOMEM;
  if (pb->M_box > 0 && !pb->vbox) return TOP_E_INVAL;
  if (pb->M_ball > 0 && (!pb->ball_c || !pb->ball_r)) return TOP_E_INVAL;
  if (pb->M_vn > 0 && !pb->vnorm) return TOP_E_INVAL;
  if (pb->M_gen > 0 && (!pb->gen_vmax || !pb->gen_amax)) return TOP_E_INVAL;
  if (pb->inner == TOP_NUMERIC && (pb->M_box || pb->M_ball || pb->M_vn)) return TOP_E_NOTSUP;
  if (pb->inner == TOP_CLOSED_FORM && pb->M_gen) return TOP_E_NOTSUP;
  if (pb->M_poly < 0 || (pb->M_poly > 0 && (pb->F_poly < 1 || !pb->poly_n || !pb->poly_h))) return TOP_E_INVAL;
  if (pb->M_poly > h->cfg.max_samples) return TOP_E_NOMEM;
  if (pb->M_poly > 0 && (pb->inner != TOP_CLOSED_FORM || pb->adaptive_rho)) return TOP_E_NOTSUP;
  if (pb->adaptive_rho != 0 && pb->adaptive_rho != 1) return TOP_E_INVAL;
  if (pb->adaptive_rho) {
    for (double v : {pb->rho_mu, pb->rho_tau_incr, pb->rho_tau_decr})
      if (v != 0.0 && !(v >= 1.0 && std::isfinite(v))) return TOP_E_INVAL;
  }
  if (pb->B > 0 && (!pb->seg_offset || !pb->waypoints || !pb->start_state || !pb->end_state))
    return TOP_E_INVAL;
  if (pb->B > 0 && (!res->cost || !res->r_primal || !res->r_dual || !res->iters || !res->status))
    return TOP_E_INVAL;  // coeffs is checked once S is known (it may be empty)
  return TOP_OK;
}

}  // namespace

extern "C" {

const char *top_strerror(int code) {
  switch (code) {
    case TOP_OK: return "success";
    case TOP_E_INVAL: return "invalid argument";
    case TOP_E_NOMEM: return "out of workspace memory or batch above the handle's capacity";
    case TOP_E_CUDA: return "CUDA runtime error";
    case TOP_E_TIMEOUT: return "bounded device wait timed out";
    case TOP_E_NOTSUP: return "unsupported combination of options";
    case TOP_E_STATE: return "call out of order";
    case TOP_E_NUMERIC: return "local KKT matrix not positive definite";
    case TOP_E_LIMIT: return "problem larger than the fixed scratch of top_solve_noalloc";
    case TOP_E_BOUNDS: return "an index outside its array (bounds-checked build)";
    default: return "unknown error code";
  }
}

int top_last_cuda_error(const top_handle *h) { return h ? h->last_cuda : 0; }

int64_t top_launch_count(const top_handle *h) { return h ? (int64_t)h->launches : -1; }

int top_set_profiling(top_handle *h, int enable) {
  if (!h) return TOP_E_INVAL;
  if (enable && !h->ev[0]) {
    for (auto &e : h->ev) {
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return cuda_fail(h, err);
    }
  }
  h->profiling = enable != 0;
  return TOP_OK;
}

int top_kernel_times(const top_handle *h, float *ms, int n) {
  if (!h || !ms || n < 0) return TOP_E_INVAL;
  if (!h->profiling) return TOP_E_STATE;
  int w = 0;
  for (int q = 0; q < 4 && w < n; ++q, ++w) {
    ms[q] = 0.0f;
    if (h->ran[q] && cudaEventElapsedTime(&ms[q], h->ev[2 * q], h->ev[2 * q + 1]) != cudaSuccess) ms[q] = -1.0f;
  }
  return w;
}

void top_destroy(top_handle *h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaFree(h->G);
  cudaFree(h->E);
  cudaFree(h->P);
  cudaFree(h->d_pstage);
  cudaFree(h->d_aux);
  cudaFree(h->d_ypoly);
  cudaFree(h->d_copy);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  cudaFree(h->d_packs);
  cudaFree(h->d_err);
  cudaFree(h->d_stall);
  cudaFree(h->d_stage);
  cudaFree(h->d_stream);
  cudaFreeHost(h->h_off);
  cudaFreeHost(h->h_packs);
  cudaFreeHost(h->h_lt);
  cudaFreeHost(h->h_tlist);
  cudaFree(h->d_tlist);
  std::free(h->plan_off);
  cudaFreeHost(h->h_err);
  cudaFreeHost(h->h_ctraj);
  std::free(h->layout_off);
  cudaFree(h->d_ctraj);
  cudaFree(h->d_ws);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete h;
}

int top_create(const top_config *cfg, top_handle **out) {
  if (!cfg || !out) return TOP_E_INVAL;
  *out = nullptr;
  if (cfg->max_batch <= 0 || cfg->max_segments <= 0 || cfg->max_samples < 0) return TOP_E_INVAL;
  if (cfg->precision != TOP_FP32 && cfg->precision != TOP_FP64) return TOP_E_INVAL;
  if (cfg->schedule < TOP_SCHED_AUTO || cfg->schedule > TOP_SCHED_STREAM) return TOP_E_INVAL;
  if (cfg->numeric_form < TOP_NUMERIC_AUTO || cfg->numeric_form > TOP_NUMERIC_THREAD) return TOP_E_INVAL;
  if (cfg->gemm_form != TOP_GEMM_CUDA_CORES && cfg->gemm_form != TOP_GEMM_TENSOR) return TOP_E_INVAL;
  if (cfg->stream_form != TOP_STREAM_FUSED && cfg->stream_form != TOP_STREAM_PHASES) return TOP_E_INVAL;
  for (int q = 0; q < 6; ++q)
    if (cfg->reserved[q] != 0) return TOP_E_INVAL;
  top_handle *h = new (std::nothrow) top_handle;
  if (!h) return TOP_E_NOMEM;
  h->cfg = *cfg;
  if (h->cfg.ckpt_interval <= 0) h->cfg.ckpt_interval = 10;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  const size_t S = (size_t)cfg->max_segments, B = (size_t)cfg->max_batch;
  if (e == cudaSuccess) e = cudaMalloc(&h->G, (size_t)NG * S * rbytes(h));
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_packs, sizeof(Pack) * std::max(S, B));
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_stall, sizeof(double) * 3 * B);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_copy, sizeof(int) * (2 * (size_t)S + 1));
  if (e == cudaSuccess) {
    h->stage_bytes = stage_plan((int)B, (int)S).total;
    e = cudaMalloc((void **)&h->d_stage, h->stage_bytes);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_off, sizeof(int32_t) * (B + 1));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_packs, sizeof(Pack) * std::max(S, B));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_lt, sizeof(int) * (2 * B + 1));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_tlist, sizeof(int) * B);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_tlist, sizeof(int) * B);
  if (e == cudaSuccess) {
    h->plan_off = (int32_t *)std::malloc(sizeof(int32_t) * (B + 1));
    if (!h->plan_off) e = cudaErrorMemoryAllocation;
  }
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_ctraj, sizeof(int) * B);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_ctraj, sizeof(int) * B);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? TOP_E_NOMEM : TOP_E_CUDA;
    h->last_cuda = (int)e;
    top_destroy(h);
    cudaGetLastError();
    return code;
  }
  *out = h;
  return TOP_OK;
}

// The streaming form indexes its per-segment state as row * S + g in 32-bit
// integers (row < 6 M_box, 3 M_ball, 3 M_vn, 2 M_gen, F M_poly, or the 108
// values of the polytope inverses): such products must stay below 2^31.
static bool index_fits(const top_problem *pb, int S) {
  long long rows = 108;
  rows = std::max(rows, 6LL * pb->M_box);
  rows = std::max(rows, 3LL * pb->M_ball);
  rows = std::max(rows, 3LL * pb->M_vn);
  rows = std::max(rows, 2LL * pb->M_gen);
  rows = std::max(rows, (long long)pb->F_poly * pb->M_poly);
  return rows * (long long)S < (1LL << 31);
}

}  // extern "C"

namespace {

// top_solve and top_resume: `from` / `to` (may be null) are the state to start
// from and to save, in the problem's memory kind
int solve_impl(top_handle *h, const top_problem *pb_in, top_result *res_in, const top_state *from, top_state *to,
               void *stream) {
  Range range("top_solve");
  int rc = validate(h, pb_in, res_in);
  if (rc != TOP_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  TOP_CUDA(h, cudaSetDevice(h->device));
  const int B = pb_in->B;
  if (B == 0) return TOP_OK;
  // ---- batch layout on the host ----
  const bool async = pb_in->memory == TOP_MEM_DEVICE && h->layout_B == B && h->layout_off;
  if (pb_in->memory == TOP_MEM_HOST) {
    std::memcpy(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1));
  } else if (async) {
    std::memcpy(h->h_off, h->layout_off, sizeof(int32_t) * (B + 1));
  } else {
    TOP_CUDA(h, cudaMemcpyAsync(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1),
                                cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaStreamSynchronize(st));
  }
  const int32_t *off = h->h_off;
  if (off[0] != 0) return TOP_E_INVAL;
  for (int b = 0; b < B; ++b)
    if (off[b + 1] < off[b]) return TOP_E_INVAL;
  const int S = off[B];
  if (S > h->cfg.max_segments) return TOP_E_NOMEM;
  if (S > 0 && (!pb_in->durations || !res_in->coeffs)) return TOP_E_INVAL;
  if (!index_fits(pb_in, S)) return TOP_E_LIMIT;
  const bool resume = from || to;
  if (resume) {
    if (pb_in->adaptive_rho || pb_in->inner != TOP_CLOSED_FORM || pb_in->M_poly > 0 ||
        h->cfg.schedule == TOP_SCHED_STREAM)
      return TOP_E_NOTSUP;
    for (const top_state *x : {from, (const top_state *)to}) {
      if (!x) continue;
      if (!x->p || !x->m || !x->iters || (pb_in->M_box && !x->ybox) || (pb_in->M_ball && !x->qball) ||
          (pb_in->M_vn && !x->qvn))
        return TOP_E_INVAL;
    }
  }
  // ---- device views of inputs and outputs ----
  top_problem pb = *pb_in;
  top_result res = *res_in;
  const bool host = pb_in->memory == TOP_MEM_HOST;
  const StagePlan SP = stage_plan(h->cfg.max_batch, h->cfg.max_segments);
  double *d_hist = nullptr;
  double *coef_mapped = nullptr;  // device view of page-locked caller memory for the coefficients
  if (host) {
    unsigned char *base = h->d_stage;
    auto up = [&](const void *src, size_t off_, size_t bytes) -> const void * {
      if (!src || bytes == 0) return nullptr;
      cudaMemcpyAsync(base + off_, src, bytes, cudaMemcpyHostToDevice, st);
      return base + off_;
    };
    pb.seg_offset = (const int32_t *)up(pb_in->seg_offset, SP.off_seg, sizeof(int32_t) * (B + 1));
    pb.waypoints = (const double *)up(pb_in->waypoints, SP.off_wp, sizeof(double) * 3 * (S + B));
    pb.durations = (const double *)up(pb_in->durations, SP.off_T, sizeof(double) * S);
    pb.start_state = (const double *)up(pb_in->start_state, SP.off_s0, sizeof(double) * 12 * B);
    pb.end_state = (const double *)up(pb_in->end_state, SP.off_s1, sizeof(double) * 12 * B);
    pb.vbox = pb.M_box ? (const double *)up(pb_in->vbox, SP.off_vbox, sizeof(double) * B) : nullptr;
    pb.ball_c = pb.M_ball ? (const double *)up(pb_in->ball_c, SP.off_bc, sizeof(double) * 3 * S) : nullptr;
    pb.ball_r = pb.M_ball ? (const double *)up(pb_in->ball_r, SP.off_br, sizeof(double) * S) : nullptr;
    pb.vnorm = pb.M_vn ? (const double *)up(pb_in->vnorm, SP.off_vn, sizeof(double) * B) : nullptr;
    pb.gen_vmax = pb.M_gen ? (const double *)up(pb_in->gen_vmax, SP.off_gv, sizeof(double) * B) : nullptr;
    pb.gen_amax = pb.M_gen ? (const double *)up(pb_in->gen_amax, SP.off_ga, sizeof(double) * B) : nullptr;
    if (pb.M_poly > 0) {
      const size_t bn = sizeof(double) * 3 * (size_t)pb.F_poly * S, bh = sizeof(double) * (size_t)pb.F_poly * S;
      cudaError_t e = grow((void **)&h->d_pstage, &h->pstage_bytes, align_up(bn, 256) + bh);
      if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, e);
      TOP_CUDA(h, cudaMemcpyAsync(h->d_pstage, pb_in->poly_n, bn, cudaMemcpyHostToDevice, st));
      TOP_CUDA(h, cudaMemcpyAsync(h->d_pstage + align_up(bn, 256), pb_in->poly_h, bh, cudaMemcpyHostToDevice, st));
      pb.poly_n = (const double *)h->d_pstage;
      pb.poly_h = (const double *)(h->d_pstage + align_up(bn, 256));
    }
    TOP_CUDA(h, cudaGetLastError());
    // page-locked (mapped) caller memory takes the coefficients directly: the
    // kernels write them over the chip-to-host link as their CTAs finish, and
    // the copy back after the solve is skipped
    coef_mapped = nullptr;
    {
      cudaPointerAttributes pa{};
      if (res_in->coeffs && cudaPointerGetAttributes(&pa, res_in->coeffs) == cudaSuccess &&
          pa.type == cudaMemoryTypeHost && pa.devicePointer)
        coef_mapped = (double *)pa.devicePointer;
      cudaGetLastError();
    }
    res.coeffs = coef_mapped ? coef_mapped : (double *)(base + SP.off_coef);
    res.cost = (double *)(base + SP.off_cost);
    res.r_primal = (double *)(base + SP.off_rp);
    res.r_dual = (double *)(base + SP.off_rd);
    res.iters = (int32_t *)(base + SP.off_it);
    res.status = (int32_t *)(base + SP.off_st);
    res.rho = res_in->rho ? (double *)(base + SP.off_rho) : nullptr;
    res.history = nullptr;
    if (res_in->history && pb.max_iters > 0) {
      TOP_CUDA(h, cudaMalloc((void **)&d_hist, sizeof(double) * 2 * (size_t)pb.max_iters * B));
      TOP_CUDA(h, cudaMemcpyAsync(d_hist, res_in->history, sizeof(double) * 2 * (size_t)pb.max_iters * B,
                                  cudaMemcpyHostToDevice, st));
      res.history = d_hist;
    }
  }
  DevProblem dp{};
  dp.B = B; dp.S = S; dp.err = h->d_err; dp.stall = pb.stall_checks;
  dp.seg_offset = pb.seg_offset; dp.waypoints = pb.waypoints; dp.durations = pb.durations;
  dp.start_state = pb.start_state; dp.end_state = pb.end_state;
  dp.mode = pb.mode; dp.inner = pb.inner; dp.rho = pb.rho; dp.eps = pb.eps;
  dp.max_iters = pb.max_iters; dp.check_every = pb.check_every > 0 ? pb.check_every : 1;
  dp.M_box = pb.M_box; dp.vbox = pb.vbox;
  dp.M_ball = pb.M_ball; dp.ball_c = pb.ball_c; dp.ball_r = pb.ball_r;
  dp.M_vn = pb.M_vn; dp.vnorm = pb.vnorm;
  dp.M_gen = pb.M_gen; dp.gen_vmax = pb.gen_vmax; dp.gen_amax = pb.gen_amax;
  dp.lbfgs_mem = pb.lbfgs_mem > 0 ? pb.lbfgs_mem : 8;
  dp.lbfgs_max_iters = pb.lbfgs_max_iters > 0 ? pb.lbfgs_max_iters : 50;
  dp.lbfgs_tol = pb.lbfgs_tol > 0 ? pb.lbfgs_tol : (h->cfg.precision == TOP_FP64 ? 1e-12 : 1e-6);
  dp.M_poly = pb.M_poly; dp.F_poly = pb.M_poly > 0 ? pb.F_poly : 0;
  dp.poly_n = pb.poly_n; dp.poly_h = pb.poly_h;
  dp.adaptive = pb.adaptive_rho;
  dp.rho_mu = pb.rho_mu > 0 ? pb.rho_mu : 10.0;
  dp.rho_incr = pb.rho_tau_incr > 0 ? pb.rho_tau_incr : 1.1;
  dp.rho_decr = pb.rho_tau_decr > 0 ? pb.rho_tau_decr : 1.1;
  DevResult dr{};
  dr.coeffs = res.coeffs; dr.cost = res.cost; dr.r_primal = res.r_primal; dr.r_dual = res.r_dual;
  dr.history = res.history; dr.iters = res.iters; dr.status = res.status; dr.rho = res.rho;

  // ---- per-trajectory outputs start at zero (covers empty trajectories) ----
  TOP_CUDA(h, cudaMemsetAsync(dr.cost, 0, sizeof(double) * B, st));
  TOP_CUDA(h, cudaMemsetAsync(dr.r_primal, 0, sizeof(double) * B, st));
  TOP_CUDA(h, cudaMemsetAsync(dr.r_dual, 0, sizeof(double) * B, st));
  TOP_CUDA(h, cudaMemsetAsync(dr.iters, 0, sizeof(int32_t) * B, st));
  TOP_CUDA(h, cudaMemsetAsync(dr.status, 0, sizeof(int32_t) * B, st));
  if (dr.rho) {
    int e = launch_fill(dr.rho, B, pb.rho, st);
    h->launches += 1;
    if (e) return cuda_fail(h, (cudaError_t)e);
  }
  // ---- adaptive-rho data: grow-only workspace ----
  const bool adapt = pb.adaptive_rho != 0;
  if (adapt && (size_t)NE * S * rbytes(h) > h->E_bytes) {
    cudaFree(h->E);
    h->E = nullptr;
    h->E_bytes = 0;
    const size_t want = (size_t)NE * h->cfg.max_segments * rbytes(h);
    cudaError_t e = cudaMalloc(&h->E, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (d_hist) cudaFree(d_hist);
      return e == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, e);
    }
    h->E_bytes = want;
  }
  // ---- FP64 local-matrix inverses (Eq. 18a) ----
  TOP_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
  const bool fp64 = h->cfg.precision == TOP_FP64;
  h->ran[0] = h->ran[1] = h->ran[2] = h->ran[3] = false;
  PolyData pdata{nullptr, nullptr, nullptr, nullptr};
  {
    Range r0("precompute (FP64 local inverses)");
    if (h->profiling) cudaEventRecord(h->ev[0], st);
    int e = 0;
    if (pb.M_poly > 0) {
      const size_t rb = rbytes(h), Sz = (size_t)S, Fp = (size_t)pb.F_poly;
      const size_t bG = align_up(rb * 3 * NG * Sz, 256), bU = align_up(rb * 9 * Sz, 256);
      const size_t bN = align_up(rb * 3 * Fp * Sz, 256), bH = align_up(rb * Fp * Sz, 256);
      cudaError_t ge = grow(&h->P, &h->P_bytes, bG + bU + bN + bH);
      if (ge != cudaSuccess) {
        if (d_hist) cudaFree(d_hist);
        return ge == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, ge);
      }
      unsigned char *pbase = (unsigned char *)h->P;
      pdata = PolyData{pbase, pbase + bG, pbase + bG + bU, pbase + bG + bU + bN};
      e = launch_kinv_poly(dp, pb.rho, fp64, pdata, h->d_err, st);
      h->launches += S > 0 ? 1 : 0;
    } else {
      e = launch_kinv(dp, pb.rho, fp64 ? nullptr : h->G, fp64 ? h->G : nullptr, h->d_err, st, h->d_copy);
      h->launches += S > 0 ? 3 : 0;  // mark, invert, copy
    }
    if (e) return cuda_fail(h, (cudaError_t)e);
    if (adapt) {
      e = launch_keig(dp, fp64 ? nullptr : h->E, fp64 ? h->E : nullptr, h->d_err, st);
      h->launches += S > 0 ? 1 : 0;
      if (e) return cuda_fail(h, (cudaError_t)e);
    }
    if (h->profiling) { cudaEventRecord(h->ev[1], st); h->ran[0] = true; }
  }
  // ---- plan: resident packs of whole trajectories ----
  const int fam = families(&pb);
  const int cap = (h->cfg.schedule == TOP_SCHED_STREAM || pb.inner == TOP_NUMERIC || pb.M_poly > 0)
                      ? 0 : resident_capacity(h, &pb);
  const int ntp_cap = std::max(1, cap / 4);
  // the plan is reused while the batch layout and the capacity repeat
  const bool same_plan = h->plan_valid && h->plan_B == B && h->plan_cap == cap &&
                         std::memcmp(h->plan_off, off, sizeof(int32_t) * (B + 1)) == 0;
  if (!same_plan) {
    plan_packs(off, B, cap, ntp_cap, h->h_packs, h->h_tlist, h->plan_npack, h->plan_max_nseg,
               h->plan_max_ntraj, h->plan_has_long);
    std::memcpy(h->plan_off, off, sizeof(int32_t) * (B + 1));
    h->plan_B = B;
    h->plan_cap = cap;
    h->plan_valid = false;  // set once the device copies are enqueued
  }
  const int npack = h->plan_npack, max_nseg = h->plan_max_nseg, max_ntraj = h->plan_max_ntraj;
  // a resumable run keeps its state resident or in clusters: every long
  // trajectory must fit a cluster (the streaming form has no state export)
  if (resume && h->plan_has_long) {
    const int Mb = (fam & FAM_BOX) ? pb.M_box : 0, Mq = (fam & FAM_BALL) ? pb.M_ball : 0,
              Mv = (fam & FAM_VN) ? pb.M_vn : 0;
    const bool ok = h->cfg.schedule == TOP_SCHED_AUTO && cap > 0 && (fam & ~(FAM_BOX | FAM_BALL | FAM_VN)) == 0;
    const int cc = ok ? cluster_capacity(h, &pb) : 0;
    const int cm =
        cc > 0 ? cluster_max_size(cc, 1, res_layout(cc, kClusterNtp, Mb, Mq, Mv, (int)rbytes(h)).total, fam, fp64) : 0;
    for (int b = 0; b < B; ++b) {
      const int nb = off[b + 1] - off[b];
      if (nb > cap && !(cm >= 2 && (long long)nb <= (long long)cm * cc)) {
        if (d_hist) cudaFree(d_hist);
        return TOP_E_NOTSUP;
      }
    }
  }
  StateView fromv{}, tov{};
  if (resume) {
    const size_t np = sizeof(double) * 21 * (size_t)(S + B), nyb = sizeof(double) * 6 * pb.M_box * (size_t)S,
                 nqb = sizeof(double) * 3 * pb.M_ball * (size_t)S, nqv = sizeof(double) * 3 * pb.M_vn * (size_t)S,
                 nit = sizeof(int32_t) * B;
    auto view = [&](const top_state *x, unsigned char *at) -> StateView {
      StateView v{};
      if (!host) {
        v = StateView{x->p, x->m, x->ybox, x->qball, x->qvn, x->iters};
      } else {
        size_t o = 0;
        auto take = [&](size_t n) { unsigned char *q = at + o; o = align_up(o + n, 256); return q; };
        v.p = (double *)take(np);
        v.m = (double *)take(np);
        v.ybox = (double *)take(nyb);
        v.qball = (double *)take(nqb);
        v.qvn = (double *)take(nqv);
        v.iters = (int32_t *)take(nit);
      }
      if (!pb.M_box) v.ybox = nullptr;
      if (!pb.M_ball) v.qball = nullptr;
      if (!pb.M_vn) v.qvn = nullptr;
      return v;
    };
    const size_t one = 2 * align_up(np, 256) + align_up(nyb, 256) + align_up(nqb, 256) + align_up(nqv, 256) +
                       align_up(nit, 256);
    if (host) {
      cudaError_t ge = grow((void **)&h->d_ws, &h->ws_bytes, 2 * one);
      if (ge != cudaSuccess) {
        if (d_hist) cudaFree(d_hist);
        return ge == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, ge);
      }
    }
    if (from) {
      fromv = view(from, h->d_ws);
      if (host) {
        TOP_CUDA(h, cudaMemcpyAsync(fromv.p, from->p, np, cudaMemcpyHostToDevice, st));
        TOP_CUDA(h, cudaMemcpyAsync(fromv.m, from->m, np, cudaMemcpyHostToDevice, st));
        if (fromv.ybox) TOP_CUDA(h, cudaMemcpyAsync(fromv.ybox, from->ybox, nyb, cudaMemcpyHostToDevice, st));
        if (fromv.qball) TOP_CUDA(h, cudaMemcpyAsync(fromv.qball, from->qball, nqb, cudaMemcpyHostToDevice, st));
        if (fromv.qvn) TOP_CUDA(h, cudaMemcpyAsync(fromv.qvn, from->qvn, nqv, cudaMemcpyHostToDevice, st));
        TOP_CUDA(h, cudaMemcpyAsync(fromv.iters, from->iters, nit, cudaMemcpyHostToDevice, st));
      }
    }
    if (to) {
      tov = view(to, h->d_ws + (host ? one : 0));
      // junctions of empty trajectories and the boundary rows no segment writes start at zero
      TOP_CUDA(h, cudaMemsetAsync(tov.p, 0, np, st));
      TOP_CUDA(h, cudaMemsetAsync(tov.m, 0, np, st));
      TOP_CUDA(h, cudaMemsetAsync(tov.iters, 0, nit, st));
    }
  }
  if (h->plan_has_long && npack > 0) {  // fork point for the cluster launches (after the precompute)
    if (!h->side) {
      TOP_CUDA(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
      TOP_CUDA(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
      TOP_CUDA(h, cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
    }
    TOP_CUDA(h, cudaEventRecord(h->fork_ev, st));
  }
  const bool has_long = h->plan_has_long;
  if (has_long && h->cfg.schedule == TOP_SCHED_RESIDENT) {
    if (d_hist) cudaFree(d_hist);
    return TOP_E_NOTSUP;
  }
  if (npack > 0) {
    if (!same_plan) {
      TOP_CUDA(h, cudaMemcpyAsync(h->d_packs, h->h_packs, sizeof(Pack) * npack, cudaMemcpyHostToDevice, st));
      int ntl = 0;
      for (int q = 0; q < npack; ++q) ntl += h->h_packs[q].ntraj;
      TOP_CUDA(h, cudaMemcpyAsync(h->d_tlist, h->h_tlist, sizeof(int) * ntl, cudaMemcpyHostToDevice, st));
      h->plan_valid = true;
    }
    const int C = std::max(32, (max_nseg + 31) / 32 * 32);
    const int ntp = std::max(1, max_ntraj);
    const int Mb = (fam & FAM_BOX) ? pb.M_box : 0, Mq = (fam & FAM_BALL) ? pb.M_ball : 0,
              Mv = (fam & FAM_VN) ? pb.M_vn : 0;
    // the tensor-core form of the G product (top_config.gemm_form) where it applies and fits
    int tc = (h->cfg.gemm_form == TOP_GEMM_TENSOR && !fp64 && fam == 0 && !adapt) ? 1 : 0;
    if (tc && res_layout_resident(C, ntp, Mb, Mq, Mv, (int)rbytes(h), true).total > (size_t)h->smem_optin) tc = 0;
    const ResLayout L = res_layout_resident(C, ntp, Mb, Mq, Mv, (int)rbytes(h), tc != 0);
    ResidentArgs ra{};
    ra.p = dp; ra.r = dr; ra.G = h->G; ra.packs = h->d_packs; ra.traj_list = h->d_tlist; ra.ntp = ntp;
    ra.tc = tc;
    ra.stall = pb.stall_checks > 0 ? h->d_stall : nullptr;
    ra.E = adapt ? h->E : nullptr;
    ra.from = fromv; ra.to = tov;
    Range r1("resident packs");
    if (h->profiling) cudaEventRecord(h->ev[2], st);
    int e = fp64 ? launch_resident_f64(ra, npack, C, L.total, fam, st)
                 : launch_resident_f32(ra, npack, C, L.total, fam, st);
    h->launches += 1;
    if (e) return cuda_fail(h, (cudaError_t)e);
    if (h->profiling) { cudaEventRecord(h->ev[3], st); h->ran[1] = true; }
  }
  // ---- cluster-resident form for trajectories longer than a CTA but within a cluster ----
  // (closed-form step with the box / ball / velocity-norm / polytope families, fixed or
  // adaptive rho)
  // polytope trajectories of any length use the cluster form (a cluster of one CTA
  // for short ones): the resident packs have no room for their per-axis inverses
  // cluster groups: lanes per segment, segments per CTA, shared memory, largest cluster.  With
  // sample rows (FP32, fixed rho) a segment's rows are split over 4 or 2 lanes (at least two
  // rows per lane) where the trajectory fits a cluster of such CTAs; the rest run one lane per
  // segment.
  struct CGroup { int ln, C, cmax; size_t smem; };
  CGroup grp[3];
  int ngrp = 0;
  const bool poly = (fam & FAM_POLY) != 0;
  const bool cluster_ok = has_long && (cap > 0 || poly) && h->cfg.schedule == TOP_SCHED_AUTO &&
                          (fam & ~(FAM_BOX | FAM_BALL | FAM_VN | FAM_POLY)) == 0;
  const int cmin = poly ? 1 : 2;
  if (cluster_ok) {
    const int ccap = cluster_capacity(h, &pb);
    if (ccap > 0) {
      const int Mb = (fam & FAM_BOX) ? pb.M_box : 0, Mq = (fam & FAM_BALL) ? pb.M_ball : 0,
                Mv = (fam & FAM_VN) ? pb.M_vn : 0;
      const int Mp = poly ? pb.M_poly : 0;
      const int rows = Mb + Mq + Mv + Mp;  // sample rows per segment
      const int lns[3] = {4, 2, 1};  // (8 lanes measured no faster: the rows a lane repeats dominate)
      for (int q = 0; q < 3; ++q) {
        const int ln = lns[q];
        if (ln > 1 && (fp64 || adapt || rows < 2 * ln)) continue;  // at least two rows per lane
        const int C = ln == 1 ? ccap : std::min(ccap, max_cta_threads(h) / ln / 32 * 32);
        if (C < 32) continue;
        const size_t sm = res_layout(C, kClusterNtp, Mb, Mq, Mv, (int)rbytes(h), Mp).total;
        if (h->csz_key_C[q] != C || h->csz_key_fam[q] != fam || h->csz_key_smem[q] != sm) {
          h->csz_val[q] = cluster_max_size(C, ln, sm, fam, fp64);
          h->csz_key_C[q] = C;
          h->csz_key_fam[q] = fam;
          h->csz_key_smem[q] = sm;
        }
        if (h->csz_val[q] >= cmin) grp[ngrp++] = CGroup{ln, C, h->csz_val[q], sm};
      }
    }
  }
  // a long trajectory's cluster: the first group (most lanes) and the smallest power of two
  // of its CTAs that hold it, as group * 32 + CTAs; 0 = none
  auto placement = [&](int nb) -> int {
    for (int q = 0; q < ngrp; ++q)
      for (int c = cmin; c <= grp[q].cmax; c <<= 1)
        if ((long long)c * grp[q].C >= nb) return q * 32 + c;
    return 0;
  };
  bool any_cluster = false;
  if (ngrp > 0) {
    DevResult drc = dr;
    ClusterArgs ca{};
    ca.p = dp; ca.r = drc; ca.G = h->G; ca.E = adapt ? h->E : nullptr; ca.traj = h->d_ctraj;
    ca.from = fromv; ca.to = tov;
    ca.poly = pdata;
    if (poly) {
      const size_t want = rbytes(h) * (size_t)dp.F_poly * dp.M_poly * (size_t)S + 256;
      cudaError_t ge = grow(&h->d_ypoly, &h->ypoly_bytes, want);
      if (ge != cudaSuccess) {
        if (d_hist) cudaFree(d_hist);
        return ge == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, ge);
      }
      ca.ypoly = h->d_ypoly;
    }
    // one launch per (group, cluster size), trajectories listed back to back in d_ctraj
    int nlist = 0;
    for (int q = 0; q < ngrp; ++q)
      for (int c = cmin; c <= grp[q].cmax; c <<= 1)
        for (int b = 0; b < B; ++b) {
          const int nb = off[b + 1] - off[b];
          if (nb > 0 && (cap == 0 || nb > cap) && placement(nb) == q * 32 + c) h->h_ctraj[nlist++] = b;
        }
    if (nlist > 0) {
      any_cluster = true;
      cudaStream_t cs = (npack > 0 && h->side) ? h->side : st;  // beside the resident packs when there are any
      if (cs != st) TOP_CUDA(h, cudaStreamWaitEvent(cs, h->fork_ev, 0));
      TOP_CUDA(h, cudaMemcpyAsync(h->d_ctraj, h->h_ctraj, sizeof(int) * nlist, cudaMemcpyHostToDevice, cs));
      Range r3("cluster-resident trajectories");
      if (h->profiling) cudaEventRecord(h->ev[6], cs);
      int at = 0;
      for (int q = 0; q < ngrp; ++q)
        for (int c = cmin; c <= grp[q].cmax; c <<= 1) {
          int n = 0;
          while (at + n < nlist && placement(off[h->h_ctraj[at + n] + 1] - off[h->h_ctraj[at + n]]) == q * 32 + c) ++n;
          if (n == 0) continue;
          ca.traj = h->d_ctraj + at;
          int e = fp64 ? launch_cluster_f64(ca, n, c, grp[q].C, grp[q].ln, grp[q].smem, fam, cs)
                       : launch_cluster_f32(ca, n, c, grp[q].C, grp[q].ln, grp[q].smem, fam, cs);
          h->launches += 1;
          if (e) return cuda_fail(h, (cudaError_t)e);
          at += n;
        }
      if (h->profiling) { cudaEventRecord(h->ev[7], cs); h->ran[3] = true; }
      if (cs != st) {
        TOP_CUDA(h, cudaEventRecord(h->join_ev, cs));
        TOP_CUDA(h, cudaStreamWaitEvent(st, h->join_ev, 0));
      }
    }
  }
  // ---- streaming form for the remaining long trajectories ----
  int n_stream_traj = 0;
  if (has_long)
    for (int b = 0; b < B; ++b) {
      const int nb = off[b + 1] - off[b];
      if (nb > 0 && (cap == 0 || nb > cap) && !(any_cluster && placement(nb) > 0)) ++n_stream_traj;
    }
  if (n_stream_traj > 0) {
    int nl = 0, total = 0, nchunk = 1;
    h->h_lt[0] = 0;  // h_lt = [lt_b (B) | lt_prefix (B+1)]
    int *lt_b = h->h_lt, *lt_pre = h->h_lt + h->cfg.max_batch;
    lt_pre[0] = 0;
    for (int b = 0; b < B; ++b) {
      const int nb = off[b + 1] - off[b];
      if (nb > 0 && (cap == 0 || nb > cap) && !(any_cluster && placement(nb) > 0)) {
        lt_b[nl] = b;
        total += nb;
        lt_pre[++nl] = total;
        nchunk = std::max(nchunk, (nb + kReduceChunk - 1) / kReduceChunk);
      }
    }
    const size_t rb = rbytes(h);
    const size_t Jn = (size_t)S + B;
    const int Mb = (fam & FAM_BOX) ? pb.M_box : 0, Mq = (fam & FAM_BALL) ? pb.M_ball : 0,
              Mv = (fam & FAM_VN) ? pb.M_vn : 0;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    const size_t o_z = take(rb * 21 * Jn), o_uL = take(rb * 21 * Jn), o_dz = take(rb * 21 * Jn);
    const size_t o_uRp = take(rb * 3 * Jn), o_uR0 = take(rb * 12 * (size_t)B);
    const size_t o_eS = take(rb * 21 * (size_t)S), o_eE = take(rb * 21 * (size_t)S), o_ch = take(rb * 24 * (size_t)S);
    const size_t o_yb = take(rb * 6 * Mb * (size_t)S), o_qb = take(rb * 3 * Mq * (size_t)S);
    const size_t o_qv = take(rb * 3 * Mv * (size_t)S);
    const int Mg = (fam & FAM_GEN) ? pb.M_gen : 0;
    const size_t o_yg = take(rb * 2 * Mg * (size_t)S);
    const size_t o_yp = take(rb * (size_t)dp.F_poly * dp.M_poly * (size_t)S);
    const size_t o_rp = take(sizeof(double) * total), o_rd = take(sizeof(double) * total);
    const size_t o_done = take(sizeof(int) * nl), o_trp = take(sizeof(double) * nl), o_trd = take(sizeof(double) * nl);
    const size_t o_rho = take(sizeof(double) * nl), o_fac = take(sizeof(double) * nl);
    const size_t o_kc = take(sizeof(int) * nl);
    const size_t o_nw = take(sizeof(int) * (Mg > 0 ? (size_t)total + 2 : 2));
    // fused iterations: second halves of the junction state and of the end values
    const bool fuse = h->cfg.stream_form == TOP_STREAM_FUSED;
    const size_t o_zB = take(fuse ? rb * 21 * Jn : 0), o_uLB = take(fuse ? rb * 21 * Jn : 0);
    const size_t o_uRpB = take(fuse ? rb * 3 * Jn : 0);
    const size_t o_eSB = take(fuse ? rb * 21 * (size_t)S : 0), o_eEB = take(fuse ? rb * 21 * (size_t)S : 0);
    const size_t o_lt = take(sizeof(int) * (2 * (size_t)nl + 1));
    const size_t o_part = take(sizeof(double) * 2 * (size_t)nl * nchunk), o_tk = take(sizeof(int) * nl);
    const size_t o_segt = take(sizeof(int) * (size_t)total);
    if (o > h->stream_bytes) {
      cudaFree(h->d_stream);
      h->d_stream = nullptr;
      h->stream_bytes = 0;
      cudaError_t e = cudaMalloc((void **)&h->d_stream, o);
      if (e != cudaSuccess) {
        cudaGetLastError();
        if (d_hist) cudaFree(d_hist);
        return e == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, e);
      }
      h->stream_bytes = o;
    }
    unsigned char *base = h->d_stream;
    TOP_CUDA(h, cudaMemcpyAsync(base + o_lt, lt_b, sizeof(int) * nl, cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(base + o_lt + sizeof(int) * nl, lt_pre, sizeof(int) * (nl + 1),
                                cudaMemcpyHostToDevice, st));
    StreamArgs sa{};
    sa.p = dp; sa.r = dr; sa.G = h->G;
    sa.lt_b = (const int *)(base + o_lt);
    sa.lt_prefix = (const int *)(base + o_lt) + nl;
    sa.nl = nl; sa.total = total; sa.S = S; sa.Jn = (int)Jn;
    sa.z = base + o_z; sa.uL = base + o_uL; sa.dz = base + o_dz; sa.uRp = base + o_uRp; sa.uR0 = base + o_uR0;
    sa.eS = base + o_eS; sa.eE = base + o_eE; sa.ch = base + o_ch;
    sa.ybox = base + o_yb; sa.qball = base + o_qb; sa.qvn = base + o_qv;
    sa.ygen = base + o_yg; sa.inner_iters = nullptr;
    sa.ypoly = base + o_yp; sa.poly = pdata;
    sa.rp2 = (double *)(base + o_rp); sa.rd2 = (double *)(base + o_rd);
    sa.done = (int *)(base + o_done); sa.tr_rp = (double *)(base + o_trp); sa.tr_rd = (double *)(base + o_trd);
    sa.rho_t = (double *)(base + o_rho); sa.fac_t = (double *)(base + o_fac);
    sa.kcount = (int *)(base + o_kc); sa.cev = 1;
    sa.part = (double *)(base + o_part); sa.ticket = (int *)(base + o_tk); sa.nchunk = nchunk;
    // a few trajectories: the search over lt_prefix is as short as the map's extra load
    sa.seg_t = nl > 4 ? (int *)(base + o_segt) : nullptr;
    // segments with a violated general bound: one warp each (an extra, short
    // launch per iteration; the default), or one thread each
    const bool warp_num = Mg > 0 && h->cfg.numeric_form != TOP_NUMERIC_THREAD;
    sa.nwork = warp_num ? (int *)(base + o_nw) : nullptr;  // two counts, then the list
    sa.work = warp_num ? (int *)(base + o_nw) + 2 : nullptr;
    if (fuse) {
      sa.zB = base + o_zB; sa.uLB = base + o_uLB; sa.uRpB = base + o_uRpB;
      sa.eSB = base + o_eSB; sa.eEB = base + o_eEB;
    }
    sa.E = adapt ? h->E : nullptr;
    sa.launches = &h->launches;
    Range r2("streaming trajectories");
    if (h->profiling) cudaEventRecord(h->ev[4], st);
    int e = fp64 ? launch_stream_f64(sa, fam, st) : launch_stream_f32(sa, fam, st);
    if (e) return cuda_fail(h, (cudaError_t)e);
    if (h->profiling) { cudaEventRecord(h->ev[5], st); h->ran[2] = true; }
  }
  // ---- outputs back to the host, error flags ----
  if (host && to) {
    const size_t np = sizeof(double) * 21 * (size_t)(S + B);
    TOP_CUDA(h, cudaMemcpyAsync(to->p, tov.p, np, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(to->m, tov.m, np, cudaMemcpyDeviceToHost, st));
    if (tov.ybox) TOP_CUDA(h, cudaMemcpyAsync(to->ybox, tov.ybox, sizeof(double) * 6 * pb.M_box * (size_t)S, cudaMemcpyDeviceToHost, st));
    if (tov.qball) TOP_CUDA(h, cudaMemcpyAsync(to->qball, tov.qball, sizeof(double) * 3 * pb.M_ball * (size_t)S, cudaMemcpyDeviceToHost, st));
    if (tov.qvn) TOP_CUDA(h, cudaMemcpyAsync(to->qvn, tov.qvn, sizeof(double) * 3 * pb.M_vn * (size_t)S, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(to->iters, tov.iters, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
  }
  if (host) {
    if (!coef_mapped)
      TOP_CUDA(h, cudaMemcpyAsync(res_in->coeffs, res.coeffs, sizeof(double) * 24 * S, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(res_in->cost, res.cost, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(res_in->r_primal, res.r_primal, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(res_in->r_dual, res.r_dual, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(res_in->iters, res.iters, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(res_in->status, res.status, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
    if (res.rho)
      TOP_CUDA(h, cudaMemcpyAsync(res_in->rho, res.rho, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    if (d_hist)
      TOP_CUDA(h, cudaMemcpyAsync(res_in->history, d_hist, sizeof(double) * 2 * (size_t)pb.max_iters * B,
                                  cudaMemcpyDeviceToHost, st));
  }
  if (async) return TOP_OK;  // the error flag is read by top_sync
  TOP_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOP_CUDA(h, cudaStreamSynchronize(st));
  if (d_hist) cudaFree(d_hist);
  if (*h->h_err & 1) return TOP_E_INVAL;
  if (*h->h_err & 2) return TOP_E_NUMERIC;
  if (*h->h_err & 4) return TOP_E_BOUNDS;
  return TOP_OK;
}

}  // namespace

extern "C" {

int top_solve(top_handle *h, const top_problem *pb, top_result *res, void *stream) {
  return solve_impl(h, pb, res, nullptr, nullptr, stream);
}

int top_resume(top_handle *h, const top_problem *pb, const top_state *from, top_result *res, top_state *to,
               void *stream) {
  return solve_impl(h, pb, res, from, to, stream);
}

int top_set_layout(top_handle *h, int32_t B, const int32_t *host_seg_offset) {
  if (!h || B < 0) return TOP_E_INVAL;
  if (B == 0) {
    h->layout_B = 0;
    return TOP_OK;
  }
  if (!host_seg_offset) return TOP_E_INVAL;
  if (B > h->cfg.max_batch) return TOP_E_NOMEM;
  if (host_seg_offset[0] != 0) return TOP_E_INVAL;
  for (int b = 0; b < B; ++b)
    if (host_seg_offset[b + 1] < host_seg_offset[b]) return TOP_E_INVAL;
  if (host_seg_offset[B] > h->cfg.max_segments) return TOP_E_NOMEM;
  if (!h->layout_off) {
    h->layout_off = (int32_t *)std::malloc(sizeof(int32_t) * (h->cfg.max_batch + 1));
    if (!h->layout_off) return TOP_E_NOMEM;
  }
  std::memcpy(h->layout_off, host_seg_offset, sizeof(int32_t) * (B + 1));
  h->layout_B = B;
  return TOP_OK;
}

int top_sync(top_handle *h, void *stream) {
  if (!h) return TOP_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TOP_CUDA(h, cudaSetDevice(h->device));
  TOP_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOP_CUDA(h, cudaStreamSynchronize(st));
  if (*h->h_err & 1) return TOP_E_INVAL;
  if (*h->h_err & 2) return TOP_E_NUMERIC;
  if (*h->h_err & 4) return TOP_E_BOUNDS;
  return TOP_OK;
}

int top_grad(top_handle *h, const top_problem *pb_in, const double *dJ, double *dwaypoints, double *ddurations,
             void *stream) {
  Range range("top_grad");
  if (!h || !pb_in || !dJ || !dwaypoints || !ddurations) return TOP_E_INVAL;
  top_result fake{};
  fake.coeffs = fake.cost = fake.r_primal = fake.r_dual = ddurations;
  fake.iters = fake.status = (int32_t *)ddurations;
  int rc = validate(h, pb_in, &fake);
  if (rc != TOP_OK) return rc;
  if (pb_in->inner != TOP_CLOSED_FORM || pb_in->M_gen || pb_in->M_poly) return TOP_E_NOTSUP;
  if (pb_in->adaptive_rho) return TOP_E_NOTSUP;
  const int fam = families(pb_in) & (FAM_BOX | FAM_BALL | FAM_VN);
  cudaStream_t st = (cudaStream_t)stream;
  TOP_CUDA(h, cudaSetDevice(h->device));
  const int B = pb_in->B;
  if (B == 0) return TOP_OK;
  const bool host = pb_in->memory == TOP_MEM_HOST;
  if (host) {
    std::memcpy(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1));
  } else {
    TOP_CUDA(h, cudaMemcpyAsync(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1),
                                cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaStreamSynchronize(st));
  }
  const int32_t *off = h->h_off;
  if (off[0] != 0) return TOP_E_INVAL;
  for (int b = 0; b < B; ++b)
    if (off[b + 1] < off[b]) return TOP_E_INVAL;
  const int S = off[B];
  if (S > h->cfg.max_segments) return TOP_E_NOMEM;
  if (S > 0 && !pb_in->durations) return TOP_E_INVAL;
  const size_t Jn = (size_t)S + B;
  const int K = pb_in->max_iters;
  const int ckpt = h->cfg.ckpt_interval > 0 ? h->cfg.ckpt_interval : 10;
  const int nblk = K > 0 ? (K + ckpt - 1) / ckpt : 0;
  // segment list: every non-empty trajectory
  int nl = 0, total = 0;
  int *lt_b = h->h_lt, *lt_pre = h->h_lt + h->cfg.max_batch;
  lt_pre[0] = 0;
  for (int b = 0; b < B; ++b) {
    const int nb = off[b + 1] - off[b];
    if (nb > 0) { lt_b[nl] = b; total += nb; lt_pre[++nl] = total; }
  }
  // ---- workspace ----
  const size_t rb = rbytes(h);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
  const size_t bz = rb * 21 * Jn, buRp = rb * 3 * Jn, buR0 = rb * 12 * (size_t)B;
  const size_t o_z = take(bz), o_uL = take(bz), o_dz = take(bz), o_uRp = take(buRp), o_uR0 = take(buR0);
  const size_t o_eS = take(rb * 21 * (size_t)S), o_eE = take(rb * 21 * (size_t)S), o_ch = take(rb * 24 * (size_t)S);
  const size_t o_rp = take(sizeof(double) * total), o_rd = take(sizeof(double) * total);
  const size_t o_done = take(sizeof(int) * nl), o_trp = take(sizeof(double) * nl), o_trd = take(sizeof(double) * nl);
  const size_t o_rho = take(sizeof(double) * nl), o_fac = take(sizeof(double) * nl);
  const size_t o_lt = take(sizeof(int) * (2 * (size_t)nl + 1));
  // the rows' states (box slack/dual, ball and velocity-norm projections) and their adjoints
  const int Mb = (fam & FAM_BOX) ? pb_in->M_box : 0, Mq = (fam & FAM_BALL) ? pb_in->M_ball : 0,
            Mv = (fam & FAM_VN) ? pb_in->M_vn : 0;
  const size_t byb = rb * 6 * Mb * (size_t)S, bqb = rb * 3 * Mq * (size_t)S, bqv = rb * 3 * Mv * (size_t)S;
  const size_t o_yb = take(byb), o_qb = take(bqb), o_qv = take(bqv);
  const size_t o_ybb = take(byb), o_qbb = take(bqb), o_qvb = take(bqv);
  const size_t one_state = bz * 2 + buRp + buR0 + byb + bqb + bqv + 7 * 256;
  const size_t o_ck = take(one_state * (size_t)nblk);
  const size_t o_tape = take(one_state * (size_t)ckpt);
  const size_t o_zb = take(bz), o_uLb = take(bz), o_uRb = take(bz), o_uR0b = take(buR0);
  const size_t o_eSb = take(rb * 21 * (size_t)S), o_eEb = take(rb * 21 * (size_t)S);
  const size_t o_wbS = take(rb * 21 * (size_t)S), o_wbE = take(rb * 21 * (size_t)S);
  const size_t o_Tb = take(sizeof(double) * S), o_Pb = take(sizeof(double) * 3 * Jn);
  const size_t o_dJ = take(sizeof(double) * B), o_dw = take(sizeof(double) * 3 * Jn), o_dT = take(sizeof(double) * S);
  if (o > h->stream_bytes) {
    cudaFree(h->d_stream);
    h->d_stream = nullptr;
    h->stream_bytes = 0;
    cudaError_t e = cudaMalloc((void **)&h->d_stream, o);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, e);
    }
    h->stream_bytes = o;
  }
  unsigned char *base = h->d_stream;
  // ---- device views of the inputs and outputs ----
  top_problem pb = *pb_in;
  const double *d_dJ = dJ;
  double *d_dw = dwaypoints, *d_dT = ddurations;
  if (host) {
    const StagePlan SP = stage_plan(h->cfg.max_batch, h->cfg.max_segments);
    unsigned char *sb = h->d_stage;
    TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_seg, pb_in->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_wp, pb_in->waypoints, sizeof(double) * 3 * Jn, cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_T, pb_in->durations, sizeof(double) * S, cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_s0, pb_in->start_state, sizeof(double) * 12 * B, cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_s1, pb_in->end_state, sizeof(double) * 12 * B, cudaMemcpyHostToDevice, st));
    if (Mb) TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_vbox, pb_in->vbox, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    if (Mq) {
      TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_bc, pb_in->ball_c, sizeof(double) * 3 * S, cudaMemcpyHostToDevice, st));
      TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_br, pb_in->ball_r, sizeof(double) * S, cudaMemcpyHostToDevice, st));
    }
    if (Mv) TOP_CUDA(h, cudaMemcpyAsync(sb + SP.off_vn, pb_in->vnorm, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(base + o_dJ, dJ, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    pb.seg_offset = (const int32_t *)(sb + SP.off_seg);
    pb.waypoints = (const double *)(sb + SP.off_wp);
    pb.durations = (const double *)(sb + SP.off_T);
    pb.start_state = (const double *)(sb + SP.off_s0);
    pb.end_state = (const double *)(sb + SP.off_s1);
    pb.vbox = Mb ? (const double *)(sb + SP.off_vbox) : nullptr;
    pb.ball_c = Mq ? (const double *)(sb + SP.off_bc) : nullptr;
    pb.ball_r = Mq ? (const double *)(sb + SP.off_br) : nullptr;
    pb.vnorm = Mv ? (const double *)(sb + SP.off_vn) : nullptr;
    d_dJ = (const double *)(base + o_dJ);
    d_dw = (double *)(base + o_dw);
    d_dT = (double *)(base + o_dT);
  }
  DevProblem dp{};
  dp.B = B; dp.S = S; dp.err = h->d_err;
  dp.seg_offset = pb.seg_offset; dp.waypoints = pb.waypoints; dp.durations = pb.durations;
  dp.start_state = pb.start_state; dp.end_state = pb.end_state;
  dp.mode = pb.mode; dp.inner = TOP_CLOSED_FORM; dp.rho = pb.rho; dp.eps = 0.0;
  dp.max_iters = K; dp.check_every = 1;
  dp.M_box = Mb; dp.vbox = pb.vbox;
  dp.M_ball = Mq; dp.ball_c = pb.ball_c; dp.ball_r = pb.ball_r;
  dp.M_vn = Mv; dp.vnorm = pb.vnorm;
  DevResult dr{};
  TOP_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
  const bool fp64 = h->cfg.precision == TOP_FP64;
  h->ran[0] = h->ran[1] = h->ran[2] = h->ran[3] = false;
  {
    if (h->profiling) cudaEventRecord(h->ev[0], st);
    int e = launch_kinv(dp, pb.rho, fp64 ? nullptr : h->G, fp64 ? h->G : nullptr, h->d_err, st);
    if (e) return cuda_fail(h, (cudaError_t)e);
    if (h->profiling) { cudaEventRecord(h->ev[1], st); h->ran[0] = true; }
  }
  TOP_CUDA(h, cudaMemsetAsync(d_dw, 0, sizeof(double) * 3 * Jn, st));
  TOP_CUDA(h, cudaMemsetAsync(d_dT, 0, sizeof(double) * S, st));
  // resident adjoint when every trajectory fits one CTA (the whole reverse
  // sweep in one launch, state in shared memory); the streaming form otherwise
  int maxN = 0;
  for (int b = 0; b < B; ++b) maxN = std::max(maxN, off[b + 1] - off[b]);
  int rcap = 0;
  if (h->cfg.schedule != TOP_SCHED_STREAM)
    for (int C = 256; C >= 32 && rcap == 0; C -= 32)
      if (adjres_layout(C, C / 4, (int)rb).total <= (size_t)h->smem_optin) rcap = C;
  if (nl > 0 && K > 0 && maxN <= rcap && fam == 0) {
    int npack = 0, max_nseg = 0, max_ntraj = 0;
    bool has_long = false;
    plan_packs(off, B, rcap, std::max(1, rcap / 4), h->h_packs, h->h_tlist, npack, max_nseg, max_ntraj, has_long);
    h->plan_valid = false;  // the pack buffers now hold this plan
    const size_t st_bytes = rb * 2 * 21 * Jn;  // one saved slot state
    size_t o2 = o_dT + align_up(sizeof(double) * S, 256);
    const size_t o_rck = o2;
    o2 = align_up(o2 + st_bytes * nblk, 256);
    const size_t o_rtape = o2;
    o2 = align_up(o2 + st_bytes * ckpt, 256);
    if (o2 > h->stream_bytes) {
      cudaFree(h->d_stream);
      h->d_stream = nullptr;
      h->stream_bytes = 0;
      cudaError_t e = cudaMalloc((void **)&h->d_stream, o2);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, e);
      }
      h->stream_bytes = o2;
      base = h->d_stream;
      if (host) {  // the staged seeds and outputs live in this buffer
        TOP_CUDA(h, cudaMemcpyAsync(base + o_dJ, dJ, sizeof(double) * B, cudaMemcpyHostToDevice, st));
        d_dJ = (const double *)(base + o_dJ);
        d_dw = (double *)(base + o_dw);
        d_dT = (double *)(base + o_dT);
        TOP_CUDA(h, cudaMemsetAsync(d_dw, 0, sizeof(double) * 3 * Jn, st));
        TOP_CUDA(h, cudaMemsetAsync(d_dT, 0, sizeof(double) * S, st));
      }
    }
    TOP_CUDA(h, cudaMemcpyAsync(h->d_packs, h->h_packs, sizeof(Pack) * npack, cudaMemcpyHostToDevice, st));
    int ntl = 0;
    for (int q = 0; q < npack; ++q) ntl += h->h_packs[q].ntraj;
    TOP_CUDA(h, cudaMemcpyAsync(h->d_tlist, h->h_tlist, sizeof(int) * ntl, cudaMemcpyHostToDevice, st));
    const int C = std::max(32, (max_nseg + 31) / 32 * 32);
    const int ntp = std::max(1, max_ntraj);
    AdjResArgs ra{};
    ra.p = dp; ra.G = h->G; ra.packs = h->d_packs; ra.traj_list = h->d_tlist; ra.ntp = ntp;
    ra.ckpt = ckpt; ra.Jn = (int)Jn; ra.ck = base + o_rck; ra.tape = base + o_rtape;
    ra.dJ = d_dJ; ra.dw = d_dw; ra.dT = d_dT;
    const size_t smem = adjres_layout(C, ntp, (int)rb).total;
    Range r1("resident adjoint");
    if (h->profiling) cudaEventRecord(h->ev[2], st);
    int e = fp64 ? launch_adjres_f64(ra, npack, C, smem, st) : launch_adjres_f32(ra, npack, C, smem, st);
    h->launches += 1;
    if (e) return cuda_fail(h, (cudaError_t)e);
    if (h->profiling) { cudaEventRecord(h->ev[3], st); h->ran[1] = true; }
  } else if (nl > 0 && K > 0) {
    TOP_CUDA(h, cudaMemcpyAsync(base + o_lt, lt_b, sizeof(int) * nl, cudaMemcpyHostToDevice, st));
    TOP_CUDA(h, cudaMemcpyAsync(base + o_lt + sizeof(int) * nl, lt_pre, sizeof(int) * (nl + 1),
                                cudaMemcpyHostToDevice, st));
    StreamArgs sa{};
    sa.p = dp; sa.r = dr; sa.G = h->G;
    sa.lt_b = (const int *)(base + o_lt);
    sa.lt_prefix = (const int *)(base + o_lt) + nl;
    sa.nl = nl; sa.total = total; sa.S = S; sa.Jn = (int)Jn;
    sa.z = base + o_z; sa.uL = base + o_uL; sa.dz = base + o_dz; sa.uRp = base + o_uRp; sa.uR0 = base + o_uR0;
    sa.eS = base + o_eS; sa.eE = base + o_eE; sa.ch = base + o_ch;
    sa.ybox = base + o_yb; sa.qball = base + o_qb; sa.qvn = base + o_qv;
    sa.ygen = nullptr;
    sa.inner_iters = nullptr;
    sa.rp2 = (double *)(base + o_rp); sa.rd2 = (double *)(base + o_rd);
    sa.done = (int *)(base + o_done); sa.tr_rp = (double *)(base + o_trp); sa.tr_rd = (double *)(base + o_trd);
    sa.rho_t = (double *)(base + o_rho); sa.fac_t = (double *)(base + o_fac);
    sa.E = nullptr;
    AdjArgs aa{};
    aa.f = sa;
    aa.zb = base + o_zb; aa.uLb = base + o_uLb; aa.uRb = base + o_uRb; aa.uR0b = base + o_uR0b;
    aa.eSb = base + o_eSb; aa.eEb = base + o_eEb; aa.wbS = base + o_wbS; aa.wbE = base + o_wbE;
    aa.Tbar = (double *)(base + o_Tb); aa.Pbar = (double *)(base + o_Pb); aa.dJ = d_dJ;
    aa.ybb = base + o_ybb; aa.qbb = base + o_qbb; aa.qvb = base + o_qvb;
    TOP_CUDA(h, cudaMemsetAsync(base + o_zb, 0, o_eSb - o_zb, st));        // zb, uLb, uRb, uR0b
    TOP_CUDA(h, cudaMemsetAsync(base + o_wbS, 0, o_Tb - o_wbS, st));       // wbS, wbE
    TOP_CUDA(h, cudaMemsetAsync(base + o_Tb, 0, o_dJ - o_Tb, st));         // Tbar, Pbar
    TOP_CUDA(h, cudaMemsetAsync(base + o_ybb, 0, o_ck - o_ybb, st));       // the rows' adjoints
    const size_t bytes[7] = {bz, bz, buRp, buR0, byb, bqb, bqv};
    std::vector<void *> ck((size_t)nblk * 7), tape((size_t)ckpt * 7);
    size_t oc = o_ck, ot = o_tape;
    for (int c = 0; c < nblk; ++c)
      for (int q = 0; q < 7; ++q) { ck[(size_t)c * 7 + q] = base + oc; oc = align_up(oc + bytes[q], 256); }
    for (int c = 0; c < ckpt; ++c)
      for (int q = 0; q < 7; ++q) { tape[(size_t)c * 7 + q] = base + ot; ot = align_up(ot + bytes[q], 256); }
    if (h->profiling) cudaEventRecord(h->ev[4], st);
    int e = fp64 ? launch_adjoint_f64(sa, aa, fam, ckpt, ck.data(), tape.data(), bytes, d_dw, d_dT, st)
                 : launch_adjoint_f32(sa, aa, fam, ckpt, ck.data(), tape.data(), bytes, d_dw, d_dT, st);
    if (e) return cuda_fail(h, (cudaError_t)e);
    if (h->profiling) { cudaEventRecord(h->ev[5], st); h->ran[2] = true; }
  }
  if (host) {
    TOP_CUDA(h, cudaMemcpyAsync(dwaypoints, d_dw, sizeof(double) * 3 * Jn, cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaMemcpyAsync(ddurations, d_dT, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  }
  TOP_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOP_CUDA(h, cudaStreamSynchronize(st));
  if (*h->h_err & 1) return TOP_E_INVAL;
  if (*h->h_err & 2) return TOP_E_NUMERIC;
  if (*h->h_err & 4) return TOP_E_BOUNDS;
  return TOP_OK;
}

int top_autotune(top_handle *h, const top_problem *pb_in, int32_t iters, int32_t *out_segs_per_cta, float *ms,
                 int32_t n_ms, void *stream) {
  if (!h || !pb_in || iters < 1 || (ms && n_ms < 0)) return TOP_E_INVAL;
  if (pb_in->B < 0 || pb_in->B > h->cfg.max_batch) return pb_in->B < 0 ? TOP_E_INVAL : TOP_E_NOMEM;
  const int B = pb_in->B;
  if (B == 0 || !pb_in->seg_offset) return B == 0 ? TOP_OK : TOP_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TOP_CUDA(h, cudaSetDevice(h->device));
  const bool host = pb_in->memory == TOP_MEM_HOST;
  if (host) {
    std::memcpy(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1));
  } else {
    TOP_CUDA(h, cudaMemcpyAsync(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaStreamSynchronize(st));
  }
  const int S = h->h_off[B];
  if (S < 0 || S > h->cfg.max_segments) return TOP_E_NOMEM;
  // scratch outputs in the problem's memory kind
  const size_t bytes = sizeof(double) * (24 * (size_t)S + 3 * (size_t)B) + 2 * sizeof(int32_t) * B + 64;
  unsigned char *buf = nullptr;
  if (host) {
    buf = (unsigned char *)std::malloc(bytes);
    if (!buf) return TOP_E_NOMEM;
  } else {
    cudaError_t e = cudaMalloc((void **)&buf, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, e); }
  }
  top_result r{};
  r.coeffs = (double *)buf;
  r.cost = r.coeffs + 24 * (size_t)S;
  r.r_primal = r.cost + B;
  r.r_dual = r.r_primal + B;
  r.iters = (int32_t *)(r.r_dual + B);
  r.status = r.iters + B;
  top_problem pb = *pb_in;
  pb.max_iters = iters;
  pb.eps = 0.0;
  const int saved = h->cfg.segs_per_cta;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = TOP_OK, best = saved, q = 0;
  float best_ms = -1.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = cuda_fail(h, cudaErrorUnknown);
  for (int C = 512; rc == TOP_OK && C >= 128; C -= 64, ++q) {
    h->cfg.segs_per_cta = C;
    float t = -1.0f;
    if (resident_capacity(h, &pb) == C) {
      rc = top_solve(h, &pb, &r, stream);  // untimed: plan, workspace, first-touch
      if (rc == TOP_OK) {
        cudaEventRecord(e0, st);
        rc = top_solve(h, &pb, &r, stream);
        cudaEventRecord(e1, st);
        if (rc == TOP_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
      }
      if (rc == TOP_OK && t > 0.0f && (best_ms < 0.0f || t < best_ms)) { best_ms = t; best = C; }
    }
    if (ms && q < n_ms) ms[q] = t;
  }
  for (; ms && q < n_ms; ++q) ms[q] = -1.0f;
  h->cfg.segs_per_cta = (rc == TOP_OK && best_ms > 0.0f) ? best : saved;
  h->plan_valid = false;
  // the two forms of the G product at the chosen capacity, where the choice applies
  const bool gemm_applies = h->cfg.precision == TOP_FP32 && pb.inner == TOP_CLOSED_FORM && pb.M_box == 0 &&
                            pb.M_ball == 0 && pb.M_vn == 0 && pb.M_gen == 0 && pb.M_poly == 0 && !pb.adaptive_rho;
  float tg[2] = {-1.0f, -1.0f};
  if (rc == TOP_OK && best_ms > 0.0f && gemm_applies) {
    const int saved_form = h->cfg.gemm_form;
    for (int f = 0; f < 2 && rc == TOP_OK; ++f) {
      h->cfg.gemm_form = f == 0 ? TOP_GEMM_CUDA_CORES : TOP_GEMM_TENSOR;
      rc = top_solve(h, &pb, &r, stream);  // untimed
      if (rc == TOP_OK) {
        cudaEventRecord(e0, st);
        rc = top_solve(h, &pb, &r, stream);
        cudaEventRecord(e1, st);
        if (rc == TOP_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&tg[f], e0, e1);
      }
    }
    h->cfg.gemm_form = (rc == TOP_OK && tg[0] > 0.0f && tg[1] > 0.0f)
                           ? (tg[1] < tg[0] ? TOP_GEMM_TENSOR : TOP_GEMM_CUDA_CORES)
                           : saved_form;
  }
  if (ms && n_ms > 7) ms[7] = tg[0];
  if (ms && n_ms > 8) ms[8] = tg[1];
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (host) std::free(buf); else cudaFree(buf);
  if (rc == TOP_OK && out_segs_per_cta) *out_segs_per_cta = h->cfg.segs_per_cta;
  return rc;
}

int top_sample(top_handle *h, const top_problem *pb, const double *coeffs, int32_t M, int32_t order, double *out,
               void *stream) {
  if (!h || !pb || !coeffs || !out || M < 2 || order < 0 || order > 3) return TOP_E_INVAL;
  if (pb->B < 0 || (pb->memory != TOP_MEM_DEVICE && pb->memory != TOP_MEM_HOST)) return TOP_E_INVAL;
  if (pb->B > h->cfg.max_batch) return TOP_E_NOMEM;
  const int B = pb->B;
  if (B == 0) return TOP_OK;
  if (!pb->seg_offset) return TOP_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TOP_CUDA(h, cudaSetDevice(h->device));
  const bool host = pb->memory == TOP_MEM_HOST;
  if (host) {
    std::memcpy(h->h_off, pb->seg_offset, sizeof(int32_t) * (B + 1));
  } else {
    TOP_CUDA(h, cudaMemcpyAsync(h->h_off, pb->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaStreamSynchronize(st));
  }
  const int32_t *off = h->h_off;
  if (off[0] != 0) return TOP_E_INVAL;
  for (int b = 0; b < B; ++b)
    if (off[b + 1] < off[b]) return TOP_E_INVAL;
  const int S = off[B];
  if (S > h->cfg.max_segments) return TOP_E_NOMEM;
  if (S > 0 && !pb->durations) return TOP_E_INVAL;
  // workspace: start times, totals, and for host memory the staged inputs and samples
  const size_t b_ts = align_up(sizeof(double) * (size_t)S + 8, 256), b_tt = align_up(sizeof(double) * B, 256);
  const size_t b_off = align_up(sizeof(int32_t) * (B + 1), 256), b_T = align_up(sizeof(double) * (size_t)S + 8, 256);
  const size_t b_c = align_up(sizeof(double) * 24 * (size_t)S + 8, 256);
  const size_t b_out = align_up(sizeof(double) * 3 * (size_t)B * M, 256);
  const size_t want = b_ts + b_tt + (host ? b_off + b_T + b_c + b_out : 0);
  cudaError_t ge = grow((void **)&h->d_aux, &h->aux_bytes, want);
  if (ge != cudaSuccess) return ge == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, ge);
  unsigned char *base = h->d_aux;
  double *tstart = (double *)base, *ttot = (double *)(base + b_ts);
  const int32_t *d_off = pb->seg_offset;
  const double *d_T = pb->durations, *d_c = coeffs;
  double *d_out = out;
  if (host) {
    unsigned char *p = base + b_ts + b_tt;
    TOP_CUDA(h, cudaMemcpyAsync(p, pb->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, st));
    d_off = (const int32_t *)p;
    p += b_off;
    if (S > 0) TOP_CUDA(h, cudaMemcpyAsync(p, pb->durations, sizeof(double) * S, cudaMemcpyHostToDevice, st));
    d_T = (const double *)p;
    p += b_T;
    if (S > 0) TOP_CUDA(h, cudaMemcpyAsync(p, coeffs, sizeof(double) * 24 * (size_t)S, cudaMemcpyHostToDevice, st));
    d_c = (const double *)p;
    p += b_c;
    d_out = (double *)p;
  }
  int e = launch_sample(d_off, d_T, B, M, order, d_c, tstart, ttot, d_out, st);
  if (e) return cuda_fail(h, (cudaError_t)e);
  if (host)
    TOP_CUDA(h, cudaMemcpyAsync(out, d_out, sizeof(double) * 3 * (size_t)B * M, cudaMemcpyDeviceToHost, st));
  TOP_CUDA(h, cudaStreamSynchronize(st));
  return TOP_OK;
}

int top_time_alloc(top_handle *h, const top_problem *pb_in, double k_T, double lr, int32_t steps,
                   double *durations_io, top_result *res, void *stream) {
  if (!h || !pb_in || !durations_io) return TOP_E_INVAL;
  if (!(k_T >= 0.0) || !(lr > 0.0) || steps < 0) return TOP_E_INVAL;
  if (pb_in->M_gen || pb_in->M_poly || pb_in->adaptive_rho || pb_in->inner != TOP_CLOSED_FORM) return TOP_E_NOTSUP;
  if (pb_in->B < 0 || pb_in->B > h->cfg.max_batch) return pb_in->B < 0 ? TOP_E_INVAL : TOP_E_NOMEM;
  const int B = pb_in->B;
  if (B == 0) return TOP_OK;
  if (!pb_in->seg_offset || !pb_in->waypoints || !pb_in->start_state || !pb_in->end_state) return TOP_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TOP_CUDA(h, cudaSetDevice(h->device));
  const bool host = pb_in->memory == TOP_MEM_HOST;
  if (host) {
    std::memcpy(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1));
  } else {
    TOP_CUDA(h, cudaMemcpyAsync(h->h_off, pb_in->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyDeviceToHost, st));
    TOP_CUDA(h, cudaStreamSynchronize(st));
  }
  const int32_t *off = h->h_off;
  if (off[0] != 0) return TOP_E_INVAL;
  for (int b = 0; b < B; ++b)
    if (off[b + 1] < off[b]) return TOP_E_INVAL;
  const int S = off[B];
  if (S > h->cfg.max_segments) return TOP_E_NOMEM;
  const size_t Jn = (size_t)S + B;
  // workspace: durations, their gradient, dJ = 1, the waypoint-gradient scratch,
  // and for host problems device copies of the inputs
  const size_t bS = align_up(sizeof(double) * (size_t)S + 8, 256), bB = align_up(sizeof(double) * B, 256);
  const size_t bW = align_up(sizeof(double) * 3 * Jn, 256), bOff = align_up(sizeof(int32_t) * (B + 1), 256);
  const size_t bSt = align_up(sizeof(double) * 12 * B, 256);
  // the rows' parameters of a host problem: vbox [B], ball_c [S][3], ball_r [S], vnorm [B]
  const size_t bRows = host ? 2 * bB + align_up(sizeof(double) * 3 * (size_t)S + 8, 256) + bS : 0;
  const size_t want = 2 * bS + bB + bW + (host ? bOff + bW + 2 * bSt + bRows : 0);
  cudaError_t ge = grow((void **)&h->d_aux, &h->aux_bytes, want);
  if (ge != cudaSuccess) return ge == cudaErrorMemoryAllocation ? TOP_E_NOMEM : cuda_fail(h, ge);
  unsigned char *p = h->d_aux;
  double *dT_cur = (double *)p; p += bS;
  double *dT_grad = (double *)p; p += bS;
  double *d_ones = (double *)p; p += bB;
  double *d_wgrad = (double *)p; p += bW;
  top_problem pbd = *pb_in;
  pbd.memory = TOP_MEM_DEVICE;
  if (host) {
    TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, st));
    pbd.seg_offset = (const int32_t *)p; p += bOff;
    TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->waypoints, sizeof(double) * 3 * Jn, cudaMemcpyHostToDevice, st));
    pbd.waypoints = (const double *)p; p += bW;
    TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->start_state, sizeof(double) * 12 * B, cudaMemcpyHostToDevice, st));
    pbd.start_state = (const double *)p; p += bSt;
    TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->end_state, sizeof(double) * 12 * B, cudaMemcpyHostToDevice, st));
    pbd.end_state = (const double *)p; p += bSt;
    if (pb_in->M_box > 0) {
      TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->vbox, sizeof(double) * B, cudaMemcpyHostToDevice, st));
      pbd.vbox = (const double *)p;
    }
    p += bB;
    if (pb_in->M_vn > 0) {
      TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->vnorm, sizeof(double) * B, cudaMemcpyHostToDevice, st));
      pbd.vnorm = (const double *)p;
    }
    p += bB;
    if (pb_in->M_ball > 0) {
      TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->ball_c, sizeof(double) * 3 * S, cudaMemcpyHostToDevice, st));
      pbd.ball_c = (const double *)p;
    }
    p += align_up(sizeof(double) * 3 * (size_t)S + 8, 256);
    if (pb_in->M_ball > 0) {
      TOP_CUDA(h, cudaMemcpyAsync(p, pb_in->ball_r, sizeof(double) * S, cudaMemcpyHostToDevice, st));
      pbd.ball_r = (const double *)p;
    }
    p += bS;
  }
  if (S > 0)
    TOP_CUDA(h, cudaMemcpyAsync(dT_cur, durations_io, sizeof(double) * S,
                                host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  int e = launch_fill(d_ones, B, 1.0, st);
  if (e) return cuda_fail(h, (cudaError_t)e);
  pbd.durations = dT_cur;
  for (int it = 0; it < steps; ++it) {
    int rc = top_grad(h, &pbd, d_ones, d_wgrad, dT_grad, stream);
    if (rc != TOP_OK) return rc;
    e = launch_time_step(dT_cur, dT_grad, S, k_T, lr, st);
    if (e) return cuda_fail(h, (cudaError_t)e);
  }
  if (S > 0)
    TOP_CUDA(h, cudaMemcpyAsync(durations_io, dT_cur, sizeof(double) * S,
                                host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  TOP_CUDA(h, cudaStreamSynchronize(st));
  if (res) {
    top_problem pbs = *pb_in;  // the caller's memory kind, the final durations
    pbs.durations = durations_io;
    return top_solve(h, &pbs, res, stream);
  }
  return TOP_OK;
}

}  // extern "C"
