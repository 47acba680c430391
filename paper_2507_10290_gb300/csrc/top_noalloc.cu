// top_noalloc.cu -- top_solve_noalloc: a solve that allocates nothing.
//
// Some callers cannot allocate device memory at solve time: code running
// under an allocator they do not own (a host framework's pool that forbids
// side allocations), a real-time control loop that must not call cudaMalloc
// (it can synchronise the device and take unbounded time), or an embedded
// process whose memory budget is fixed at start-up.  They cannot create a
// top_handle, because top_create allocates its workspace.  This entry point
// instead keeps the solver's scratch (the packed local-matrix inverses, the
// CTA pack table and an error flag) in one file-scope device array of fixed
// size, which every GPU that loads the library holds until the process exits.
//
// The caller still passes its own input and output buffers (device memory).
// Limits: at most TOP_NOALLOC_MAX_SEGMENTS segments and TOP_NOALLOC_MAX_BATCH
// trajectories per call, and every trajectory must fit one CTA of the
// resident kernel (the streaming form needs allocated state); larger problems
// are rejected with TOP_E_LIMIT.  Every call shares the one array and leaves
// its contents behind; the inverses and the pack table are rewritten and the
// error flag cleared by each call, so no state leaks between calls, but calls
// whose work overlaps on the GPU (other streams, other host threads) race on
// the array and must be serialised by the caller.
//
// Host code never uses the array's name as a device address (in host code it
// is only a stand-in symbol): the first call on each device, with that device
// current, looks the address up once with cudaGetSymbolAddress and keeps it.
// The kept address belongs to the device's primary context: it stays valid
// while that context lives, which is the whole process unless the caller
// resets the device (cudaDeviceReset), after which no call may be made on
// that device.  No cudaMalloc, cudaFree or allocating library routine is
// called here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/top.h"
#include "top_internal.h"
#include "top_math.cuh"

using namespace top;

namespace {

constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kMaxSeg = TOP_NOALLOC_MAX_SEGMENTS;
constexpr size_t kMaxBatch = TOP_NOALLOC_MAX_BATCH;
constexpr size_t kGBytes = (size_t)NG * kMaxSeg * sizeof(double);      // FP64 worst case
constexpr size_t kPackOff = round256(kGBytes);
constexpr size_t kPackBytes = sizeof(Pack) * kMaxBatch;                 // at most one pack per trajectory
constexpr size_t kListOff = round256(kPackOff + kPackBytes);
constexpr size_t kListBytes = sizeof(int) * kMaxBatch;                  // trajectory list of the packs
constexpr size_t kErrOff = round256(kListOff + kListBytes);
constexpr size_t kStallOff = round256(kErrOff + 256);                    // [B][3] stall-rule state
constexpr size_t kScratchBytes = kStallOff + sizeof(double) * 3 * kMaxBatch;

constexpr int kMaxDevices = 64;
struct DevSlot {
  bool ready = false;
  unsigned char *ptr = nullptr;  // device address of the scratch array on this device
  int smem_optin = 0;
};
DevSlot g_slots[kMaxDevices];
std::mutex g_setup_mutex;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

int setup_device(int dev, DevSlot **out) {
  if (dev < 0 || dev >= kMaxDevices) return TOP_E_NOTSUP;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DevSlot &s = g_slots[dev];
  if (!s.ready) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return TOP_E_CUDA;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return TOP_E_CUDA;
    s.ptr = (unsigned char *)p;
    s.smem_optin = optin;
    s.ready = true;
  }
  *out = &s;
  return TOP_OK;
}

}  // namespace

extern "C" int top_solve_noalloc(const top_problem *pb, top_result *res, int precision, void *stream) {
  if (!pb || !res) return TOP_E_INVAL;
  if (precision != TOP_FP32 && precision != TOP_FP64) return TOP_E_INVAL;
  if (pb->memory != TOP_MEM_DEVICE) return TOP_E_NOTSUP;
  if (pb->B < 0 || pb->max_iters < 0 || pb->check_every < 0 || pb->stall_checks < 0 || !(pb->rho > 0.0) || !(pb->rho < 1e300) ||
      !(pb->eps >= 0.0))
    return TOP_E_INVAL;
  if (pb->mode != TOP_PIN && pb->mode != TOP_FREE) return TOP_E_INVAL;
  if (pb->inner != TOP_CLOSED_FORM && pb->inner != TOP_NUMERIC) return TOP_E_INVAL;  // as top_solve
  if (pb->inner != TOP_CLOSED_FORM || pb->M_gen != 0) return TOP_E_NOTSUP;
  if (pb->adaptive_rho != 0) return TOP_E_NOTSUP;  // the fixed scratch has no room for the adaptive-rho data
  if (pb->M_poly != 0) return TOP_E_NOTSUP;        // nor for the polytope family's per-axis inverses
  if (pb->M_box < 0 || pb->M_ball < 0 || pb->M_vn < 0) return TOP_E_INVAL;
  if ((pb->M_box && !pb->vbox) || (pb->M_ball && (!pb->ball_c || !pb->ball_r)) || (pb->M_vn && !pb->vnorm))
    return TOP_E_INVAL;
  if ((size_t)pb->B > kMaxBatch) return TOP_E_LIMIT;
  if (pb->B == 0) return TOP_OK;
  if (!pb->seg_offset || !pb->waypoints || !pb->start_state || !pb->end_state || !res->coeffs || !res->cost ||
      !res->r_primal || !res->r_dual || !res->iters || !res->status)
    return TOP_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TOP_E_CUDA;
  DevSlot *slot = nullptr;
  int rc = setup_device(dev, &slot);
  if (rc != TOP_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int B = pb->B;
  int32_t off[kMaxBatch + 1];
  if (cudaMemcpyAsync(off, pb->seg_offset, sizeof(int32_t) * (B + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TOP_E_CUDA;
  if (off[0] != 0) return TOP_E_INVAL;
  for (int b = 0; b < B; ++b)
    if (off[b + 1] < off[b]) return TOP_E_INVAL;
  const int S = off[B];
  if ((size_t)S > kMaxSeg) return TOP_E_LIMIT;
  if (S > 0 && !pb->durations) return TOP_E_INVAL;

  // resident capacity for this problem's families in this precision
  int fam = 0;
  if (pb->M_box > 0) fam |= FAM_BOX;
  if (pb->M_ball > 0) fam |= FAM_BALL;
  if (pb->M_vn > 0) fam |= FAM_VN;
  const int rb = precision == TOP_FP64 ? 8 : 4;
  int cap = 0;
  for (int C = (precision == TOP_FP64 ? 256 : 512); C >= 32 && cap == 0; C -= 32)  // FP64: 256 threads per CTA
    if (res_layout_resident(C, C / 4, pb->M_box, pb->M_ball, pb->M_vn, rb).total <= (size_t)slot->smem_optin) cap = C;
  if (cap == 0) return TOP_E_LIMIT;
  Pack packs[kMaxBatch];
  int npack = 0, max_nseg = 0, max_ntraj = 0;
  const int ntp_cap = std::max(1, cap / 4);
  for (int b = 0; b < B;) {
    if (off[b + 1] - off[b] > cap) return TOP_E_LIMIT;
    Pack pk{b, 0, 0, 0};  // consecutive trajectories: the list is the identity
    while (b < B) {
      const int n2 = off[b + 1] - off[b];
      if (n2 > cap || pk.nseg + n2 > cap || pk.ntraj + 1 > ntp_cap) break;
      pk.nseg += n2;
      pk.ntraj += 1;
      ++b;
    }
    packs[npack++] = pk;
    max_nseg = std::max(max_nseg, pk.nseg);
    max_ntraj = std::max(max_ntraj, pk.ntraj);
  }

  unsigned char *base = slot->ptr;
  void *G = base;
  Pack *d_packs = (Pack *)(base + kPackOff);
  int *d_list = (int *)(base + kListOff);
  int *d_err = (int *)(base + kErrOff);
  DevProblem dp{};
  dp.B = B; dp.S = S; dp.err = d_err; dp.stall = pb->stall_checks;
  dp.seg_offset = pb->seg_offset; dp.waypoints = pb->waypoints; dp.durations = pb->durations;
  dp.start_state = pb->start_state; dp.end_state = pb->end_state;
  dp.mode = pb->mode; dp.inner = pb->inner; dp.rho = pb->rho; dp.eps = pb->eps;
  dp.max_iters = pb->max_iters; dp.check_every = pb->check_every > 0 ? pb->check_every : 1;
  dp.M_box = pb->M_box; dp.vbox = pb->vbox;
  dp.M_ball = pb->M_ball; dp.ball_c = pb->ball_c; dp.ball_r = pb->ball_r;
  dp.M_vn = pb->M_vn; dp.vnorm = pb->vnorm;
  DevResult dr{};
  dr.coeffs = res->coeffs; dr.cost = res->cost; dr.r_primal = res->r_primal; dr.r_dual = res->r_dual;
  dr.history = res->history; dr.iters = res->iters; dr.status = res->status; dr.rho = res->rho;

  if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return TOP_E_CUDA;
  if (cudaMemsetAsync(dr.cost, 0, sizeof(double) * B, st) != cudaSuccess ||
      cudaMemsetAsync(dr.r_primal, 0, sizeof(double) * B, st) != cudaSuccess ||
      cudaMemsetAsync(dr.r_dual, 0, sizeof(double) * B, st) != cudaSuccess ||
      cudaMemsetAsync(dr.iters, 0, sizeof(int32_t) * B, st) != cudaSuccess ||
      cudaMemsetAsync(dr.status, 0, sizeof(int32_t) * B, st) != cudaSuccess)
    return TOP_E_CUDA;
  const bool fp64 = precision == TOP_FP64;
  if (launch_kinv(dp, pb->rho, fp64 ? nullptr : G, fp64 ? G : nullptr, d_err, st) != 0) return TOP_E_CUDA;
  if (cudaMemcpyAsync(d_packs, packs, sizeof(Pack) * npack, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return TOP_E_CUDA;
  int ident[kMaxBatch];
  for (int b = 0; b < B; ++b) ident[b] = b;
  if (cudaMemcpyAsync(d_list, ident, sizeof(int) * B, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return TOP_E_CUDA;
  const int C = std::max(32, (max_nseg + 31) / 32 * 32);
  const int ntp = std::max(1, max_ntraj);
  const ResLayout L = res_layout_resident(C, ntp, (fam & FAM_BOX) ? pb->M_box : 0, (fam & FAM_BALL) ? pb->M_ball : 0,
                                 (fam & FAM_VN) ? pb->M_vn : 0, rb);
  ResidentArgs ra{};
  ra.p = dp; ra.r = dr; ra.G = G; ra.packs = d_packs; ra.traj_list = d_list; ra.ntp = ntp;
  ra.stall = pb->stall_checks > 0 ? (double *)(base + kStallOff) : nullptr;
  const int e = fp64 ? launch_resident_f64(ra, npack, C, L.total, fam, st)
                     : launch_resident_f32(ra, npack, C, L.total, fam, st);
  if (e != 0) return TOP_E_CUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TOP_E_CUDA;
  if (herr & 1) return TOP_E_INVAL;
  if (herr & 2) return TOP_E_NUMERIC;
  if (herr & 4) return TOP_E_BOUNDS;
  return TOP_OK;
}
