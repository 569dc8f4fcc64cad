// leb_bounds_static: the path-based Hessian bounds without any caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need bounds: a real-time control
// loop whose memory is fixed after start-up (an allocation can block for an unbounded time and may fail),
// a host without a general-purpose allocator around the CUDA context, or a framework that hands over only
// input and output buffers. For them this entry point keeps its scratch (the work-list counter and the
// per-trajectory prefix sums of uneven batches) in a file-scope device array owned by the library.
//
// That array lives in every GPU that loads the library until the process exits. In host code its name
// is only a host-side stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call on that device and cached (a device
// reset reloads the module and makes the cached address stale: no call after a reset). All
// calls share the array: the counter is cleared at the start of every call, and calls whose work overlaps
// on the GPU (different streams, or different host threads on one device) race on it and must not be
// issued concurrently.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace leb {

constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr size_t kStaticHeader = 256;
// prefix sums: two 8-byte entries per trajectory, plus one
constexpr int kStaticMaxTraj = (int)((kStaticScratchBytes - kStaticHeader) / 16) - 1;

static __device__ __align__(256) unsigned char leb_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, leb_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace leb

using namespace leb;

extern "C" leb_status leb_bounds_static(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                        const float* u_nom, const leb_set* set, float* r_lo, float* r_hi, float* A,
                                        float* B, int* dev_flags, void* stream) {
  if (!h || !set || T < 0 || !dev_flags) return LEB_ERR_INVALID_ARG;
  const Ctx& c = *reinterpret_cast<const Ctx*>(h);
  if (c.kind == LEB_DYN_MLP) return LEB_ERR_UNSUPPORTED;
  if (T > 0 && (!x_nom || !u_nom || !r_lo || !r_hi)) return LEB_ERR_INVALID_ARG;
  if (c.kind == LEB_DYN_SATELLITE || c.kind == LEB_DYN_QUAD3D) {   // no scratch needed
    if (set->kind != LEB_SET_BOX && set->kind != LEB_SET_ZONO) return LEB_ERR_INVALID_ARG;
    if (T > 0 && set->kind == LEB_SET_BOX && !set->radii) return LEB_ERR_INVALID_ARG;
    // what these models do not support is refused before anything is queued on the stream
    if (set->kind != LEB_SET_BOX || (batch && batch->traj_nquads)) return LEB_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
    if (T == 0) return LEB_OK;
    return pbh_sys_bounds(c, batch, T, x_nom, u_nom, set, r_lo, r_hi, A, B, nullptr, dev_flags, s);
  }
  if (set->kind != LEB_SET_BOX && set->kind != LEB_SET_ZONO) return LEB_ERR_INVALID_ARG;
  if (T > 0 && set->kind == LEB_SET_BOX && !set->radii) return LEB_ERR_INVALID_ARG;
  if (T > 0 && set->kind == LEB_SET_ZONO && (!set->G || set->n_gen < 1)) return LEB_ERR_INVALID_ARG;
  const int n_traj = batch ? batch->n_traj : 0;
  if (batch && (n_traj < 1 || !batch->traj_offsets)) return LEB_ERR_INVALID_ARG;
  const bool uneven = batch && batch->traj_nquads;
  if (uneven && n_traj > kStaticMaxTraj) return LEB_ERR_WORKSPACE;  // beyond the fixed scratch
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return LEB_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
  if (T == 0) return LEB_OK;
  char* ws = (char*)scratch;
  PbhArgs a{};
  a.x_nom = x_nom;
  a.u_nom = u_nom;
  a.center = set->center;
  a.radii = set->radii;
  a.G = set->G;
  a.n_gen = set->n_gen;
  a.zono = set->kind == LEB_SET_ZONO;
  a.r_lo = r_lo;
  a.r_hi = r_hi;
  a.A = A;
  a.B = B;
  a.flags = dev_flags;
  a.T = T;
  a.nq = c.nq;
  a.n_traj = n_traj;
  a.traj_offsets = batch ? batch->traj_offsets : nullptr;
  a.traj_nquads = uneven ? batch->traj_nquads : nullptr;
  a.counter = (int*)ws;
  a.pre1 = (const long long*)(ws + kStaticHeader);
  a.pre2 = (const long long*)(ws + kStaticHeader) + (n_traj + 1);
  a.k = c.qk;
  // the counter must start at zero on every call (the array keeps the previous call's contents)
  if (cudaMemsetAsync(ws, 0, kStaticHeader, s) != cudaSuccess) return LEB_ERR_CUDA;
  if (uneven && launch_prefix(batch->traj_offsets, batch->traj_nquads, n_traj, (long long*)a.pre1, (long long*)a.pre2,
                              s) != cudaSuccess)
    return LEB_ERR_CUDA;
  const PbhPlan& p = (c.plan_index >= 0 && c.plan_index < (int)c.pbh_candidates.size()) ? c.pbh_candidates[c.plan_index]
                                                                                          : c.pbh_plan;
  return launch_pbh(c, a, p, s) == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

extern "C" int leb_bounds_static_max_traj(void) { return kStaticMaxTraj; }
