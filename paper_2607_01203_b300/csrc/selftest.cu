// Diagnostic entry points: the point enclosures of sin/cos/tanh and the tan/sec enclosures used by the
// bound kernels.
#include "internal.h"
#include "interval.cuh"
#include "mlp_math.cuh"
#include "sync.cuh"

namespace leb {
__global__ void point_enclosure_kernel(const float* x, int n, float2* s, float2* c, float2* th) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = x[i];
  const ivl a = point_sin(v), b = point_cos(v), t = point_tanh(v);
  s[i] = make_float2(a.lo, a.hi);
  c[i] = make_float2(b.lo, b.hi);
  th[i] = make_float2(t.lo, t.hi);
}
__global__ void tan_sec_kernel(const float* x, int n, float2* t, float2* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ivl a = iv_tan(iv(x[i])), b = iv_sec(iv(x[i]));
  t[i] = make_float2(a.lo, a.hi);
  sc[i] = make_float2(b.lo, b.hi);
}
// A wait that nothing ends: an mbarrier expecting one arrival that never comes, waited on with the
// kernels' bounded wait and the given limit. It must give up, report LEB_ASYNC_TIMEOUT and return.
__global__ void wait_timeout_kernel(int* flags, unsigned long long limit_ns, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  const unsigned long long t0 = global_ns();
  const bool ok = mbar_wait_for(&bar, 0u, limit_ns);
  *waited_ns = global_ns() - t0;
  if (!ok) atomicOr(flags, LEB_ASYNC_TIMEOUT);
}
}  // namespace leb

extern "C" leb_status leb_selftest_wait_timeout(int* dev_flags, unsigned long long limit_ns,
                                                unsigned long long* dev_waited_ns, void* stream) {
  if (!dev_flags || !dev_waited_ns || limit_ns > 4000000000ull) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
  leb::wait_timeout_kernel<<<1, 32, 0, s>>>(dev_flags, limit_ns, dev_waited_ns);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

extern "C" leb_status leb_selftest_point_enclosures(const float* x, int n, float* out_sin, float* out_cos,
                                                     float* out_tanh, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out_sin || !out_cos || !out_tanh))) return LEB_ERR_INVALID_ARG;
  if (n == 0) return LEB_OK;
  leb::point_enclosure_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      x, n, (float2*)out_sin, (float2*)out_cos, (float2*)out_tanh);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

extern "C" leb_status leb_selftest_tan_sec(const float* x, int n, float* out_tan, float* out_sec, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out_tan || !out_sec))) return LEB_ERR_INVALID_ARG;
  if (n == 0) return LEB_OK;
  leb::tan_sec_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, n, (float2*)out_tan, (float2*)out_sec);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

extern "C" leb_status leb_selftest_set_wait_limit(leb_handle h, unsigned long long limit_ns) {
  if (!h || limit_ns > 4000000000ull) return LEB_ERR_INVALID_ARG;
  leb::Ctx& c = *reinterpret_cast<leb::Ctx*>(h);
  if (c.kind != LEB_DYN_QUAD_CHAIN) return LEB_ERR_UNSUPPORTED;
  c.wait_ns = limit_ns ? limit_ns : 2000000000ull;
  return LEB_OK;
}
