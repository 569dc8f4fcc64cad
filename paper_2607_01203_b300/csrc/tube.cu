// The step after the LEB (Sec. V-A): the zonotope generator matrix Ebar_j = [E(z_j) R_j] (Eq. 18b) of
// every timestep and the tube centre and width of Eqs. 20-21,
//
//     h^mu_k[l]    = sum_{j<k} sum_i Phi_{k,j}[l,i] c_j[i],
//     h^sigma_k[l] = sum_{j<k} || (Phi_{k,j} Ebar_j)[l,:] ||_1 = sum_{j<k} sum_i |Phi_{k,j}[l,i]| (|e_j[i]| + r_j[i]),
//
// the second form because E(z_j) = diag(e_j) and R_j = diag(r_j) are diagonal (the Gamma map of
// Sec. IV-C and the paper's constant disturbance scaling), so the row-wise l1 norm of the product splits
// column by column. Both are read-once streams of the packed responses Phi: HBM-bound.
//
// Soundness: h^sigma is summed with every product and sum rounded up (all terms are non-negative);
// h^mu is enclosed with directed roundings, returned at its midpoint, and the enclosure's half-width is
// added to the width, so [mu - sigma, mu + sigma] contains the exact box of the FP32 inputs.
//
// Layout: one CTA per (k, trajectory, 32 rows), CTAs ordered by decreasing k (the work of a CTA grows
// with k, so the longest start first and the short ones fill in); the CTA stages c_j and
// w_j = |e_j| + r_j (rounded up) of its trajectory's timesteps j < k in shared memory, and each warp
// walks its rows l of the k-th block row as one range of float4 chunks over all j (n_x a multiple of 4;
// scalar otherwise), three FMAs per element, four chunks in flight per lane.
#include <math_constants.h>

#include <cstdint>

#include "internal.h"

namespace leb {
namespace {

constexpr int kTubeThreads = 256;
constexpr int kTubeRows = 32;   // rows of a block row per CTA (4 per warp)

struct TubeArgs {
  const float* Phi;
  const float* e;
  int e_per_step;
  const float* c;
  const float* r;
  float* mu;
  float* sigma;
  int* flags;
  int n_traj, N, n_x, n_rows;
  unsigned long long magic;   // ceil(2^32 / (n_x / 4)): exact q / (n_x / 4) for the chunk indices used
};

template <bool kVec>
__global__ void __launch_bounds__(kTubeThreads, 4) tube_kernel(TubeArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int N = a.N, n_x = a.n_x, n_rows = a.n_rows;
  // CTA = (k, trajectory, chunk of kTubeRows rows), k-major and largest k first
  const int nchunk = (n_rows + kTubeRows - 1) / kTubeRows;
  const int kidx = blockIdx.x / (a.n_traj * nchunk), rem = blockIdx.x - kidx * a.n_traj * nchunk;
  const int b = rem / nchunk, chunk = rem - b * nchunk;
  const int k = N - kidx;                                  // 1 .. N, largest first
  float* s_c = sm;                                         // [k][n_x]
  float* s_w = sm + (size_t)k * n_x;                       // [k][n_x]
  const long long t0 = (long long)b * N;                   // timestep 0 of the trajectory
  for (int e = threadIdx.x; e < k * n_x; e += blockDim.x) {
    const int j = e / n_x, i = e - j * n_x;
    const float ev = a.e[(a.e_per_step ? (t0 + j) * n_x : 0) + i];
    s_c[e] = a.c[(t0 + j) * n_x + i];
    s_w[e] = __fadd_ru(fabsf(ev), a.r[(t0 + j) * n_x + i]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const long long P = (long long)N * (N + 1) / 2;
  const float* blk0 = a.Phi + ((long long)b * P + (long long)k * (k - 1) / 2) * n_rows * n_x;   // Phi_{k,0}
  const long long out_k = ((long long)b * (N + 1) + k) * n_rows;
  bool bad = false;
  const int l_end = min(n_rows, (chunk + 1) * kTubeRows);
  for (int l = chunk * kTubeRows + warp; l < l_end; l += nwarps) {
    float s = 0.f, lo = 0.f, hi = 0.f;
    if constexpr (kVec) {
      // the row's k blocks as one range of k * n_x / 4 float4 chunks: chunk q is column group
      // q - j cpr of block j = q / cpr, and the staged c_j, w_j are indexed by q directly
      const int cpr = n_x >> 2, total = k * cpr;
      const float4* row0 = reinterpret_cast<const float4*>(blk0 + (long long)l * n_x);
      const float4* c4 = reinterpret_cast<const float4*>(s_c);
      const float4* w4 = reinterpret_cast<const float4*>(s_w);
      const long long jstride = (long long)n_rows * cpr;   // float4 between blocks j and j + 1
      auto chunk = [&](int q) {   // address of chunk q of this row
        const int j = (int)(((unsigned long long)(unsigned)q * a.magic) >> 32);   // q / cpr
        return row0 + (long long)j * jstride + (q - j * cpr);
      };
      auto acc = [&](const float4& p, int q) {
        const float4 cc = c4[q];
        const float4 ww = w4[q];
        s = __fmaf_ru(fabsf(p.x), ww.x, s);
        s = __fmaf_ru(fabsf(p.y), ww.y, s);
        s = __fmaf_ru(fabsf(p.z), ww.z, s);
        s = __fmaf_ru(fabsf(p.w), ww.w, s);
        lo = __fmaf_rd(p.x, cc.x, lo);
        lo = __fmaf_rd(p.y, cc.y, lo);
        lo = __fmaf_rd(p.z, cc.z, lo);
        lo = __fmaf_rd(p.w, cc.w, lo);
        hi = __fmaf_ru(p.x, cc.x, hi);
        hi = __fmaf_ru(p.y, cc.y, hi);
        hi = __fmaf_ru(p.z, cc.z, hi);
        hi = __fmaf_ru(p.w, cc.w, hi);
      };
      // four chunks per lane in flight: issue the loads first, then consume (read once: stream past L2)
      int q = lane;
      for (; q + 96 < total; q += 128) {
        const float4 p0 = __ldcs(chunk(q)), p1 = __ldcs(chunk(q + 32)), p2 = __ldcs(chunk(q + 64)),
                     p3 = __ldcs(chunk(q + 96));
        acc(p0, q);
        acc(p1, q + 32);
        acc(p2, q + 64);
        acc(p3, q + 96);
      }
      for (; q < total; q += 32) acc(__ldcs(chunk(q)), q);
    } else {
      for (int j = 0; j < k; ++j) {
        const float* row = blk0 + ((long long)j * n_rows + l) * n_x;
        const float* cj = s_c + j * n_x;
        const float* wj = s_w + j * n_x;
        for (int i = lane; i < n_x; i += 32) {
          const float p = __ldcs(row + i);
          s = __fmaf_ru(fabsf(p), wj[i], s);
          lo = __fmaf_rd(p, cj[i], lo);
          hi = __fmaf_ru(p, cj[i], hi);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s = __fadd_ru(s, __shfl_xor_sync(0xffffffffu, s, o));
      lo = __fadd_rd(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = __fadd_ru(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      float m = 0.5f * lo + 0.5f * hi;
      float w = __fadd_ru(s, fmaxf(__fsub_ru(hi, m), __fsub_ru(m, lo)));
      if (!(isfinite(m) && isfinite(w))) {
        m = 0.f;
        w = CUDART_INF_F;
        bad = true;
      }
      a.mu[out_k + l] = m;
      a.sigma[out_k + l] = w;
    }
  }
  if (k == 1) {   // timestep 0: empty sums
    const long long out0 = (long long)b * (N + 1) * n_rows;
    for (int l = chunk * kTubeRows + threadIdx.x; l < l_end; l += blockDim.x) {
      a.mu[out0 + l] = 0.f;
      a.sigma[out0 + l] = 0.f;
    }
  }
  if (bad) atomicOr(a.flags, LEB_ASYNC_NONFINITE);
}

}  // namespace
}  // namespace leb

using namespace leb;

extern "C" leb_status leb_tube(int n_traj, int N, int n_x, int n_u, const float* Phi, const float* e, int e_per_step,
                               const float* c, const float* r, float* mu, float* sigma, int* dev_flags,
                               void* stream) {
  if (n_traj < 0 || N < 0 || n_x < 1 || n_u < 0 || !dev_flags) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
  if (n_traj == 0) return LEB_OK;
  if (!mu || !sigma) return LEB_ERR_INVALID_ARG;
  const int n_rows = n_x + n_u;
  if (N == 0) {   // only timestep 0: empty sums
    if (cudaMemsetAsync(mu, 0, (size_t)n_traj * n_rows * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(sigma, 0, (size_t)n_traj * n_rows * sizeof(float), s) != cudaSuccess)
      return LEB_ERR_CUDA;
    return LEB_OK;
  }
  if (!Phi || !e || !c || !r) return LEB_ERR_INVALID_ARG;
  const size_t smem = (size_t)2 * N * n_x * sizeof(float);   // c_j and w_j of the largest k
  if (smem > 200 * 1024) return LEB_ERR_UNSUPPORTED;
  if ((long long)n_traj * N > 0x7fffffffLL) return LEB_ERR_UNSUPPORTED;
  const unsigned long long cpr = (unsigned long long)(n_x / 4 > 0 ? n_x / 4 : 1);
  TubeArgs a{Phi, e, e_per_step, c, r, mu, sigma, dev_flags, n_traj, N, n_x, n_rows, (0x100000000ULL + cpr - 1) / cpr};
  const bool vec = (n_x % 4 == 0) && ((reinterpret_cast<uintptr_t>(Phi) & 15u) == 0);
  const cudaError_t ea = vec ? cudaFuncSetAttribute(tube_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem)
                             : cudaFuncSetAttribute(tube_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem);
  if (ea != cudaSuccess) return LEB_ERR_CUDA;
  const long long grid_ll = (long long)n_traj * N * ((n_rows + kTubeRows - 1) / kTubeRows);
  if (grid_ll > 0x7fffffffLL) return LEB_ERR_UNSUPPORTED;
  const int grid = (int)grid_ll;
  if (vec) tube_kernel<true><<<grid, kTubeThreads, smem, s>>>(a);
  else tube_kernel<false><<<grid, kTubeThreads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}
