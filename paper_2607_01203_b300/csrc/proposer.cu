// Learned LEB proposer: a ReLU MLP n_in -> H -> H -> n_out that maps (x~_k, u~_k, state radii) to
// standardised (r_lo, r_hi). It only proposes bounds; the certified kernels stay the final answer and
// the measure of its error. (An addition to the paper's method.)
//
// Training and inference run in this file's kernels: GEMMs with operands rounded to BF16 and FP32
// accumulation, bias/ReLU epilogues, mean-squared-error gradient, column sums for the bias gradients,
// and a fused Adam update of the FP32 master weights.
#include <cmath>
#include <cstring>
#include <cuda_bf16.h>
#include <new>
#include <vector>
#include <algorithm>

#include "internal.h"
#include "tc_ptx.cuh"

struct leb_proposer_s {
  int n_in = 0, H = 0, n_out = 0;
  float* W[3] = {};
  float* b[3] = {};
  float* gW[3] = {};
  float* gb[3] = {};
  float* mW[3] = {};
  float* vW[3] = {};
  float* mb[3] = {};
  float* vb[3] = {};
  float* norm = nullptr;  // in_mean [n_in], in_std [n_in], out_mean [n_out], out_std [n_out]
  int* periodic = nullptr;  // [n_in] 1: the input is an angle, wrapped to [-pi, pi) before standardising
  int step = 0;
  // inference on the tensor cores: BF16 copies of the weights (refreshed by every forward call) and their
  // tensor maps; tc = false when the shapes do not fit the tcgen05 GEMM (then the CUDA-core GEMMs run)
  bool tc = false;
  int w_version = 0, wb_version = -1;   // bumped by every weight change; the BF16 copies' version
  __nv_bfloat16* Wb[3] = {};
  CUtensorMap wmap[3];
  int parts[3] = {};                    // column parts of each layer (one CTA each per 128-row tile)
};

namespace leb {

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------------------------------------------
// Inference GEMM on the tensor cores: C[M, N] = A[M, K] W[N, K]^T + bias (ReLU), A and W in BF16
// (K-major, 128-byte swizzled tiles by TMA, zero fill past K and M), FP32 accumulation in TMEM.
// One CTA = 128 rows of A and the N columns [n0, n0 + N) of part n0 = blockIdx.y N of the layer's output
// (TMEM columns), issued as nchunk MMAs of N / nchunk columns (a multiple of 16, at most 256). The layers
// are split into parts of at most 128 columns, so that a tile's epilogue is spread over several CTAs. Warp 0 lane 0 loads, warp 1 lane 0 issues the MMAs, all four
// warps read TMEM (thread = row) for the epilogue, which writes BF16 (the next layer's operand) or FP32
// (the output, optionally taken back out of its standardisation: y std + mean).
// Every wait is bounded; a wait that runs out leaves the tile's outputs NaN.
// ---------------------------------------------------------------------------------------------------
constexpr int kPtMaxStages = 8;
constexpr int kPtATile = 128 * 64 * 2;     // 16 KB
constexpr int kPtSmem = 227 * 1024 - 64;   // the largest launch: as many ring stages of (16 KB + N x 128 B) as fit

// Stages of the K ring for N output columns. Up to 256 columns, two stages, so that two CTAs share an SM
// (their TMEM, 2 x 256 columns, fits too) and one CTA's epilogue overlaps the other's MMAs; wider
// layers take as many stages as fit one CTA per SM.
static inline int pt_stages(int N) {
  if (N <= 256) return 2;
  const int per = kPtATile + N * 128;
  const int st = (kPtSmem - 1024 - 2 * kPtMaxStages * 8 - 8) / per;
  return st < kPtMaxStages ? st : kPtMaxStages;
}
// Dynamic shared memory of a launch: alignment slack, the ring, its barriers and the accumulator barrier.
static inline int pt_smem(int N, int stages) { return 1024 + stages * (kPtATile + N * 128) + (2 * stages + 1) * 8; }

__global__ void __launch_bounds__(128, 2) prop_tc_gemm_kernel(const __grid_constant__ CUtensorMap amap,
                                                              const __grid_constant__ CUtensorMap wmap, int M, int N,
                                                              int K, int nchunk, const float* bias, int relu,
                                                              __nv_bfloat16* outb, float* outf, int ldo,
                                                              const float* omean, const float* ostd, int stages) {
  extern __shared__ uint8_t sraw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sraw) + 1023) & ~uintptr_t(1023));
  const int btile = N * 128;                              // N rows x 64 K x 2 bytes (a multiple of 1 KB)
  uint8_t* At = base;                                        // [stages][16 KB]
  uint8_t* Bt = base + stages * kPtATile;                 // [stages][N x 128 B]
  uint64_t* full = reinterpret_cast<uint64_t*>(Bt + stages * btile);
  uint64_t* empty = full + stages;
  uint64_t* acc = empty + stages;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128, nK = (K + 63) / 64, nb = N / nchunk;
  const int n0 = blockIdx.y * N;   // this CTA's columns [n0, n0 + N) of the layer's output
  const uint32_t tcols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : (N <= 256 ? 256 : 512)));
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc, 1);
    mbar_fence_init();
    s_fail = 0;
  }
  if (warp == 1) tmem_alloc(&tmem_slot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t abytes = kPtATile, bbytes = (uint32_t)N * 128u;
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&amap);
    tma_prefetch_desc(&wmap);
    for (int kb = 0; kb < nK; ++kb) {
      const int s = kb % stages;
      if (kb >= stages && !mbar_wait(&empty[s], ((kb / stages) - 1) & 1u)) { s_fail = 1; break; }
      mbar_arrive_expect_tx(&full[s], abytes + bbytes);
      tma_load_2d(At + s * kPtATile, &amap, kb * 64, m0, &full[s]);
      for (int c = 0; c < nchunk; ++c)
        tma_load_2d(Bt + s * btile + c * nb * 128, &wmap, kb * 64, n0 + c * nb, &full[s]);
    }
    // every posted copy lands before the block can exit
    for (int kb = nK > stages ? nK - stages : 0; kb < nK; ++kb) mbar_wait(&full[kb % stages], (kb / stages) & 1u);
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_f16(128, nb, 1);
    bool ok = true;
    for (int kb = 0; kb < nK && ok; ++kb) {
      const int s = kb % stages;
      if (!mbar_wait(&full[s], (kb / stages) & 1u)) { ok = false; s_fail = 1; break; }
      tc_fence_after();
      const uint32_t a0 = smem_u32(At + s * kPtATile), b0 = smem_u32(Bt + s * btile);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        for (int c = 0; c < nchunk; ++c)
          tc_mma_f16(tmem + (uint32_t)(c * nb), sw128_desc(a0 + kk * 32), sw128_desc(b0 + c * nb * 128 + kk * 32),
                     idesc, (kb > 0 || kk > 0) ? 1u : 0u);
      tc_commit(&empty[s]);
    }
    tc_commit(acc);
  }
  __syncwarp();
  // ---- epilogue: thread = row m0 + 32 warp + lane, TMEM lane of the same index ---------------------
  const bool ok = mbar_wait_warp(acc, 0u) && !*(volatile int*)&s_fail;
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < N; c0 += 16) {
    float v[16];
    tmem_ld16(tl + (uint32_t)c0, v);   // every thread of the warp takes part (sync.aligned)
    if (row >= M) continue;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      float x = ok ? v[e] + bias[n0 + c0 + e] : __int_as_float(0x7fc00000);
      x = relu ? fmaxf(x, 0.f) : x;
      v[e] = omean ? fmaf(x, ostd[n0 + c0 + e], omean[n0 + c0 + e]) : x;   // back to the bounds' units
    }
    if (outb) {
      uint32_t w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        w[e] = *reinterpret_cast<const uint32_t*>(&h);
      }
      uint4* dst = reinterpret_cast<uint4*>(outb + (long long)row * ldo + n0 + c0);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
      float4* dst = reinterpret_cast<float4*>(outf + (long long)row * ldo + n0 + c0);
#pragma unroll
      for (int e = 0; e < 4; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, tcols);
}

// The three weight matrices to their BF16 copies in one launch.
__global__ void prop_weights_bf16_kernel(const float* W0, long long n0, const float* W1, long long n1, const float* W2,
                                         long long n2, __nv_bfloat16* B0, __nv_bfloat16* B1, __nv_bfloat16* B2) {
  const long long total = n0 + n1 + n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    if (i < n0) B0[i] = __float2bfloat16_rn(W0[i]);
    else if (i < n0 + n1) B1[i - n0] = __float2bfloat16_rn(W1[i - n0]);
    else B2[i - n0 - n1] = __float2bfloat16_rn(W2[i - n0 - n1]);
  }
}

__global__ void prop_to_bf16_kernel(long long total, const float* x, __nv_bfloat16* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// C[M, N] = op(A) op(B) (+ bias[N]) (ReLU) or (* (Mask > 0)); operands rounded to BF16, FP32 accumulate.
// op(A)[m, k] = tA ? A[k * lda + m] : A[m * lda + k];  op(B)[k, n] = tB ? B[n * ldb + k] : B[k * ldb + n].
// epi: 0 store, 1 + bias, 2 + bias then ReLU, 3 multiply by (Mask[m, n] > 0).
__global__ void __launch_bounds__(256) prop_gemm_kernel(int M, int N, int K, const float* A, int lda, int tA,
                                                        const float* B, int ldb, int tB, float* C, int ldc,
                                                        const float* bias, const float* Mask, int epi) {
  __shared__ float sa[16][68];
  __shared__ float sb[16][68];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int mm, kk;
      if (tA) { kk = e / 64; mm = e - kk * 64; }
      else { mm = e / 16; kk = e - mm * 16; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < K) v = tA ? A[(long long)k * lda + m] : A[(long long)m * lda + k];
      sa[kk][mm] = bf16r(v);
      int nn, kb;
      if (tB) { nn = e / 16; kb = e - nn * 16; }
      else { kb = e / 64; nn = e - kb * 64; }
      const int n = n0 + nn, k2 = k0 + kb;
      float w = 0.f;
      if (n < N && k2 < K) w = tB ? B[(long long)n * ldb + k2] : B[(long long)k2 * ldb + n];
      sb[kb][nn] = bf16r(w);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sa[kk][4 * ty + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = sb[kk][4 * tx + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + 4 * ty + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + 4 * tx + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (epi == 1 || epi == 2) v += bias[n];
      if (epi == 2) v = fmaxf(v, 0.f);
      if (epi == 3) v = Mask[(long long)m * ldc + n] > 0.f ? v : 0.f;
      C[(long long)m * ldc + n] = v;
    }
  }
}

__device__ __forceinline__ float wrap_pi(float x) {
  const float two_pi = 6.283185307179586f;
  float r = fmodf(x + 3.141592653589793f, two_pi);
  if (r < 0.f) r += two_pi;
  return r - 3.141592653589793f;
}

__global__ void prop_standardize_kernel(long long total, int n, const float* X, const int* periodic, const float* mean,
                                        const float* stdv, float* Xs) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n);
    const float x = periodic[j] ? wrap_pi(X[e]) : X[e];
    Xs[e] = (x - mean[j]) / stdv[j];
  }
}

__global__ void prop_destandardize_kernel(long long total, int n, const float* y, const float* mean, const float* stdv,
                                          float* Y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n);
    Y[e] = fmaf(y[e], stdv[j], mean[j]);
  }
}

// Standardised inputs straight into the BF16 operand of the first layer: a thread per column pair (n
// even) keeps that pair's angle flags, means and deviations in registers and walks kStdRows rows, whose
// loads are independent; a row's pairs are consecutive threads (coalesced).
constexpr int kStdRows = 16;
__global__ void prop_standardize_bf16_kernel(int B, int n, const float* X, const int* periodic, const float* mean,
                                             const float* stdv, __nv_bfloat16* Xb) {
  const int r0 = blockIdx.x * kStdRows, r1 = min(B, r0 + kStdRows);
  for (int c = threadIdx.x; c < (n >> 1); c += blockDim.x) {
    const int j = 2 * c;
    const bool w0 = periodic[j] != 0, w1 = periodic[j + 1] != 0;
    const float m0 = mean[j], m1 = mean[j + 1], s0 = stdv[j], s1 = stdv[j + 1];
#pragma unroll 4
    for (int row = r0; row < r1; ++row) {
      float2 x = reinterpret_cast<const float2*>(X + (long long)row * n)[c];
      if (w0) x.x = wrap_pi(x.x);
      if (w1) x.y = wrap_pi(x.y);
      reinterpret_cast<__nv_bfloat162*>(Xb + (long long)row * n)[c] =
          __floats2bfloat162_rn((x.x - m0) / s0, (x.y - m1) / s1);
    }
  }
}

// dy = 2 (y - t) / (B n) with t the standardised target; loss += mean (y - t)^2
__global__ void prop_mse_kernel(long long total, int n, const float* y, const float* Y, const float* mean,
                                const float* stdv, float* dy, float* loss) {
  float part = 0.f;
  const float scale = 2.f / (float)total;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n);
    const float tgt = (Y[e] - mean[j]) / stdv[j];
    const float d = y[e] - tgt;
    dy[e] = scale * d;
    part = fmaf(d, d, part);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, part / (float)total);
}

__global__ void prop_colsum_kernel(int M, int N, const float* G, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += G[(long long)m * N + n];
  out[n] = s;
}

// column mean and standard deviation (two passes, FP64 accumulation); std floored at 1e-6 (+ tiny)
__global__ void prop_colstats_kernel(int M, int N, const float* X, const int* periodic, float* mean, float* stdv) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const bool wrap = periodic && periodic[n];
  double s = 0.0;
  for (int m = 0; m < M; ++m) s += wrap ? wrap_pi(X[(long long)m * N + n]) : X[(long long)m * N + n];
  const double mu = s / M;
  double v = 0.0;
  for (int m = 0; m < M; ++m) {
    const double d = (wrap ? wrap_pi(X[(long long)m * N + n]) : X[(long long)m * N + n]) - mu;
    v += d * d;
  }
  mean[n] = (float)mu;
  stdv[n] = (float)fmax(sqrt(v / M), 1e-6 * (fabs(mu) + 1e-30)) + 1e-30f;
}

// out_std[j] = max(out_std[j], rel * max_j out_std): one block. Outputs whose spread is far below the
// others' (bounds that are zero up to rounding) are standardised by the floor, so their rounding noise
// does not weigh in the loss like a real target.
__global__ void prop_std_floor_kernel(int N, float* stdv, float rel) {
  __shared__ float red[256];
  float m = 0.f;
  for (int j = threadIdx.x; j < N; j += blockDim.x) m = fmaxf(m, stdv[j]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const float f = rel * red[0];
  for (int j = threadIdx.x; j < N; j += blockDim.x) stdv[j] = fmaxf(stdv[j], f);
}

__global__ void prop_adam_kernel(long long total, float* p, const float* g, float* m, float* v, float lr, float b1,
                                 float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// He-uniform initialisation from a counter-based hash (splitmix64 of seed and index).
__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void prop_init_kernel(long long total, float* W, float bound, unsigned long long seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r = splitmix(seed ^ (unsigned long long)e * 0xD1B54A32D192ED03ull);
    const float u = (float)(r >> 40) * (1.f / 16777216.f);  // [0, 1)
    W[e] = (2.f * u - 1.f) * bound;
  }
}

namespace {

inline int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 16); }

cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, int tA, const float* B, int ldb, int tB,
                 float* C, int ldc, const float* bias, const float* Mask, int epi) {
  dim3 grid((M + 63) / 64, (N + 63) / 64);
  prop_gemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, bias, Mask, epi);
  return cudaGetLastError();
}

// workspace (floats): Xs [B, n_in], h0 [B, H], h1 [B, H], y [B, n_out], dy [B, n_out], d1 [B, H], d0 [B, H]
size_t ws_floats(const leb_proposer_s* p, int B) {
  return (size_t)B * (p->n_in + 4 * p->H + 2 * p->n_out) + 64;
}

}  // namespace
}  // namespace leb

using namespace leb;

// Chunks of an N-column product for the tcgen05 GEMM: the fewest with N / c a multiple of 16, at most 256.
// Column parts of a layer of N outputs: the fewest parts of at most 128 columns (a multiple of 16) each,
// else of at most 256; 0 if N has no such split. Each part is one CTA's single MMA chunk.
static int mma_parts(int N) {
  for (int lim : {128, 256})
    for (int c = 1; c <= N / 16; ++c)
      if (N % c == 0 && (N / c) % 16 == 0 && N / c <= lim) return c;
  return 0;
}

// BF16 weight copies and their tensor maps for tensor-core inference; false only on an allocation
// failure (shapes the GEMM does not take leave p->tc false).
static bool setup_tc(leb_proposer p) {
  const int ins[3] = {p->n_in, p->H, p->H}, outs[3] = {p->H, p->H, p->n_out};
  auto enc = tensor_map_encoder();
  if (!enc || p->n_in % 8 != 0 || p->H % 8 != 0 || p->H > 512 || p->n_out > 512) return true;
  for (int i = 0; i < 3; ++i) {
    p->parts[i] = mma_parts(outs[i]);
    if (p->parts[i] == 0) return true;
  }
  for (int i = 0; i < 3; ++i) {
    if (cudaMalloc(&p->Wb[i], (size_t)ins[i] * outs[i] * 2) != cudaSuccess) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ins[i], (cuuint64_t)outs[i]};
    cuuint64_t strides[1] = {(cuuint64_t)ins[i] * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)(outs[i] / p->parts[i])};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&p->wmap[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p->Wb[i], dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return true;
  }
  if (cudaFuncSetAttribute(prop_tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPtSmem) != cudaSuccess)
    return true;
  p->tc = true;
  return true;
}

// Activations [rows, cols] BF16 as the A operand of the tcgen05 GEMM (box 64 x 128, zero fill).
static bool act_map(CUtensorMap* m, const __nv_bfloat16* x, int rows, int cols) {
  auto enc = tensor_map_encoder();
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  return enc && enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(x), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Inference forward on the tensor cores, written to Y in the bounds' units; false: not taken.
static bool forward_tc(leb_proposer p, int B, const float* X, float* ws, float* Y, cudaStream_t s, leb_status* st) {
  const int n_in = p->n_in, H = p->H, n_out = p->n_out;
  const size_t o1 = 0, o2 = (o1 + ((size_t)B * n_in + 1) / 2 + 3) & ~size_t(3);
  const size_t o3 = (o2 + ((size_t)B * H + 1) / 2 + 3) & ~size_t(3);
  const size_t end = o3 + ((size_t)B * H + 1) / 2;
  // TMA needs 16-byte aligned operands, the epilogue stores Y rows as float4
  if (!p->tc || end > ws_floats(p, B) || ((reinterpret_cast<uintptr_t>(ws) | reinterpret_cast<uintptr_t>(Y)) & 15u) ||
      (reinterpret_cast<uintptr_t>(X) & 7u))
    return false;
  __nv_bfloat16* Xb = reinterpret_cast<__nv_bfloat16*>(ws + o1);
  __nv_bfloat16* H1 = reinterpret_cast<__nv_bfloat16*>(ws + o2);
  __nv_bfloat16* H2 = reinterpret_cast<__nv_bfloat16*>(ws + o3);
  CUtensorMap m0, m1, m2;
  if (!act_map(&m0, Xb, B, n_in) || !act_map(&m1, H1, B, H) || !act_map(&m2, H2, B, H)) return false;
  *st = LEB_ERR_CUDA;
  if (p->wb_version != p->w_version) {   // the weights changed since their last BF16 copy
    const long long n0 = (long long)n_in * H, n1 = (long long)H * H, n2 = (long long)H * n_out;
    prop_weights_bf16_kernel<<<blocks_for(n0 + n1 + n2), 256, 0, s>>>(p->W[0], n0, p->W[1], n1, p->W[2], n2, p->Wb[0],
                                                                        p->Wb[1], p->Wb[2]);
    p->wb_version = p->w_version;
  }
  const int sthreads = std::min(1024, ((n_in / 2) + 31) / 32 * 32);
  prop_standardize_bf16_kernel<<<(B + kStdRows - 1) / kStdRows, sthreads, 0, s>>>(B, n_in, X, p->periodic, p->norm,
                                                                                 p->norm + n_in, Xb);
  const int tiles = (B + 127) / 128;
  const float* omean = p->norm + 2 * n_in;
  // layer i: a CTA per (128-row tile, column part of N / parts columns)
  auto layer = [&](int i, const CUtensorMap& am, int N, int K, int relu, __nv_bfloat16* ob, float* of,
                   const float* mn, const float* sd) {
    const int np = N / p->parts[i], ns = pt_stages(np);
    prop_tc_gemm_kernel<<<dim3(tiles, p->parts[i]), 128, pt_smem(np, ns), s>>>(am, p->wmap[i], B, np, K, 1, p->b[i],
                                                                                relu, ob, of, N, mn, sd, ns);
  };
  layer(0, m0, H, n_in, 1, H1, nullptr, nullptr, nullptr);
  layer(1, m1, H, H, 1, H2, nullptr, nullptr, nullptr);
  layer(2, m2, n_out, H, 0, nullptr, Y, omean, omean + n_out);
  *st = cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
  return true;
}

extern "C" {

leb_status leb_proposer_create(int n_in, int n_hidden, int n_out, unsigned long long seed, leb_proposer* out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 65536 || n_hidden > 65536 || n_out > 65536)
    return LEB_ERR_INVALID_ARG;
  *out = nullptr;
  leb_proposer p = new (std::nothrow) leb_proposer_s();
  if (!p) return LEB_ERR_CUDA;
  p->n_in = n_in;
  p->H = n_hidden;
  p->n_out = n_out;
  const int ins[3] = {n_in, n_hidden, n_hidden}, outs[3] = {n_hidden, n_hidden, n_out};
  bool ok = true;
  for (int i = 0; i < 3 && ok; ++i) {
    const size_t nw = (size_t)ins[i] * outs[i], nb = outs[i];
    for (float** q : {&p->W[i], &p->gW[i], &p->mW[i], &p->vW[i]}) ok = ok && cudaMalloc(q, nw * 4) == cudaSuccess;
    for (float** q : {&p->b[i], &p->gb[i], &p->mb[i], &p->vb[i]}) ok = ok && cudaMalloc(q, nb * 4) == cudaSuccess;
    if (!ok) break;
    ok = cudaMemset(p->mW[i], 0, nw * 4) == cudaSuccess && cudaMemset(p->vW[i], 0, nw * 4) == cudaSuccess &&
         cudaMemset(p->mb[i], 0, nb * 4) == cudaSuccess && cudaMemset(p->vb[i], 0, nb * 4) == cudaSuccess &&
         cudaMemset(p->b[i], 0, nb * 4) == cudaSuccess;
    const float bound = std::sqrt(6.f / (float)ins[i]);
    prop_init_kernel<<<blocks_for((long long)nw), 256>>>((long long)nw, p->W[i], bound, seed * 7919ull + i);
    ok = ok && cudaGetLastError() == cudaSuccess;
  }
  ok = ok && cudaMalloc(&p->norm, (size_t)2 * (n_in + n_out) * 4) == cudaSuccess;
  ok = ok && cudaMalloc(&p->periodic, (size_t)n_in * sizeof(int)) == cudaSuccess &&
       cudaMemset(p->periodic, 0, (size_t)n_in * sizeof(int)) == cudaSuccess;
  if (ok) {
    // identity normalisation until set
    std::vector<float> h(2 * (n_in + n_out), 0.f);
    for (int j = 0; j < n_in; ++j) h[n_in + j] = 1.f;
    for (int j = 0; j < n_out; ++j) h[2 * n_in + n_out + j] = 1.f;
    ok = cudaMemcpy(p->norm, h.data(), h.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (ok) ok = setup_tc(p);
  if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
    leb_proposer_destroy(p);
    return LEB_ERR_CUDA;
  }
  *out = p;
  return LEB_OK;
}

leb_status leb_proposer_destroy(leb_proposer p) {
  if (!p) return LEB_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    for (float* q : {p->W[i], p->gW[i], p->mW[i], p->vW[i], p->b[i], p->gb[i], p->mb[i], p->vb[i]}) cudaFree(q);
  for (int i = 0; i < 3; ++i) cudaFree(p->Wb[i]);
  cudaFree(p->norm);
  cudaFree(p->periodic);
  delete p;
  return LEB_OK;
}

leb_status leb_proposer_set_norm(leb_proposer p, const float* in_mean, const float* in_std, const float* out_mean,
                                 const float* out_std, void* stream) {
  if (!p || !in_mean || !in_std || !out_mean || !out_std) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t a = (size_t)p->n_in * 4, b = (size_t)p->n_out * 4;
  bool ok = cudaMemcpyAsync(p->norm, in_mean, a, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(p->norm + p->n_in, in_std, a, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(p->norm + 2 * p->n_in, out_mean, b, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(p->norm + 2 * p->n_in + p->n_out, out_std, b, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
  return ok ? LEB_OK : LEB_ERR_CUDA;
}

leb_status leb_proposer_fit_norm(leb_proposer p, int B, const float* X, const float* Y, void* stream) {
  if (!p || B < 1 || !X || !Y) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  prop_colstats_kernel<<<(p->n_in + 127) / 128, 128, 0, s>>>(B, p->n_in, X, p->periodic, p->norm, p->norm + p->n_in);
  prop_colstats_kernel<<<(p->n_out + 127) / 128, 128, 0, s>>>(B, p->n_out, Y, nullptr, p->norm + 2 * p->n_in,
                                                              p->norm + 2 * p->n_in + p->n_out);
  prop_std_floor_kernel<<<1, 256, 0, s>>>(p->n_out, p->norm + 2 * p->n_in + p->n_out, 1e-2f);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status leb_proposer_set_periodic(leb_proposer p, const int* mask) {
  if (!p || !mask) return LEB_ERR_INVALID_ARG;
  return cudaMemcpy(p->periodic, mask, (size_t)p->n_in * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess
             ? LEB_OK
             : LEB_ERR_CUDA;
}

leb_status leb_proposer_workspace_size(leb_proposer p, int B_max, size_t* bytes) {
  if (!p || !bytes || B_max < 0) return LEB_ERR_INVALID_ARG;
  *bytes = ws_floats(p, B_max) * sizeof(float);
  return LEB_OK;
}

static leb_status forward_impl(leb_proposer p, int B, const float* X, float* ws, cudaStream_t s) {
  const int n_in = p->n_in, H = p->H, n_out = p->n_out;
  float* Xs = ws;
  float* h0 = Xs + (size_t)B * n_in;
  float* h1 = h0 + (size_t)B * H;
  float* y = h1 + (size_t)B * H;
  prop_standardize_kernel<<<blocks_for((long long)B * n_in), 256, 0, s>>>((long long)B * n_in, n_in, X, p->periodic,
                                                                            p->norm, p->norm + n_in, Xs);
  if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  // h0 = relu(Xs W0^T + b0), h1 = relu(h0 W1^T + b1), y = h1 W2^T + b2   (W_i [out, in])
  if (gemm(s, B, H, n_in, Xs, n_in, 0, p->W[0], n_in, 1, h0, H, p->b[0], nullptr, 2) != cudaSuccess ||
      gemm(s, B, H, H, h0, H, 0, p->W[1], H, 1, h1, H, p->b[1], nullptr, 2) != cudaSuccess ||
      gemm(s, B, n_out, H, h1, H, 0, p->W[2], H, 1, y, n_out, p->b[2], nullptr, 1) != cudaSuccess)
    return LEB_ERR_CUDA;
  return LEB_OK;
}

leb_status leb_proposer_forward(leb_proposer p, int B, const float* X, float* Y, void* workspace, size_t ws_bytes,
                                void* stream) {
  if (!p || B < 0 || (B > 0 && (!X || !Y))) return LEB_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < ws_floats(p, B) * sizeof(float)) return LEB_ERR_WORKSPACE;
  if (B == 0) return LEB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  float* ws = (float*)workspace;
  leb_status st = LEB_OK;
  if (forward_tc(p, B, X, ws, Y, s, &st)) return st;   // Y written by the last GEMM's epilogue
  st = forward_impl(p, B, X, ws, s);
  if (st != LEB_OK) return st;
  const float* y = ws + (size_t)B * (p->n_in + 2 * p->H);
  const long long tot = (long long)B * p->n_out;
  prop_destandardize_kernel<<<blocks_for(tot), 256, 0, s>>>(tot, p->n_out, y, p->norm + 2 * p->n_in,
                                                             p->norm + 2 * p->n_in + p->n_out, Y);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status leb_proposer_train_step(leb_proposer p, int B, const float* X, const float* Ytgt, float lr, float* loss,
                                   void* workspace, size_t ws_bytes, void* stream) {
  if (!p || B < 1 || !X || !Ytgt || !(lr > 0.f)) return LEB_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < ws_floats(p, B) * sizeof(float)) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  float* ws = (float*)workspace;
  leb_status st = forward_impl(p, B, X, ws, s);
  if (st != LEB_OK) return st;
  const int n_in = p->n_in, H = p->H, n_out = p->n_out;
  float* Xs = ws;
  float* h0 = Xs + (size_t)B * n_in;
  float* h1 = h0 + (size_t)B * H;
  float* y = h1 + (size_t)B * H;
  float* dy = y + (size_t)B * n_out;
  float* d1 = dy + (size_t)B * n_out;
  float* d0 = d1 + (size_t)B * H;
  if (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return LEB_ERR_CUDA;
  const long long tot = (long long)B * n_out;
  prop_mse_kernel<<<blocks_for(tot), 256, 0, s>>>(tot, n_out, y, Ytgt, p->norm + 2 * n_in, p->norm + 2 * n_in + n_out,
                                                   dy, loss);
  if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  // layer 2: dW2 = dy^T h1, db2 = sum dy, d1 = (dy W2) o (h1 > 0)
  if (gemm(s, n_out, H, B, dy, n_out, 1, h1, H, 0, p->gW[2], H, nullptr, nullptr, 0) != cudaSuccess) return LEB_ERR_CUDA;
  prop_colsum_kernel<<<(n_out + 255) / 256, 256, 0, s>>>(B, n_out, dy, p->gb[2]);
  if (gemm(s, B, H, n_out, dy, n_out, 0, p->W[2], H, 0, d1, H, nullptr, h1, 3) != cudaSuccess) return LEB_ERR_CUDA;
  // layer 1
  if (gemm(s, H, H, B, d1, H, 1, h0, H, 0, p->gW[1], H, nullptr, nullptr, 0) != cudaSuccess) return LEB_ERR_CUDA;
  prop_colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(B, H, d1, p->gb[1]);
  if (gemm(s, B, H, H, d1, H, 0, p->W[1], H, 0, d0, H, nullptr, h0, 3) != cudaSuccess) return LEB_ERR_CUDA;
  // layer 0
  if (gemm(s, H, n_in, B, d0, H, 1, Xs, n_in, 0, p->gW[0], n_in, nullptr, nullptr, 0) != cudaSuccess) return LEB_ERR_CUDA;
  prop_colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(B, H, d0, p->gb[0]);
  if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  // Adam
  p->step += 1;
  p->w_version += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
  const int ins[3] = {n_in, H, H}, outs[3] = {H, H, n_out};
  for (int i = 0; i < 3; ++i) {
    const long long nw = (long long)ins[i] * outs[i];
    prop_adam_kernel<<<blocks_for(nw), 256, 0, s>>>(nw, p->W[i], p->gW[i], p->mW[i], p->vW[i], lr, b1, b2, 1e-8f, c1, c2);
    prop_adam_kernel<<<blocks_for(outs[i]), 256, 0, s>>>(outs[i], p->b[i], p->gb[i], p->mb[i], p->vb[i], lr, b1, b2,
                                                          1e-8f, c1, c2);
  }
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

static leb_status layer_dims(leb_proposer p, int i, int* in, int* out) {
  if (!p || i < 0 || i > 2) return LEB_ERR_INVALID_ARG;
  const int ins[3] = {p->n_in, p->H, p->H}, outs[3] = {p->H, p->H, p->n_out};
  *in = ins[i];
  *out = outs[i];
  return LEB_OK;
}

leb_status leb_proposer_get_layer(leb_proposer p, int i, float* W, float* b, void* stream) {
  int in, out;
  if (layer_dims(p, i, &in, &out) != LEB_OK || !W || !b) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return (cudaMemcpyAsync(W, p->W[i], (size_t)in * out * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
          cudaMemcpyAsync(b, p->b[i], (size_t)out * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess)
             ? LEB_OK
             : LEB_ERR_CUDA;
}

leb_status leb_proposer_set_layer(leb_proposer p, int i, const float* W, const float* b, void* stream) {
  int in, out;
  if (layer_dims(p, i, &in, &out) != LEB_OK || !W || !b) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  p->w_version += 1;   // the BF16 inference copies are stale
  return (cudaMemcpyAsync(p->W[i], W, (size_t)in * out * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
          cudaMemcpyAsync(p->b[i], b, (size_t)out * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess)
             ? LEB_OK
             : LEB_ERR_CUDA;
}

leb_status leb_proposer_get_grad(leb_proposer p, int i, float* dW, float* db, void* stream) {
  int in, out;
  if (layer_dims(p, i, &in, &out) != LEB_OK || !dW || !db) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return (cudaMemcpyAsync(dW, p->gW[i], (size_t)in * out * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
          cudaMemcpyAsync(db, p->gb[i], (size_t)out * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess)
             ? LEB_OK
             : LEB_ERR_CUDA;
}

// ---- checkpoint / resume ----------------------------------------------------------------------
namespace {
struct StateHeader {
  uint32_t magic;   // 'LEBP'
  int32_t n_in, H, n_out, step;
  int32_t pad[3];
};
constexpr uint32_t kStateMagic = 0x5042454Cu;

// The device arrays of the state in a fixed order, with their sizes in bytes.
std::vector<std::pair<void*, size_t>> state_arrays(leb_proposer p) {
  std::vector<std::pair<void*, size_t>> v;
  const int ins[3] = {p->n_in, p->H, p->H}, outs[3] = {p->H, p->H, p->n_out};
  for (int i = 0; i < 3; ++i) {
    const size_t nw = (size_t)ins[i] * outs[i] * 4, nb = (size_t)outs[i] * 4;
    v.push_back({p->W[i], nw});
    v.push_back({p->b[i], nb});
    v.push_back({p->mW[i], nw});
    v.push_back({p->vW[i], nw});
    v.push_back({p->mb[i], nb});
    v.push_back({p->vb[i], nb});
  }
  v.push_back({p->norm, (size_t)2 * (p->n_in + p->n_out) * 4});
  v.push_back({p->periodic, (size_t)p->n_in * sizeof(int)});
  return v;
}
}  // namespace

leb_status leb_proposer_state_size(leb_proposer p, size_t* bytes) {
  if (!p || !bytes) return LEB_ERR_INVALID_ARG;
  size_t n = sizeof(StateHeader);
  for (const auto& a : state_arrays(p)) n += a.second;
  *bytes = n;
  return LEB_OK;
}

leb_status leb_proposer_save_state(leb_proposer p, void* host_buf, size_t bytes, void* stream) {
  size_t need = 0;
  if (leb_proposer_state_size(p, &need) != LEB_OK || !host_buf || bytes < need) return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StateHeader h{kStateMagic, p->n_in, p->H, p->n_out, p->step, {0, 0, 0}};
  std::memcpy(host_buf, &h, sizeof h);
  char* dst = static_cast<char*>(host_buf) + sizeof h;
  for (const auto& a : state_arrays(p)) {
    if (cudaMemcpyAsync(dst, a.first, a.second, cudaMemcpyDeviceToHost, s) != cudaSuccess) return LEB_ERR_CUDA;
    dst += a.second;
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status leb_proposer_load_state(leb_proposer p, const void* host_buf, size_t bytes, void* stream) {
  size_t need = 0;
  if (leb_proposer_state_size(p, &need) != LEB_OK || !host_buf || bytes < need) return LEB_ERR_INVALID_ARG;
  StateHeader h;
  std::memcpy(&h, host_buf, sizeof h);
  if (h.magic != kStateMagic || h.n_in != p->n_in || h.H != p->H || h.n_out != p->n_out || h.step < 0)
    return LEB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const char* src = static_cast<const char*>(host_buf) + sizeof h;
  for (const auto& a : state_arrays(p)) {
    if (cudaMemcpyAsync(a.first, src, a.second, cudaMemcpyHostToDevice, s) != cudaSuccess) return LEB_ERR_CUDA;
    src += a.second;
  }
  // the host buffer may be released once the call returns: wait for the copies out of it
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEB_ERR_CUDA;
  p->step = h.step;
  p->w_version += 1;   // the BF16 inference copies are stale
  return LEB_OK;
}

}  // extern "C"
