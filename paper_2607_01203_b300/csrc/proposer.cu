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

#include <math_constants.h>

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
  // training on the tensor cores: transposed BF16 copies W_i^T [in, out] of layers 1 and 2 (the B operand
  // of the input gradients d_{i-1} = (d_i W_i) o (h_{i-1} > 0)), refreshed with the copies above
  __nv_bfloat16* WbT[3] = {};
  CUtensorMap wTmap[3];
  // calibration: per-output additive offset of the proposals (leb_proposer_calibrate)
  float* offset = nullptr;
  bool calibrated = false;
  // the training step's operand maps, kept while the workspace and the batch stay the same
  const void* tr_ws = nullptr;
  int tr_B = 0;
  CUtensorMap tr_maps[11];
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

// What the epilogue does with a tile (every pointer optional). Column n is global (n0 + local column),
// row m global. In order: x = acc + bias[n]; ReLU; x = 0 where mask[m, n] <= 0 (the ReLU derivative of a
// stored BF16 activation); x = x std[n] + mean[n] (back to the bounds' units); x += offset[n]. Then
// stores: BF16 outb[m, n] (row stride ldo, rows 16-byte aligned), BF16 outbT[n, m] (stride ldT), FP32
// outf[m, n] (stride ldf, + blockIdx.z zstride: one slice per K part), FP32 outfT[n, m] (stride ldfT).
struct PtEpi {
  const float* bias;
  int relu;
  const __nv_bfloat16* mask;
  int ldm;
  const float* omean;
  const float* ostd;
  const float* offset;
  __nv_bfloat16* outb;
  int ldo;
  __nv_bfloat16* outbT;
  int ldT;
  float* outf;
  int ldf;
  long long zstride;
  float* outfT;
  int ldfT;
};

// kpb: K blocks (of 64) per K part; blockIdx.z takes blocks [z kpb, min(nK, (z + 1) kpb)). kTrain: the
// training instance (masks, transposed and K-part outputs); the inference instance keeps only the bias,
// ReLU, the output's standardisation and offsets and the row-major outputs.
template <bool kTrain>
__global__ void __launch_bounds__(128, 2) prop_tc_gemm_kernel(const __grid_constant__ CUtensorMap amap,
                                                              const __grid_constant__ CUtensorMap wmap, int M, int N,
                                                              int K, int nchunk, int stages, int kpb, const PtEpi e) {
  extern __shared__ uint8_t sraw[];
  // 1024-byte aligned base, as an offset from the shared array (so that every derived pointer keeps the
  // shared address space and its accesses compile to shared-memory instructions)
  uint8_t* base = sraw + ((1024u - (smem_u32(sraw) & 1023u)) & 1023u);
  const int btile = N * 128;                              // N rows x 64 K x 2 bytes (a multiple of 1 KB)
  uint8_t* At = base;                                        // [stages][16 KB]
  uint8_t* Bt = base + stages * kPtATile;                 // [stages][N x 128 B]
  uint64_t* full = reinterpret_cast<uint64_t*>(Bt + stages * btile);
  uint64_t* empty = full + stages;
  uint64_t* acc = empty + stages;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128, nb = N / nchunk;
  const int nKall = (K + 63) / 64;
  const int kb0 = blockIdx.z * kpb, kb1 = min(nKall, kb0 + kpb), nK = kb1 - kb0;   // nK >= 1 by the launch
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
      tma_load_2d(At + s * kPtATile, &amap, (kb0 + kb) * 64, m0, &full[s]);
      for (int c = 0; c < nchunk; ++c)
        tma_load_2d(Bt + s * btile + c * nb * 128, &wmap, (kb0 + kb) * 64, n0 + c * nb, &full[s]);
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
    const int nc = n0 + c0;            // global column of v[0]
    float mk[16];
    if (kTrain && e.mask) {
      const uint4* src = reinterpret_cast<const uint4*>(e.mask + (long long)row * e.ldm + nc);
      const uint4 q0 = src[0], q1 = src[1];
      const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
        mk[2 * j] = f.x;
        mk[2 * j + 1] = f.y;
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float x = ok ? v[j] + (e.bias ? e.bias[nc + j] : 0.f) : __int_as_float(0x7fc00000);
      if (e.relu) x = fmaxf(x, 0.f);
      if (kTrain && e.mask) x = mk[j] > 0.f ? x : 0.f;
      if (e.omean) x = fmaf(x, e.ostd[nc + j], e.omean[nc + j]);   // back to the bounds' units
      if (e.offset) x += e.offset[nc + j];
      v[j] = x;
    }
    if (e.outb) {
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<const uint32_t*>(&h);
      }
      uint4* dst = reinterpret_cast<uint4*>(e.outb + (long long)row * e.ldo + nc);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    if (kTrain && e.outbT) {
#pragma unroll
      for (int j = 0; j < 16; ++j) e.outbT[(long long)(nc + j) * e.ldT + row] = __float2bfloat16_rn(v[j]);
    }
    if (e.outf) {
      float4* dst = reinterpret_cast<float4*>(e.outf + (kTrain ? blockIdx.z * e.zstride : 0) + (long long)row * e.ldf + nc);
#pragma unroll
      for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
    if (kTrain && e.outfT) {
#pragma unroll
      for (int j = 0; j < 16; ++j) e.outfT[(long long)(nc + j) * e.ldfT + row] = v[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, tcols);
}

// W [out, in] FP32 -> WT [in, out] BF16 (the transposed copies of the training path).
__global__ void prop_transpose_bf16_kernel(const float* W, int out, int in, __nv_bfloat16* WT) {
  const long long total = (long long)out * in;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / out, r = e - c * out;   // WT[c][r] = W[r][c]
    WT[e] = __float2bfloat16_rn(W[r * in + c]);
  }
}

// Column sums of G [M, N] (the bias gradients), first pass: block (x, y) sums columns 32 x .. 32 x + 31 over
// the rows of slab y (kColSlab rows; each warp a strided set of them, lane = column, coalesced) into
// part[y][n], the 8 warps' partial sums added in a fixed order. prop_reduce_parts_kernel then sums the
// slabs in order (deterministic).
constexpr int kColSlab = 64;
__global__ void __launch_bounds__(256) prop_colsum_tiled_kernel(int M, int N, const float* G, float* part) {
  __shared__ float acc8[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + lane;
  const int r0 = blockIdx.y * kColSlab, r1 = min(M, r0 + kColSlab);
  float acc = 0.f;
  if (n < N)
    for (int m = r0 + warp; m < r1; m += 8) acc += G[(long long)m * N + n];
  acc8[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && n < N) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += acc8[w][lane];
    part[(long long)blockIdx.y * N + n] = t;
  }
}

// BF16 transpose in [R, C] -> out [C, R] through 32 x 32 shared-memory tiles (coalesced on both sides).
__global__ void __launch_bounds__(256) prop_transpose_act_kernel(int R, int C, const __nv_bfloat16* in,
                                                                 __nv_bfloat16* out) {
  __shared__ __nv_bfloat16 t[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    if (r < R && c < C) t[i][tx] = in[(long long)r * C + c];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + tx;
    if (r < R && c < C) out[(long long)c * R + r] = t[tx][i];
  }
}

// Sum of the K-part slices of a product, in slice order (deterministic): out[m, n] = sum_z P[z][m, n]
// (transposed: out[n, m]).
__global__ void prop_reduce_parts_kernel(int nz, int M, int N, const float* P, long long zstride, float* out,
                                         int transpose) {
  const long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int z = 0; z < nz; ++z) acc += P[z * zstride + e];
    if (transpose) {
      const long long m = e / N, n = e - m * N;
      out[n * M + m] = acc;
    } else {
      out[e] = acc;
    }
  }
}

// dy = 2 (y - t) / (B n) as in prop_mse_kernel, also rounded to BF16; the loss summed per block first
// (one atomic per block). B n < 2^31.
__global__ void __launch_bounds__(256) prop_mse_bf16_kernel(int B, int n, const float* y, const float* Y,
                                                            const float* mean, const float* stdv, float* dy,
                                                            __nv_bfloat16* dyb, float* loss) {
  __shared__ float red[8];
  float part = 0.f;
  const int total = B * n;
  const float scale = 2.f / (float)total;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int j = e % n;
    const float tgt = (Y[e] - mean[j]) / stdv[j];
    const float d = y[e] - tgt;
    const float g = scale * d;
    dy[e] = g;
    dyb[e] = __float2bfloat16_rn(g);
    part = fmaf(d, d, part);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(loss, t / (float)total);
  }
}

// Adam on several parameter arrays in one launch (segment i: n[i] entries of p, g, m, v).
struct AdamSegs {
  float* p[6];
  const float* g[6];
  float* m[6];
  float* v[6];
  long long start[7];
};
__global__ void prop_adam_multi_kernel(AdamSegs a, int nseg, float lr, float b1, float b2, float eps, float c1,
                                       float c2) {
  const long long total = a.start[nseg];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int i = 0;
    while (i + 1 < nseg && e >= a.start[i + 1]) ++i;
    const long long k = e - a.start[i];
    const float gg = a.g[i][k];
    const float mm = b1 * a.m[i][k] + (1.f - b1) * gg;
    const float vv = b2 * a.v[i][k] + (1.f - b2) * gg * gg;
    a.m[i][k] = mm;
    a.v[i][k] = vv;
    a.p[i][k] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

constexpr int kCalMax = 16384;   // calibration samples per call (sorted in shared memory)

// Calibration margin of one output per CTA: the residuals by which the proposals are narrower than the
// certified bounds (lower outputs j < n_lower: proposal - certified; upper: certified - proposal) are
// sorted in shared memory (bitonic, padded with +inf to a power of two); the margin is the k-th smallest,
// k = ceil(q (B + 1)) - 1 clamped to [0, B - 1] (the split-conformal quantile), floored at 0; the signed
// offset (-margin for lower outputs, +margin for upper) is written.
__global__ void prop_calibrate_kernel(int B, int n, int n_lower, float q, const float* P, const float* Y, float* offset) {
  extern __shared__ float sv[];
  const int j = blockIdx.x;
  int L = 1;
  while (L < B) L <<= 1;
  for (int b = threadIdx.x; b < L; b += blockDim.x) {
    float r = CUDART_INF_F;
    if (b < B) {
      const float pv = P[(long long)b * n + j], cv = Y[(long long)b * n + j];
      r = j < n_lower ? pv - cv : cv - pv;
      if (r != r) r = CUDART_INF_F;   // a NaN proposal counts as uncovered
    }
    sv[b] = r;
  }
  __syncthreads();
  for (int k = 2; k <= L; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const float a = sv[i], c = sv[ixj];
          if ((a > c) == up) {
            sv[i] = c;
            sv[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    int k = (int)ceilf(q * (float)(B + 1)) - 1;
    k = k < 0 ? 0 : (k > B - 1 ? B - 1 : k);
    const float m = fmaxf(sv[k], 0.f);
    offset[j] = j < n_lower ? -m : m;
  }
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
                                          const float* offset, float* Y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n);
    Y[e] = fmaf(y[e], stdv[j], mean[j]) + (offset ? offset[j] : 0.f);
  }
}

// Standardised inputs straight into the BF16 operand of the first layer: a thread per column pair (n
// even) keeps that pair's angle flags, means and deviations in registers and walks kStdRows rows, whose
// loads are independent; a row's pairs are consecutive threads (coalesced).
constexpr int kStdRows = 16;
// XbT (optional): the same values transposed, [n, B] (the training path's operand of the first layer's
// weight gradient).
__global__ void prop_standardize_bf16_kernel(int B, int n, const float* X, const int* periodic, const float* mean,
                                             const float* stdv, __nv_bfloat16* Xb, __nv_bfloat16* XbT) {
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
      const __nv_bfloat162 v = __floats2bfloat162_rn((x.x - m0) / s0, (x.y - m1) / s1);
      reinterpret_cast<__nv_bfloat162*>(Xb + (long long)row * n)[c] = v;
      if (XbT) {
        XbT[(long long)j * B + row] = v.x;
        XbT[(long long)(j + 1) * B + row] = v.y;
      }
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

// Layout of the tensor-core training step's workspace (byte offsets, 16-byte aligned): the standardised
// inputs and the activations in BF16, row-major and transposed (the transposed copies are the K-major
// operands of the weight gradients, whose K is the batch), the FP32 outputs and input gradients (for the
// loss and the bias gradients), and the K-part slices of the weight gradients.
struct TrainLayout {
  size_t Xb, XbT, h0b, h0T, h1b, h1T, y, dy, dyb, dyT, d1, d1b, d1T, d0, d0T, part, total;
  int kpb[3], nz[3];   // weight gradient of layer i: K blocks per part, parts
};

static TrainLayout train_layout(const leb_proposer_s* p, int B) {
  TrainLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
  const size_t b = (size_t)B, n_in = p->n_in, H = p->H, n_out = p->n_out;
  L.Xb = take(2 * b * n_in);
  L.XbT = take(2 * b * n_in);
  L.h0b = take(2 * b * H);
  L.h0T = take(2 * b * H);
  L.h1b = take(2 * b * H);
  L.h1T = take(2 * b * H);
  L.y = take(4 * b * n_out);
  L.dy = take(4 * b * n_out);
  L.dyb = take(2 * b * n_out);
  L.dyT = take(2 * b * n_out);
  L.d1 = take(4 * b * H);
  L.d1b = take(2 * b * H);
  L.d1T = take(2 * b * H);
  L.d0 = take(4 * b * H);
  L.d0T = take(2 * b * H);
  // weight gradient of layer i as C[M_i, H] (layer 0 transposed: dW0^T [n_in, H]), K = B split in parts so
  // that the grid fills the SMs
  const int Ms[3] = {p->n_in, p->H, p->n_out};
  const int parts = p->parts[0] > 0 ? p->parts[0] : 1;
  const int kblocks = (B + 63) / 64;
  size_t part = 0;
  for (int i = 0; i < 3; ++i) {
    const int mt = (Ms[i] + 127) / 128;
    const int target = std::max(1, 148 / (mt * parts));
    L.kpb[i] = (kblocks + target - 1) / target;
    L.nz[i] = (kblocks + L.kpb[i] - 1) / L.kpb[i];
    part = std::max(part, (size_t)L.nz[i] * Ms[i] * H * 4);
  }
  part = std::max(part, (size_t)((B + kColSlab - 1) / kColSlab) * std::max(H, n_out) * 4);   // column-sum slabs
  L.part = take(part);
  L.total = o;
  return L;
}

// workspace (floats): the CUDA-core path's Xs [B, n_in], h0 [B, H], h1 [B, H], y [B, n_out], dy [B, n_out],
// d1 [B, H], d0 [B, H], or the tensor-core training layout, whichever is larger; then [B, n_out] for the
// proposals of a calibration call
size_t ws_base_floats(const leb_proposer_s* p, int B) {
  const size_t core = (size_t)B * (p->n_in + 4 * p->H + 2 * p->n_out) + 64;
  const size_t tc = train_layout(p, B).total / 4 + 64;
  return (std::max(core, tc) + 63) & ~size_t(63);
}
size_t ws_floats(const leb_proposer_s* p, int B) { return ws_base_floats(p, B) + (size_t)B * p->n_out; }

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
  // transposed copies of layers 1 and 2 for the training path's input gradients: W_i^T [in_i, out_i] as
  // the B operand (N = in_i = H rows, K = out_i)
  for (int i = 1; i < 3; ++i) {
    if (cudaMalloc(&p->WbT[i], (size_t)ins[i] * outs[i] * 2) != cudaSuccess) return false;
    cuuint64_t dims[2] = {(cuuint64_t)outs[i], (cuuint64_t)ins[i]};
    cuuint64_t strides[1] = {(cuuint64_t)outs[i] * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)(ins[i] / p->parts[0])};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&p->wTmap[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p->WbT[i], dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return true;
  }
  if (cudaFuncSetAttribute(prop_tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPtSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(prop_tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPtSmem) != cudaSuccess)
    return true;
  p->tc = true;
  return true;
}

// A BF16 matrix [rows, cols] (cols = K, contiguous) as an operand of the tcgen05 GEMM: box 64 x box_rows
// (128 for the A operand; a column part's width for the B operand), zero fill past the edges.
static bool act_map(CUtensorMap* m, const __nv_bfloat16* x, int rows, int cols, int box_rows = 128) {
  auto enc = tensor_map_encoder();
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc && enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(x), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Refresh the BF16 weight copies (and the transposed ones) after the weights changed.
static void refresh_bf16(leb_proposer p, cudaStream_t s) {
  if (p->wb_version == p->w_version) return;
  const int n_in = p->n_in, H = p->H, n_out = p->n_out;
  const long long n0 = (long long)n_in * H, n1 = (long long)H * H, n2 = (long long)H * n_out;
  prop_weights_bf16_kernel<<<blocks_for(n0 + n1 + n2), 256, 0, s>>>(p->W[0], n0, p->W[1], n1, p->W[2], n2, p->Wb[0],
                                                                      p->Wb[1], p->Wb[2]);
  prop_transpose_bf16_kernel<<<blocks_for(n1), 256, 0, s>>>(p->W[1], H, H, p->WbT[1]);
  prop_transpose_bf16_kernel<<<blocks_for(n2), 256, 0, s>>>(p->W[2], n_out, H, p->WbT[2]);
  p->wb_version = p->w_version;
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
  refresh_bf16(p, s);   // after a weight change
  const int sthreads = std::min(1024, ((n_in / 2) + 31) / 32 * 32);
  prop_standardize_bf16_kernel<<<(B + kStdRows - 1) / kStdRows, sthreads, 0, s>>>(B, n_in, X, p->periodic, p->norm,
                                                                                 p->norm + n_in, Xb, nullptr);
  const int tiles = (B + 127) / 128;
  const float* omean = p->norm + 2 * n_in;
  // layer i: a CTA per (128-row tile, column part of N / parts columns)
  auto layer = [&](int i, const CUtensorMap& am, int N, int K, int relu, __nv_bfloat16* ob, float* of,
                   const float* mn, const float* sd, const float* off) {
    PtEpi e{};
    e.bias = p->b[i];
    e.relu = relu;
    e.omean = mn;
    e.ostd = sd;
    e.offset = off;
    e.outb = ob;
    e.ldo = N;
    e.outf = of;
    e.ldf = N;
    const int np = N / p->parts[i], ns = pt_stages(np);
    prop_tc_gemm_kernel<false><<<dim3(tiles, p->parts[i]), 128, pt_smem(np, ns), s>>>(am, p->wmap[i], B, np, K, 1, ns,
                                                                                (K + 63) / 64, e);
  };
  layer(0, m0, H, n_in, 1, H1, nullptr, nullptr, nullptr, nullptr);
  layer(1, m1, H, H, 1, H2, nullptr, nullptr, nullptr, nullptr);
  layer(2, m2, n_out, H, 0, nullptr, Y, omean, omean + n_out, p->calibrated ? p->offset : nullptr);
  *st = cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
  return true;
}

// One training step on the tensor cores (the GEMMs of prop_tc_gemm_kernel; elementwise work in the small
// kernels above), the same arithmetic as the CUDA-core step: BF16 operands, FP32 accumulation.
//   forward: h0 = relu(Xs W0^T + b0), h1 = relu(h0 W1^T + b1), y = h1 W2^T + b2 (standardised units)
//   dy = 2 (y - t) / (B n_out);  dW2 = dy^T h1, d1 = (dy W2) o (h1 > 0);  dW1 = d1^T h0,
//   d0 = (d1 W1) o (h0 > 0);  dW0 = d0^T Xs (computed as dW0^T = Xs^T d0: 392 columns do not split into
//   parts of a multiple of 16);  db_i = column sums;  then Adam on the FP32 master weights.
// The weight gradients contract over the batch: their operands are the transposed BF16 copies the
// producing kernels write, and K is split in parts whose FP32 slices are summed in order afterwards
// (deterministic). Taken when the shapes fit the tcgen05 GEMM and B is a multiple of 8 (TMA strides);
// false: not taken (the CUDA-core step runs).
static bool train_tc(leb_proposer p, int B, const float* X, const float* Yt, float* loss, void* wsv, cudaStream_t s,
                     leb_status* st) {
  if (!p->tc || B % 8 != 0 || (reinterpret_cast<uintptr_t>(wsv) & 255u) || (reinterpret_cast<uintptr_t>(X) & 7u))
    return false;
  const int n_in = p->n_in, H = p->H, n_out = p->n_out;
  const TrainLayout L = train_layout(p, B);
  char* ws = static_cast<char*>(wsv);
  auto bf = [&](size_t o) { return reinterpret_cast<__nv_bfloat16*>(ws + o); };
  auto fp = [&](size_t o) { return reinterpret_cast<float*>(ws + o); };
  CUtensorMap* tm = p->tr_maps;
  CUtensorMap &mXb = tm[0], &mXbT = tm[1], &mh0b = tm[2], &mh0T = tm[3], &mh1b = tm[4], &mh1T = tm[5], &mdyb = tm[6],
              &mdyT = tm[7], &md1b = tm[8], &md1T = tm[9], &md0T = tm[10];
  if (p->tr_ws != wsv || p->tr_B != B) {
    const int np = H / p->parts[0];   // column part of an H-wide product
    p->tr_ws = nullptr;
    const bool ok = act_map(&mXb, bf(L.Xb), B, n_in) && act_map(&mh0b, bf(L.h0b), B, H) &&
                    act_map(&mh1b, bf(L.h1b), B, H) && act_map(&mdyb, bf(L.dyb), B, n_out) &&
                    act_map(&md1b, bf(L.d1b), B, H) && act_map(&mdyT, bf(L.dyT), n_out, B) &&
                    act_map(&md1T, bf(L.d1T), H, B) && act_map(&mXbT, bf(L.XbT), n_in, B) &&
                    act_map(&mh1T, bf(L.h1T), H, B, np) && act_map(&mh0T, bf(L.h0T), H, B, np) &&
                    act_map(&md0T, bf(L.d0T), H, B, np);
    if (!ok) return false;
    p->tr_ws = wsv;
    p->tr_B = B;
  }
  *st = LEB_ERR_CUDA;
  refresh_bf16(p, s);
  const int sthreads = std::min(1024, ((n_in / 2) + 31) / 32 * 32);
  prop_standardize_bf16_kernel<<<(B + kStdRows - 1) / kStdRows, sthreads, 0, s>>>(B, n_in, X, p->periodic, p->norm,
                                                                                 p->norm + n_in, bf(L.Xb), nullptr);
  auto transpose = [&](const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out) {
    prop_transpose_act_kernel<<<dim3((C + 31) / 32, (R + 31) / 32), 256, 0, s>>>(R, C, in, out);
  };
  auto colsum = [&](int M, int N, const float* G, float* out) {   // slabs into the part slices, then in order
    const int slabs = (M + kColSlab - 1) / kColSlab;
    prop_colsum_tiled_kernel<<<dim3((N + 31) / 32, slabs), 256, 0, s>>>(M, N, G, fp(L.part));
    prop_reduce_parts_kernel<<<blocks_for(N), 256, 0, s>>>(slabs, 1, N, fp(L.part), N, out, 0);
  };
  transpose(bf(L.Xb), B, n_in, bf(L.XbT));
  const int tiles = (B + 127) / 128;
  // C[M, N] on a grid of (128-row tiles, column parts, K parts)
  auto gemm_tc = [&](const CUtensorMap& am, const CUtensorMap& bm, int M, int N, int parts, int K, int kpb, int nz,
                     const PtEpi& e) {
    const int n = N / parts, ns = pt_stages(n);
    prop_tc_gemm_kernel<true><<<dim3((M + 127) / 128, parts, nz), 128, pt_smem(n, ns), s>>>(am, bm, M, n, K, 1, ns, kpb,
                                                                                             e);
  };
  const int kall = (H + 63) / 64;
  {   // forward
    PtEpi e{};
    e.bias = p->b[0];
    e.relu = 1;
    e.outb = bf(L.h0b);
    e.ldo = H;
    e.outbT = bf(L.h0T);
    e.ldT = B;
    gemm_tc(mXb, p->wmap[0], B, H, p->parts[0], n_in, (n_in + 63) / 64, 1, e);
    e.bias = p->b[1];
    e.outb = bf(L.h1b);
    e.outbT = bf(L.h1T);
    gemm_tc(mh0b, p->wmap[1], B, H, p->parts[1], H, kall, 1, e);
    PtEpi f{};
    f.bias = p->b[2];
    f.outf = fp(L.y);
    f.ldf = n_out;
    gemm_tc(mh1b, p->wmap[2], B, n_out, p->parts[2], H, kall, 1, f);
  }
  if (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return true;
  const long long tot = (long long)B * n_out;
  prop_mse_bf16_kernel<<<blocks_for(tot), 256, 0, s>>>(B, n_out, fp(L.y), Yt, p->norm + 2 * n_in,
                                                        p->norm + 2 * n_in + n_out, fp(L.dy), bf(L.dyb), loss);
  transpose(bf(L.dyb), B, n_out, bf(L.dyT));
  colsum(B, n_out, fp(L.dy), p->gb[2]);
  // weight gradient C[M, H] (K = B in nz parts) into the slices, then summed in order
  auto wgrad = [&](int i, const CUtensorMap& am, const CUtensorMap& bm, int M, int transpose) {
    PtEpi e{};
    e.outf = fp(L.part);
    e.ldf = H;
    e.zstride = (long long)M * H;
    gemm_tc(am, bm, M, H, p->parts[0], B, L.kpb[i], L.nz[i], e);
    prop_reduce_parts_kernel<<<blocks_for((long long)M * H), 256, 0, s>>>(L.nz[i], M, H, fp(L.part), (long long)M * H,
                                                                           p->gW[i], transpose);
  };
  wgrad(2, mdyT, mh1T, n_out, 0);
  {   // d1 = (dy W2) o (h1 > 0)
    PtEpi e{};
    e.mask = bf(L.h1b);
    e.ldm = H;
    e.outf = fp(L.d1);
    e.ldf = H;
    e.outb = bf(L.d1b);
    e.ldo = H;
    e.outbT = bf(L.d1T);
    e.ldT = B;
    gemm_tc(mdyb, p->wTmap[2], B, H, p->parts[0], n_out, (n_out + 63) / 64, 1, e);
  }
  colsum(B, H, fp(L.d1), p->gb[1]);
  wgrad(1, md1T, mh0T, H, 0);
  {   // d0 = (d1 W1) o (h0 > 0)
    PtEpi e{};
    e.mask = bf(L.h0b);
    e.ldm = H;
    e.outf = fp(L.d0);
    e.ldf = H;
    e.outbT = bf(L.d0T);
    e.ldT = B;
    gemm_tc(md1b, p->wTmap[1], B, H, p->parts[0], H, kall, 1, e);
  }
  colsum(B, H, fp(L.d0), p->gb[0]);
  wgrad(0, mXbT, md0T, n_in, 1);   // dW0^T [n_in, H] -> gW[0] [H, n_in]
  *st = cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
  return true;
}

// Adam on every weight and bias from the gradients of the step just computed (one launch; the same
// per-element arithmetic as prop_adam_kernel).
static leb_status adam_all(leb_proposer p, float lr, cudaStream_t s) {
  p->step += 1;
  p->w_version += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
  const int ins[3] = {p->n_in, p->H, p->H}, outs[3] = {p->H, p->H, p->n_out};
  AdamSegs a{};
  long long o = 0;
  for (int i = 0; i < 3; ++i) {
    a.p[2 * i] = p->W[i];
    a.g[2 * i] = p->gW[i];
    a.m[2 * i] = p->mW[i];
    a.v[2 * i] = p->vW[i];
    a.start[2 * i] = o;
    o += (long long)ins[i] * outs[i];
    a.p[2 * i + 1] = p->b[i];
    a.g[2 * i + 1] = p->gb[i];
    a.m[2 * i + 1] = p->mb[i];
    a.v[2 * i + 1] = p->vb[i];
    a.start[2 * i + 1] = o;
    o += outs[i];
  }
  a.start[6] = o;
  prop_adam_multi_kernel<<<blocks_for(o), 256, 0, s>>>(a, 6, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
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
  ok = ok && cudaMalloc(&p->offset, (size_t)n_out * 4) == cudaSuccess &&
       cudaMemset(p->offset, 0, (size_t)n_out * 4) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(prop_calibrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kCalMax * (int)sizeof(float)) == cudaSuccess;
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
  for (int i = 0; i < 3; ++i) {
    cudaFree(p->Wb[i]);
    cudaFree(p->WbT[i]);
  }
  cudaFree(p->offset);
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
                                                             p->norm + 2 * p->n_in + p->n_out,
                                                             p->calibrated ? p->offset : nullptr, Y);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status leb_proposer_train_step(leb_proposer p, int B, const float* X, const float* Ytgt, float lr, float* loss,
                                   void* workspace, size_t ws_bytes, void* stream) {
  if (!p || B < 1 || !X || !Ytgt || !(lr > 0.f)) return LEB_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < ws_floats(p, B) * sizeof(float)) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  float* ws = (float*)workspace;
  const int n_in = p->n_in, H = p->H, n_out = p->n_out;
  leb_status st = LEB_OK;
  if (train_tc(p, B, X, Ytgt, loss, workspace, s, &st)) {
    if (st != LEB_OK) return st;
    return adam_all(p, lr, s);
  }
  st = forward_impl(p, B, X, ws, s);
  if (st != LEB_OK) return st;
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
  return adam_all(p, lr, s);
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
  v.push_back({p->offset, (size_t)p->n_out * 4});
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
  StateHeader h{kStateMagic, p->n_in, p->H, p->n_out, p->step, {p->calibrated ? 1 : 0, 0, 0}};
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
  p->calibrated = h.pad[0] != 0;
  p->w_version += 1;   // the BF16 inference copies are stale
  return LEB_OK;
}

leb_status leb_proposer_calibrate(leb_proposer p, int B, const float* X, const float* Y, int n_lower, float q,
                                  void* workspace, size_t ws_bytes, void* stream) {
  if (!p || B < 1 || B > kCalMax || !X || !Y || n_lower < 0 || n_lower > p->n_out || !(q > 0.f && q < 1.f))
    return LEB_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < ws_floats(p, B) * sizeof(float)) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  float* P = static_cast<float*>(workspace) + ws_base_floats(p, B);
  p->calibrated = false;   // the residuals are those of the uncalibrated proposals
  const leb_status st = leb_proposer_forward(p, B, X, P, workspace, ws_bytes, stream);
  if (st != LEB_OK) return st;
  int L = 1;
  while (L < B) L <<= 1;
  prop_calibrate_kernel<<<p->n_out, 1024, (size_t)L * sizeof(float), s>>>(B, p->n_out, n_lower, q, P, Y, p->offset);
  if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  p->calibrated = true;
  return LEB_OK;
}

leb_status leb_proposer_get_offset(leb_proposer p, float* offset, int* calibrated, void* stream) {
  if (!p || !offset || !calibrated) return LEB_ERR_INVALID_ARG;
  *calibrated = p->calibrated ? 1 : 0;
  return cudaMemcpyAsync(offset, p->offset, (size_t)p->n_out * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) ==
                 cudaSuccess
             ? LEB_OK
             : LEB_ERR_CUDA;
}

}  // extern "C"
