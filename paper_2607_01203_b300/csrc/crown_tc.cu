// CROWN back-substitution chains (Thm. 2) on the 5th-generation tensor cores (tcgen05), with the
// Jacobian correction (Thm. 3) in the epilogue.
//
// One CTA per SM owns a tile of 128 rows of one timestep (126 for the output: 42 state rows x {lower,
// upper, Jacobian} so that the three rows of a state dimension share a tile) and carries it through
// every back-substitution stage on chip:
//   A_k = Lambda o s_k (sign-selected slopes, FP16 or BF16, 128 x K in shared memory, 128-byte swizzle)
//   Lambda' = A_k W_k  (tcgen05.mma, FP32 accumulators in TMEM: 128 lanes x N <= 512 columns)
// Warp roles: warp 0 streams W_k^T tiles with TMA (ring of NSB stages), warp 1 allocates TMEM and one of
// its threads issues the MMAs, warps 2..9 run the epilogue (two warps per TMEM lane quarter, each on one
// half of the columns): they read Lambda' out of TMEM, apply the next layer's selected slopes, accumulate
// the offsets beta and the rounding inflation, and write the next A operand; after the last stage they
// concretise over the displacement box.
//
// Rigour of the reduced-precision GEMM (per stage, per row): with A~ the rounded operand, W~ the rounded
// weights and the FP32 accumulation error bounded by gamma_K |A~| |W~| (u = 2^-23, i.e. without assuming
// round-to-nearest accumulation), the computed Lambda' differs from the exact (Lambda o s) W_k by at most
//   gamma_K |A~| |W~| + |A~ - Lambda o s| |W~| + |Lambda o s| |W~ - W|,
// and its effect on Lambda' dh_{k-1} is bounded with the per-neuron vectors v1 = |W| abar and
// v2 = |W - W~| abar (|W~| <= |W| (1 + 2^-10)); the sum is subtracted from (added to) the bound.
#include <cmath>
#include <cstdio>

#include "internal.h"
#include "interval.cuh"
#include "mlp_math.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace leb {

constexpr int kTcEpiWarps = 16;                 // 4 per TMEM lane quarter, 16-column chunks round-robin
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);
constexpr int kTcNSB = 2;                       // B ring stages
constexpr int kTcBStage = 256 * 128;            // 256 rows x 64 K x 2 bytes
constexpr int kTcARegion = 128 * 512 * 2;       // 128 rows x 512 K x 2 bytes
constexpr int kTcVec = 512 * 24;                // per-neuron vectors of one stage: float4 + float2
constexpr int kTcStat = 128 * 4 * 4 * 4;        // [row][column quarter][4]
constexpr int kTcSmem = 1024 + kTcARegion + kTcNSB * kTcBStage + 2 * kTcVec + kTcStat + 256;
static_assert(kTcSmem <= 227 * 1024, "tensor-core chain shared memory");

struct TcArgs {
  CUtensorMap tmap[kMaxLayers];  // W_k^T in FP16/BF16: [widths[k] rows, widths[k+1] cols], box {64, Nbox}
  int L;
  int widths[kMaxLayers + 1];
  int residual;
  int fmt;                       // 0 FP16, 1 BF16
  int T, target, nroles, rows_total, rows_per_tile, tiles_per_t;
  int H;
  int hoff[kMaxLayers];
  const float* W_target;
  const float *zhat, *zrad, *sL, *tL, *sU, *tU, *D, *winf, *ucon, *dlo, *dhi;
  const int* bad;
  float *lo, *hi, *bslack;
  float *r_lo, *r_hi, *A, *B, *eps, *gamma_c, *gamma_r;
  float gamma_pad;
  int tight;                     // 1: no rounding inflation (the adjoint's recompute; not a sound bound)
  int* flags;
};

// Store 16 operand values (row r, columns j0..j0+15, packed pairs) into the 128-byte-swizzled K-major tile.
__device__ __forceinline__ void store_a16(uint8_t* A, int r, int j0, const uint32_t packed[8]) {
  const int kb = j0 >> 6;                 // K block of 64 columns (16 KB each)
  const int c = (j0 & 63) >> 3;           // first 16-byte chunk inside the 128-byte row
  uint8_t* rowp = A + kb * 16384 + r * 128;
  const int sw = r & 7;
  *reinterpret_cast<uint4*>(rowp + ((c ^ sw) << 4)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  *reinterpret_cast<uint4*>(rowp + (((c + 1) ^ sw) << 4)) = make_uint4(packed[4], packed[5], packed[6], packed[7]);
}

__device__ __forceinline__ uint32_t pack2(float x, float y, int fmt) {
  if (fmt == 0) {
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Row pass over 16 columns (row role: 0 lower, 1 upper, 2 Jacobian). sv[j] = {sL, sU, tauL, tauU},
// sw[j] = {inflation weight of neuron j, sigma'(z^_j)} of the hidden layer Lambda acts on.
__device__ __forceinline__ void row_pass16(int role, int j0, const float lam[16], const float4* sv, const float2* sw,
                                           int fmt, uint32_t packed[8], float& beta0, float& beta1, float& infl0,
                                           float& infl1) {
  float av[16];
  if (role == 2) {
#pragma unroll
    for (int e = 0; e < 16; ++e) av[e] = lam[e] * sw[j0 + e].y;
  } else {
    const bool lower = role == 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float4 v = sv[j0 + e];
      const float w = sw[j0 + e].x;
      const float l = lam[e];
      const bool use_lower = lower == (l >= 0.f);
      const float s = use_lower ? v.x : v.y;
      const float tau = use_lower ? v.z : v.w;
      av[e] = l * s;
      if (e & 1) {
        beta1 = lower ? __fmaf_rd(l, tau, beta1) : __fmaf_ru(l, tau, beta1);
        infl1 = __fmaf_ru(fabsf(av[e]), w, infl1);
      } else {
        beta0 = lower ? __fmaf_rd(l, tau, beta0) : __fmaf_ru(l, tau, beta0);
        infl0 = __fmaf_ru(fabsf(av[e]), w, infl0);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) packed[e] = pack2(av[2 * e], av[2 * e + 1], fmt);
}

__global__ void __launch_bounds__(kTcThreads, 1) crown_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ uint8_t sraw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sraw) + 1023) & ~uintptr_t(1023));
  uint8_t* Asm = base;                                     // A operand (and the J-row buffer at the end)
  uint8_t* Bsm = base + kTcARegion;                        // B ring
  uint8_t* Vsm = Bsm + kTcNSB * kTcBStage;                 // 2 x per-neuron vectors (double buffered)
  float* stat = reinterpret_cast<float*>(Vsm + 2 * kTcVec);  // [128][4][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(stat) + kTcStat);
  uint64_t* b_full = bars;                 // [kTcNSB]
  uint64_t* b_empty = bars + kTcNSB;       // [kTcNSB]
  uint64_t* a_full = bars + 2 * kTcNSB;    // operand written by the epilogue
  uint64_t* acc_full = a_full + 1;         // accumulator complete
  uint64_t* drain = acc_full + 1;
  uint64_t* ebar = drain + 1;              // epilogue-warps barrier (bounded waits)
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = a.T * a.tiles_per_t;
  const int target = a.target;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcNSB; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(a_full, kTcEpiWarps);
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
    mbar_init(ebar, kTcEpiWarps);
    mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 1) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      for (int k = 0; k < target; ++k) tma_prefetch_desc(&a.tmap[k]);
      uint32_t kb = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        for (int k = target - 1; k >= 0 && ok; --k) {
          const int K = a.widths[k + 1], N = a.widths[k];
          const int nh = N > 256 ? 2 : 1, nbox = N / nh;
          const int nkc = (K + 63) / 64;
          for (int kc = 0; kc < nkc && ok; ++kc)
            for (int h = 0; h < nh; ++h, ++kb) {
              const int s = (int)(kb % kTcNSB);
              if (kb >= (uint32_t)kTcNSB && !mbar_wait(&b_empty[s], ((kb / kTcNSB) - 1) & 1u)) { ok = false; break; }
              if (*(volatile int*)&s_abort) { ok = false; break; }
              mbar_arrive_expect_tx(&b_full[s], (uint32_t)nbox * 128u);
              tma_load_2d(Bsm + (size_t)s * kTcBStage, &a.tmap[k], kc * 64, h * nbox, &b_full[s]);
            }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      // every issued load must land before the block exits
      for (uint32_t j = (kb > (uint32_t)kTcNSB ? kb - kTcNSB : 0u); j < kb; ++j)
        mbar_wait(&b_full[j % kTcNSB], (j / kTcNSB) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t a_base = smem_u32(Asm), b_base = smem_u32(Bsm);
      uint32_t kb = 0, na = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        for (int k = target - 1; k >= 0 && ok; --k) {
          const int K = a.widths[k + 1], N = a.widths[k];
          const int nh = N > 256 ? 2 : 1, nbox = N / nh;
          const int nkc = (K + 63) / 64;
          const uint32_t idesc = idesc_f16(128, nbox, a.fmt);
          if (!mbar_wait(a_full, na & 1u)) { ok = false; break; }
          ++na;
          tc_fence_after();
          for (int kc = 0; kc < nkc && ok; ++kc)
            for (int h = 0; h < nh; ++h, ++kb) {
              const int s = (int)(kb % kTcNSB);
              if (!mbar_wait(&b_full[s], (kb / kTcNSB) & 1u)) { ok = false; break; }
              tc_fence_after();
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = sw128_desc(a_base + kc * 16384 + kk * 32);
                const uint64_t bd = sw128_desc(b_base + s * kTcBStage + kk * 32);
                tc_mma_f16(tmem + (uint32_t)(h * nbox), ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
              }
              tc_commit(&b_empty[s]);
            }
          tc_commit(acc_full);
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      tc_commit(drain);             // completes once every MMA issued above has finished
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue warps
    const int ew = warp - 2;
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int cq = ew >> 2;                 // 16-column chunks cq, cq + 4, ...
    const int r = q * 32 + lane;            // tile row = TMEM lane
    const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16);
    const int ethr = kTcEpiWarps * 32, etid = threadIdx.x - 64;
    uint32_t nacc = 0, nbar = 0;
    int vbuf = 0;
    bool ok = true;
    // all epilogue warps meet here; false if the wait ran out (then every later step is skipped)
    auto epi_sync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) mbar_arrive(ebar);
      const bool res = mbar_wait(ebar, nbar & 1u);
      ++nbar;
      return res;
    };
    // stage the per-neuron vectors of hidden layer hl of timestep t (or, hl < 0, the box) into buffer b
    auto stage_vectors = [&](int t, int hl, int b) {
      float4* sv = reinterpret_cast<float4*>(Vsm + b * kTcVec);
      float2* sw = reinterpret_cast<float2*>(Vsm + b * kTcVec + 512 * 16);
      if (hl >= 0) {
        const int width = a.widths[hl + 1], wp = (width + 63) & ~63;
        const long long o = (long long)t * a.H + a.hoff[hl];
        for (int j = etid; j < wp; j += ethr) {
          if (j < width) {
            sv[j] = make_float4(a.sL[o + j], a.sU[o + j], a.tL[o + j], a.tU[o + j]);
            sw[j] = make_float2(a.winf[o + j], a.D[o + j]);
          } else {
            sv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            sw[j] = make_float2(0.f, 0.f);
          }
        }
      } else {
        const int n = a.widths[0];
        const long long o = (long long)t * n;
        for (int j = etid; j < n; j += ethr) sw[j] = make_float2(a.dlo[o + j], a.dhi[o + j]);
      }
    };

    for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      const int t = item / a.tiles_per_t, tile = item - t * a.tiles_per_t;
      const int grow = tile * a.rows_per_tile + r;
      const bool valid = r < a.rows_per_tile && grow < a.rows_total;
      const int role = valid ? grow % a.nroles : 0;
      const int idx = valid ? grow / a.nroles : 0;
      float beta0 = 0.f, beta1 = 0.f, infl0 = 0.f, infl1 = 0.f, ucon = 0.f;

      // ---- prologue: A for the stage that multiplies by W_{target-1}: W_target rows o slopes -------
      {
        const int K = a.widths[target], Kp = (K + 63) & ~63;
        stage_vectors(t, target - 1, vbuf);
        if (!epi_sync()) { ok = false; break; }
        const float4* sv = reinterpret_cast<const float4*>(Vsm + vbuf * kTcVec);
        const float2* sw = reinterpret_cast<const float2*>(Vsm + vbuf * kTcVec + 512 * 16);
        const float* Wrow = a.W_target + (long long)idx * K;
        for (int j0 = 16 * cq; j0 < Kp; j0 += 64) {
          float lam[16];
          if (valid && j0 + 16 <= K) {
#pragma unroll
            for (int e = 0; e < 16; e += 4) {
              const float4 w4 = __ldg(reinterpret_cast<const float4*>(Wrow + j0 + e));
              lam[e] = w4.x; lam[e + 1] = w4.y; lam[e + 2] = w4.z; lam[e + 3] = w4.w;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) lam[e] = (valid && j0 + e < K) ? __ldg(Wrow + j0 + e) : 0.f;
          }
          uint32_t packed[8];
          row_pass16(valid ? role : 2, j0, lam, sv, sw, a.fmt, packed, beta0, beta1, infl0, infl1);
          store_a16(Asm, r, j0, packed);
        }
        // (the per-layer constant was summed with round-to-nearest atomics: 1.001 covers their rounding)
        if (valid && role != 2) ucon = __fmaf_ru(1.001f, a.ucon[(long long)t * (a.L - 1) + target - 1], ucon);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full);
        vbuf ^= 1;
      }
      // ---- stages -------------------------------------------------------------------------------
      for (int k = target - 1; k >= 0 && ok; --k) {
        // stage the vectors of the next pass while the tensor cores work
        stage_vectors(t, k - 1, vbuf);
        if (!epi_sync()) { ok = false; break; }
        if (!mbar_wait(acc_full, nacc & 1u)) { ok = false; break; }
        ++nacc;
        tc_fence_after();
        const float4* sv = reinterpret_cast<const float4*>(Vsm + vbuf * kTcVec);
        const float2* sw = reinterpret_cast<const float2*>(Vsm + vbuf * kTcVec + 512 * 16);
        const int N = a.widths[k];
        if (k > 0) {
          const int Np = (N + 63) & ~63;
          for (int j0 = 16 * cq; j0 < Np; j0 += 64) {
            float lam[16];
            if (j0 < N) tmem_ld16(t_lane + (uint32_t)j0, lam);
            else
#pragma unroll
              for (int e = 0; e < 16; ++e) lam[e] = 0.f;
            uint32_t packed[8];
            row_pass16(valid ? role : 2, j0, lam, sv, sw, a.fmt, packed, beta0, beta1, infl0, infl1);
            store_a16(Asm, r, j0, packed);
          }
          if (valid && role != 2) ucon = __fmaf_ru(1.001f, a.ucon[(long long)t * (a.L - 1) + k - 1], ucon);
          tc_fence_before();
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(a_full);
          vbuf ^= 1;
          continue;
        }
        // ---- last stage: concretise over the displacement box (sw = {dlo, dhi}) ------------------
        const int n = N;  // = widths[0]
        const bool output = target == a.L - 1;
        const int n_x = a.widths[a.L];
        float* Jbuf = reinterpret_cast<float*>(Asm);  // [42][n + 1] Jacobian rows of this tile
        const int jstride = n + 1;
        const int l0 = output ? tile * (a.rows_per_tile / 3) : 0;
        if (output) {
          // Jacobian rows of an output tile go to shared memory first (TMEM loads are warp-collective,
          // so every lane loads and only the Jacobian lanes store)
          for (int j0 = 16 * cq; j0 < n; j0 += 64) {
            float lam[16];
            tmem_ld16(t_lane + (uint32_t)j0, lam);
            if (valid && role == 2)
#pragma unroll
              for (int e = 0; e < 16; ++e) Jbuf[(idx - l0) * jstride + j0 + e] = lam[e];
          }
          if (!epi_sync()) { ok = false; break; }
        }
        const bool bound_row = valid && role != 2;
        const bool dn = role == 0;
        const float* Jr = Jbuf + (output && bound_row ? idx - l0 : 0) * jstride;
        float sum0 = 0.f, sum1 = 0.f;
        for (int j0 = 16 * cq; j0 < n; j0 += 64) {
          float lam[16];
          tmem_ld16(t_lane + (uint32_t)j0, lam);
          if (bound_row) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int j = j0 + e;
              const float2 d = sw[j];  // the box contains the nominal: dlo <= 0 <= dhi
              float mlo = lam[e], mhi = lam[e];
              if (output) {
                const float jv = Jr[j];
                if (a.residual && j == idx) {
                  const float aret = 1.f + jv;
                  mlo = __fadd_rd(__fsub_rd(lam[e], aret), 1.f);
                  mhi = __fadd_ru(__fsub_ru(lam[e], aret), 1.f);
                } else {
                  mlo = __fsub_rd(lam[e], jv);
                  mhi = __fsub_ru(lam[e], jv);
                }
              }
              // [mlo, mhi] x [dlo, dhi] with dlo <= 0 <= dhi: min = min(mlo dhi, mhi dlo), max = max(mhi dhi, mlo dlo)
              float term;
              if (dn) term = fminf(__fmul_rd(mlo, d.y), __fmul_rd(mhi, d.x));
              else term = fmaxf(__fmul_ru(mhi, d.y), __fmul_ru(mlo, d.x));
              if (e & 1) sum1 = dn ? __fadd_rd(sum1, term) : __fadd_ru(sum1, term);
              else sum0 = dn ? __fadd_rd(sum0, term) : __fadd_ru(sum0, term);
            }
          }
        }
        tc_fence_before();
        // combine the four column quarters of each row
        float* st = stat + (r * 4 + cq) * 4;
        st[0] = dn ? __fadd_rd(sum0, sum1) : __fadd_ru(sum0, sum1);
        st[1] = dn ? __fadd_rd(beta0, beta1) : __fadd_ru(beta0, beta1);
        st[2] = a.tight ? 0.f : __fadd_ru(__fadd_ru(infl0, infl1), cq == 0 ? ucon : 0.f);
        if (!epi_sync()) { ok = false; break; }
        if (cq == 0 && bound_row) {
          const float* s0 = stat + (r * 4) * 4;
          float tot = s0[0], beta = s0[1], infl = s0[2];
          for (int c = 1; c < 4; ++c) {
            tot = dn ? __fadd_rd(tot, s0[4 * c]) : __fadd_ru(tot, s0[4 * c]);
            beta = dn ? __fadd_rd(beta, s0[4 * c + 1]) : __fadd_ru(beta, s0[4 * c + 1]);
            infl = __fadd_ru(infl, s0[4 * c + 2]);
          }
          float val = dn ? __fsub_rd(__fadd_rd(tot, beta), infl) : __fadd_ru(__fadd_ru(tot, beta), infl);
          const bool nonfinite = !isfinite(val);
          const bool badrow = a.bad[t] != 0 || nonfinite;
          const float slack = __fmul_ru(2.f, infl);
          if (!output) {
            const long long o = (long long)t * a.H + a.hoff[target] + idx;
            const float zh = a.zhat[o], e = a.zrad[o];
            val = dn ? __fadd_rd(__fsub_rd(zh, e), val) : __fadd_ru(__fadd_ru(zh, e), val);
            if (badrow) val = dn ? -CUDART_INF_F : CUDART_INF_F;
            if (dn) a.lo[o] = val; else a.hi[o] = val;
            atomicMax(reinterpret_cast<int*>(a.bslack + o), __float_as_int(isfinite(slack) ? slack : 3.0e38f));
          } else {
            if (badrow) val = dn ? -CUDART_INF_F : CUDART_INF_F;
            const long long o = (long long)t * n_x + idx;
            if (dn) a.r_lo[o] = val; else a.r_hi[o] = val;
            stat[(r * 4) * 4 + 3] = val;   // final value, read by the slack/Gamma pass below
            stat[(r * 4) * 4 + 2] = slack;
          }
          if (nonfinite && a.bad[t] == 0) atomicOr(a.flags, LEB_ASYNC_OVERFLOW);
        }
        if (output) {
          if (!epi_sync()) { ok = false; break; }
          // Jacobian rows of this tile -> A, B (coalesced), stated slack and Gamma map per state row
          const int nl = min(a.rows_per_tile / 3, n_x - l0);
          for (int e = etid; e < nl * n; e += ethr) {
            const int ll = e / n, m = e - ll * n;
            const float jv = Jbuf[ll * jstride + m];
            const int l = l0 + ll;
            if (m < n_x) {
              if (a.A) a.A[((long long)t * n_x + l) * n_x + m] = (a.residual && m == l) ? 1.f + jv : jv;
            } else if (a.B) {
              a.B[((long long)t * n_x + l) * (n - n_x) + (m - n_x)] = jv;
            }
          }
          for (int ll = etid; ll < nl; ll += ethr) {
            const float* sl = stat + (3 * ll * 4) * 4;
            const float* su = stat + ((3 * ll + 1) * 4) * 4;
            const long long o = (long long)t * n_x + l0 + ll;
            if (a.eps) a.eps[o] = fmaxf(sl[2], su[2]);
            if (a.gamma_c) {
              const float lo = sl[3], hi = su[3];
              const float c = 0.5f * lo + 0.5f * hi;
              a.gamma_c[o] = c;
              a.gamma_r[o] = __fadd_ru(fmaxf(__fsub_ru(hi, c), __fsub_ru(c, lo)), a.gamma_pad);
            }
          }
        }
        // the next item's prologue overwrites Asm (J rows), the vectors and TMEM: everyone must be done
        if (!epi_sync()) { ok = false; break; }
      }
      if (*(volatile int*)&s_abort) ok = false;
    }
    if (!ok) {
      s_abort = 1;
      if (lane == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

__device__ __forceinline__ uint16_t to_op(float a, int fmt) {
  if (fmt == 0) return __half_as_ushort(__float2half_rn(a));
  return __bfloat16_as_ushort(__float2bfloat16_rn(a));
}

__global__ void transpose_round_kernel(const float* W, int rows, int cols, uint16_t* WT, int fmt) {
  // W [rows, cols] -> WT [cols, rows] in the operand format
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / rows, r = e - c * rows;  // WT[c][r] = W[r][c]
    WT[e] = to_op(W[r * cols + c], fmt);
  }
}

}  // namespace

struct TcState {
  uint16_t* WT[kMaxLayers] = {};
  CUtensorMap maps[kMaxLayers];
};

static TcState* tc_state(const Ctx& c) { return reinterpret_cast<TcState*>(c.mlp.tc); }

leb_status tc_prepare(Ctx& c) {
  MlpModel& m = c.mlp;
  for (int i = 0; i < m.L; ++i) {
    const int w = m.widths[i];
    if (w % 32 != 0 || w > 512) return LEB_ERR_UNSUPPORTED;  // N of a stage: two halves of multiples of 16
  }
  for (int i = 1; i < m.L; ++i)
    if (m.widths[i] % 64 != 0) return LEB_ERR_UNSUPPORTED;   // K of a stage: whole 64-column blocks
  if (m.widths[m.L] > 42 * 64) return LEB_ERR_UNSUPPORTED;
  auto enc = encode_fn();
  if (!enc) return LEB_ERR_UNSUPPORTED;
  TcState* st = new TcState();
  m.tc = st;
  const int fmt = m.prec == LEB_PREC_BF16 ? 1 : 0;
  for (int k = 0; k + 1 < m.L; ++k) {
    const int K = m.widths[k + 1], N = m.widths[k];  // W_k is [K, N]; operand B = W_k^T [N, K]
    if (cudaMalloc(&st->WT[k], (size_t)K * N * 2) != cudaSuccess) return LEB_ERR_CUDA;
    transpose_round_kernel<<<256, 256>>>(m.W[k], K, N, st->WT[k], fmt);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    const int nh = N > 256 ? 2 : 1;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)(N / nh)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&st->maps[k], fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     st->WT[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return LEB_ERR_UNSUPPORTED;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return LEB_ERR_CUDA;
  if (cudaFuncSetAttribute(crown_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess)
    return LEB_ERR_CUDA;
  return LEB_OK;
}

const void* tc_weight_t(const Ctx& c, int k) {
  const TcState* st = tc_state(c);
  return st ? st->WT[k] : nullptr;
}

void tc_release(Ctx& c) {
  adj_tc_release(c);
  TcState* st = tc_state(c);
  if (!st) return;
  for (int k = 0; k < kMaxLayers; ++k) cudaFree(st->WT[k]);
  delete st;
  c.mlp.tc = nullptr;
}

float gamma_tc(int K);  // declared in internal.h
float gamma_tc(int K) {
  // accumulation of K exact products in FP32 with unit roundoff 2^-23 (no round-to-nearest assumed)
  const double u = std::ldexp(1.0, -23);
  const double g = K * u / (1.0 - K * u);
  return std::nextafterf((float)g * 1.0000002f, INFINITY);
}

leb_status tc_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, float* r_lo, float* r_hi, float* A,
                    float* B, float* eps, cudaStream_t s, const int* bad, const leb_options* opt, int* flags, bool tight) {
  const MlpModel& m = c.mlp;
  TcState* st = tc_state(c);
  if (!st) return LEB_ERR_UNSUPPORTED;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k + 1 < m.L; ++k) a.tmap[k] = st->maps[k];
  a.L = m.L;
  for (int i = 0; i <= m.L; ++i) a.widths[i] = m.widths[i];
  a.residual = m.residual;
  a.fmt = m.prec == LEB_PREC_BF16 ? 1 : 0;
  a.T = T;
  a.target = target;
  const bool output = target == m.L - 1;
  a.nroles = output ? 3 : 2;
  a.rows_total = a.nroles * m.widths[target + 1];
  a.rows_per_tile = output ? 126 : 128;
  a.tiles_per_t = (a.rows_total + a.rows_per_tile - 1) / a.rows_per_tile;
  a.H = L.H;
  for (int i = 0; i + 1 < m.L; ++i) a.hoff[i] = L.hoff[i];
  a.W_target = m.W[target];
  a.zhat = ws + L.zhat;
  a.zrad = ws + L.zrad;
  a.sL = ws + L.sL;
  a.tL = ws + L.tL;
  a.sU = ws + L.sU;
  a.tU = ws + L.tU;
  a.D = ws + L.D;
  a.winf = ws + L.winf;
  a.ucon = ws + L.ucon;
  a.dlo = ws + L.dlo;
  a.dhi = ws + L.dhi;
  a.bad = bad;
  a.lo = ws + L.lo;
  a.hi = ws + L.hi;
  a.bslack = ws + L.bslack;
  a.r_lo = r_lo;
  a.r_hi = r_hi;
  a.A = A;
  a.B = B;
  a.eps = eps;
  a.gamma_c = opt ? opt->gamma_c : nullptr;
  a.gamma_r = opt ? opt->gamma_r : nullptr;
  a.gamma_pad = opt ? opt->gamma_pad : 0.f;
  a.flags = flags;
  a.tight = tight ? 1 : 0;
  const int items = T * a.tiles_per_t;
  const int grid = items < c.sm_count ? items : c.sm_count;
  if (grid == 0) return LEB_OK;
  timer_begin(c, s, "crown_tc_kernel");
  crown_tc_kernel<<<grid, kTcThreads, kTcSmem, s>>>(a);
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

}  // namespace leb
