// Adjoint of the CROWN remainder bound (differentiable LEBs, Sec. IV-D) on the tensor cores: the chain
// part of the reverse pass for reduced-precision (FP16 / BF16) handles.
//
// For one back-substitution target (the output rows, or the lower/upper rows of hidden layer `target`)
// and 128 chain rows of one timestep, a CTA
//   1. recomputes the chain forward:  lambda_{k-1} = (lambda_k o s_k) W_k,  k = target-1 .. 0,
//      starting from lambda_{target-1} = rows of W_target, keeping each lambda_k (k >= 0) in a per-CTA
//      scratch area (it stays in L2);
//   2. forms G_{-1} = dr / d lambda_{-1}: a lower bound takes min over the displacement box [dlo, dhi] of
//      M Delta (M_m > 0 at dlo_m, M_m < 0 at dhi_m), an upper bound the max, M = lambda_{-1} minus the
//      Jacobian row of the same state for output rows; and the direct gradients of the box's ends;
//   3. runs the chain backward:  Ga_k = G_{k-1} W_k^T,  G_k = Ga_k o s_k + g tau_k,  summing per neuron
//      over the chain rows d/ds_sel += Ga_k lambda_k, d/dtau_sel += g lambda_k (lower/upper rows) and
//      d/dD += Ga_k lambda_k (Jacobian rows).
// The slopes are those of the relaxation case selected at the evaluation point (sign of lambda_k), as
// automatic differentiation of the same algorithm would take them.
//
// Layout (transposed with respect to the forward chain kernel): the products are computed as
//   lambda_{k-1}^T = W_k^T (lambda_k o s_k)^T   and   Ga_k^T = W_k G_{k-1}^T,
// so the weights are the streamed A operand (128 neurons x 64 K tiles by TMA, a ring of kAdjStages) and
// the per-row operand is the resident B operand (128 rows x K, K-major, 128-byte swizzle). TMEM holds
// D[neuron][row]: lane = neuron inside an M-tile of 128, column = 128 * M-tile + row. Every epilogue
// thread owns one neuron (16 epilogue warps: 4 M-tiles x 4 TMEM lane quarters, four per SM
// sub-partition, with most of warpgroup 0's registers handed to them by setmaxnreg), so every sum over
// chain rows is a register sum, and the role of a row (lower, upper, Jacobian) is the same across a warp.
//
// Output rows are carried in difference form: the lower and upper rows hold delta = lambda - lambda^J
// (their operand lambda o s_sel - lambda^J o sigma'(z~) is formed in FP32 from the row and the Jacobian
// row of the same state, which sit in the same thread), so M = delta_{-1} comes out of the tensor cores
// with the operand format's relative precision instead of as a difference of two rounded chains, whose
// cancellation would flip sign(M) wherever the relaxation slopes are close to sigma'(z~).
//
// G is scaled by 1 / max |g| of the tile's rows before it is rounded to the operand format (so FP16 does
// not overflow for large cotangents); the sums are scaled back when they are added to global memory.
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "internal.h"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace leb {

constexpr int kAdjNU = 1;                           // neurons per epilogue thread (M-tiles m, m + 4 / kAdjNU)
constexpr int kAdjEpiWarps = 16 / kAdjNU;           // M-tiles per thread set x 4 TMEM lane quarters
constexpr int kAdjCtlWarps = 4;                     // warpgroup 0: TMA warp, MMA warp, two idle warps
constexpr int kAdjThreads = 32 * (kAdjCtlWarps + kAdjEpiWarps);
// Register split (setmaxnreg): warpgroup 0 keeps 32 registers a thread, the epilogue warpgroups take 112.
// The increases draw on what the block was launched with, so the compiled kernel must have at least
// kAdjRegsLaunchMin registers a thread (checked before any launch).
constexpr int kAdjRegsCtl = 32, kAdjRegsEpi = 112;
constexpr int kAdjRegsLaunchMin = (128 * kAdjRegsCtl + 32 * kAdjEpiWarps * kAdjRegsEpi + kAdjThreads - 1) / kAdjThreads;
constexpr int kAdjStages = 6;                       // weight-tile ring
constexpr int kAdjATile = 128 * 64 * 2;             // 128 neurons x 64 K x 2 bytes
constexpr int kAdjBRegion = 128 * 512 * 2;          // 128 rows x K <= 512 x 2 bytes
constexpr int kAdjSmall = 1024 + 32 + 16 * 8;   // row cotangents, their scale, barriers
constexpr int kAdjSmem = 1024 + kAdjBRegion + kAdjStages * kAdjATile + kAdjSmall;
static_assert(kAdjSmem <= 227 * 1024, "adjoint tensor-core shared memory");

struct AdjTcArgs {
  CUtensorMap fwd[kMaxLayers];   // W_k^T [widths[k] rows, widths[k+1] cols] (operand format), box {64, 128}
  CUtensorMap bwd[kMaxLayers];   // W_k   [widths[k+1] rows, widths[k] cols] (operand format), box {64, 128}
  int L;
  int widths[kMaxLayers + 1];
  int fmt;                       // 0 FP16, 1 BF16
  int T, target, nroles, rows_total, rows_per_tile, tiles_per_t;
  int H;
  int hoff[kMaxLayers];
  int soff[kMaxLayers];          // scratch offset (in neurons) of lambda_k, k = 0 .. target-2
  int stot;                      // neurons per CTA scratch row block
  const float* W_target;         // FP32 [widths[target+1], widths[target]]
  const float *sL, *sU, *tL, *tU, *D;   // [T, H]
  const float *dlo, *dhi;        // [T, n] the displacement box Delta = X - alpha~ (dlo <= 0 <= dhi)
  const float *g_lo, *g_hi;      // output target: [T, n_x]
  const float *gl, *gu;          // hidden target: [T, H]
  float *gsL, *gsU, *gtL, *gtU, *gD, *gdlo, *gdhi;
  __half* scratch;               // gridDim.x x stot x 128 lambdas, FP16
  int* flags;
};

__device__ __forceinline__ uint32_t pack2(float x, float y, int fmt) {
  if (fmt == 0) {
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ uint16_t op_round(float x, int fmt) {
  if (fmt == 0) return __half_as_ushort(__float2half_rn(x));
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// The per-row operand B (N = 128 chain rows x K neurons) is MN-major with 128-byte swizzle: atom
// (row block rb = r / 64, neuron group g = j / 8) at rb * kAdjLbo + g * 1024 holds neuron j's 64 rows as
// 128 contiguous bytes at (j mod 8) * 128, the 16-byte chunk index XORed with j mod 8. Byte offset of the
// 8 rows r0 .. r0 + 7 (r0 a multiple of 8) of neuron j:
constexpr uint32_t kAdjLbo = 64 * 1024;   // 64 neuron groups x 1 KB
__device__ __forceinline__ uint32_t b_off8(int r0, int j) {
  return (uint32_t)((r0 >> 6) * kAdjLbo + (j >> 3) * 1024 + (j & 7) * 128 + ((((r0 & 63) >> 3) ^ (j & 7)) << 4));
}

__global__ void __launch_bounds__(kAdjThreads, 1) adjoint_tc_kernel(const __grid_constant__ AdjTcArgs a) {
  extern __shared__ uint8_t sraw[];
  // 1024-byte aligned base, as an offset from the shared array (so that every derived pointer keeps the
  // shared address space and its accesses compile to shared-memory instructions)
  uint8_t* base = sraw + ((1024u - (smem_u32(sraw) & 1023u)) & 1023u);
  uint8_t* Bop = base;                                   // per-row operand
  uint8_t* ring = base + kAdjBRegion;                    // weight tiles
  float* gws = reinterpret_cast<float*>(ring + kAdjStages * kAdjATile);   // [2][128] row cotangents
  float* wmax = gws + 256;                                                 // [2][4] per-warp max |g|
  uint64_t* bars = reinterpret_cast<uint64_t*>(wmax + 8);
  uint64_t* full = bars;                      // [kAdjStages]
  uint64_t* empty = bars + kAdjStages;        // [kAdjStages]
  uint64_t* a_full = bars + 2 * kAdjStages;   // operand written by the epilogue
  uint64_t* acc_full = a_full + 1;            // accumulators complete
  uint64_t* drain = acc_full + 1;
  uint64_t* ebar = drain + 1;                 // epilogue-warps barrier
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = a.T * a.tiles_per_t;
  const int target = a.target;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kAdjStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(a_full, kAdjEpiWarps);
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
    mbar_init(ebar, kAdjEpiWarps);
    mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 1) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // stage s of an item: s < target: forward stage k = target-1-s; else backward stage k = s - target
  const int n_stages = 2 * target;
  auto stage_shape = [&](int s, int& M, int& K, const CUtensorMap*& map) {
    if (s < target) {
      const int k = target - 1 - s;
      M = a.widths[k];
      K = a.widths[k + 1];
      map = &a.fwd[k];
    } else {
      const int k = s - target;
      M = a.widths[k + 1];
      K = a.widths[k];
      map = &a.bwd[k];
    }
  };

  if (warp < kAdjCtlWarps) regs_dec<kAdjRegsCtl>();   // warpgroup 0: its four warps together
  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer (weight tiles)
    if (lane == 0) {
      for (int k = 0; k < target; ++k) {
        tma_prefetch_desc(&a.fwd[k]);
        tma_prefetch_desc(&a.bwd[k]);
      }
      uint32_t kb = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        for (int s = 0; s < n_stages && ok; ++s) {
          int M, K;
          const CUtensorMap* map;
          stage_shape(s, M, K, map);
          const int nM = (M + 127) / 128, nK = (K + 63) / 64;
          for (int kc = 0; kc < nK && ok; ++kc)
            for (int c = 0; c < nM; ++c, ++kb) {
              const int slot = (int)(kb % kAdjStages);
              if (kb >= (uint32_t)kAdjStages && !mbar_wait(&empty[slot], ((kb / kAdjStages) - 1) & 1u)) {
                ok = false;
                break;
              }
              if (*(volatile int*)&s_abort) { ok = false; break; }
              mbar_arrive_expect_tx(&full[slot], (uint32_t)kAdjATile);
              tma_load_2d(ring + (size_t)slot * kAdjATile, map, kc * 64, c * 128, &full[slot]);
            }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      // every issued load must land before the block exits
      for (uint32_t j = (kb > (uint32_t)kAdjStages ? kb - kAdjStages : 0u); j < kb; ++j)
        mbar_wait(&full[j % kAdjStages], (j / kAdjStages) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t ring_base = smem_u32(ring), b_base = smem_u32(Bop);
      const uint32_t idesc = idesc_f16_bmn(128, 128, a.fmt);
      uint32_t kb = 0, na = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        for (int s = 0; s < n_stages && ok; ++s) {
          int M, K;
          const CUtensorMap* map;
          stage_shape(s, M, K, map);
          const int nM = (M + 127) / 128, nK = (K + 63) / 64;
          if (!mbar_wait(a_full, na & 1u)) { ok = false; break; }
          ++na;
          tc_fence_after();
          for (int kc = 0; kc < nK && ok; ++kc)
            for (int c = 0; c < nM; ++c, ++kb) {
              const int slot = (int)(kb % kAdjStages);
              if (!mbar_wait(&full[slot], (kb / kAdjStages) & 1u)) { ok = false; break; }
              tc_fence_after();
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = sw128_desc(ring_base + slot * kAdjATile + kk * 32);
                const uint64_t bd = sw128_mn_desc(b_base + (uint32_t)(kc * 8 + kk * 2) * 1024u, kAdjLbo, 1024u);
                tc_mma_f16(tmem + (uint32_t)(c * 128), ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
              }
              tc_commit(&empty[slot]);
            }
          tc_commit(acc_full);
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      tc_commit(drain);
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp >= kAdjCtlWarps) {
    regs_inc<kAdjRegsEpi>();   // the epilogue warpgroups
    // ------------------------------------------------------------------ epilogue warps
    // Each thread owns kAdjNU neurons: nrn[0] in M-tile mt and, with two, nrn[1] = nrn[0] + 256 in M-tile
    // mt + 2 (same TMEM lane), worked on side by side. The code below is written for up to two; with one,
    // every second-neuron branch is dead.
    const int q = warp & 3;                    // TMEM lane quarter
    const int mt = (warp - kAdjCtlWarps) >> 2;   // M-tile of the thread's first neuron
    const int nrn0 = mt * 128 + q * 32 + lane;
    const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * 128);   // + 256 for nrn[1]
    const int etid = threadIdx.x - 32 * kAdjCtlWarps;
    __half* scr = a.scratch + (size_t)blockIdx.x * a.stot * 128;
    const int n = a.widths[0];
    const bool output = target == a.L - 1;
    uint32_t nacc = 0, nbar = 0;
    int gb = 0;
    bool ok = true;
    auto epi_sync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) mbar_arrive(ebar);
      const bool res = mbar_wait_warp(ebar, nbar & 1u);
      ++nbar;
      return res;
    };
    auto operand_ready = [&]() {
      tc_fence_before();
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_full);
    };
    auto wait_acc = [&]() -> bool {
      if (!mbar_wait_warp(acc_full, nacc & 1u)) return false;
      ++nacc;
      tc_fence_after();
      return true;
    };
    // 8 consecutive rows r0 .. r0 + 7 of neuron j into the operand (one 16-byte store)
    auto put8 = [&](int r0, int j, const float* v) {
      uint4 q;
      q.x = pack2(v[0], v[1], a.fmt);
      q.y = pack2(v[2], v[3], a.fmt);
      q.z = pack2(v[4], v[5], a.fmt);
      q.w = pack2(v[6], v[7], a.fmt);
      *reinterpret_cast<uint4*>(Bop + b_off8(r0, j)) = q;
    };

    // Pulls the thread's neurons' entries of hidden layer hl's vectors (sL, sU, D and, with taus,
    // tL, tU) of timestep t into L1; issued before a wait for the tensor cores, whose work hides it.
    auto pf_vec = [&](int t, int hl, bool taus) {
      const int width = a.widths[hl + 1];
#pragma unroll
      for (int u = 0; u < kAdjNU; ++u) {
        const int j = nrn0 + 256 * u;
        if (j < width) {
          const long long o = (long long)t * a.H + a.hoff[hl] + j;
          prefetch_l1(a.sL + o);
          prefetch_l1(a.sU + o);
          prefetch_l1(a.D + o);
          if (taus) {
            prefetch_l1(a.tL + o);
            prefetch_l1(a.tU + o);
          }
        }
      }
    };

    // Rows of a tile come in groups of NR (output: lower, upper, Jacobian; hidden: lower, upper) and a
    // tile starts on a group, so the role of row r0 + e with r0 a multiple of 8 NR is e mod NR: a
    // compile-time constant in the unrolled loops. Rows past the tile's valid rows carry zero cotangents
    // and a zero first operand, so every value derived from them is zero.
    auto run_item = [&](auto nr_c, int t, int row0, int nrows, const float* gw, float ginv, float gscale) -> bool {
      constexpr int NR = decltype(nr_c)::value;
      constexpr int GS = 8 * NR;                 // rows per group: whole groups of NR, whole 8-column loads
      const int Kt = a.widths[target];
      // ---- prologue: B = (W_target rows o s_{target-1}) (difference form for output rows) ----------
      // Both neurons of the thread go through the rows together, and the W_target entries of the next
      // 8-row chunk (the row groups it touches, at most 4) are loaded while a chunk is written.
      {
        const int Kp = (Kt + 63) & ~63;
        const int nu = (kAdjNU == 2 && nrn0 + 256 < Kp) ? 2 : (nrn0 < Kp ? 1 : 0);   // neurons of this thread in the layer
        if (nu > 0) {
          bool live[2];
          float sl[2], su[2], dd[2];
          const float* wcol[2];
#pragma unroll
          for (int u = 0; u < kAdjNU; ++u) {
            const int j = nrn0 + 256 * u;
            live[u] = u < nu && j < Kt;
            const long long o = (long long)t * a.H + a.hoff[target - 1] + (live[u] ? j : 0);
            sl[u] = live[u] ? a.sL[o] : 0.f;
            su[u] = live[u] ? a.sU[o] : 0.f;
            dd[u] = live[u] ? a.D[o] : 0.f;
            wcol[u] = a.W_target + (live[u] ? j : 0);
          }
          // W_target entries of the row groups rb / NR .. rb / NR + 3 (0 for a group past the valid rows)
          auto wload = [&](int rb, float2 (&w)[4]) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int g = rb / NR + i;
              const bool grp = NR * g + NR - 1 < nrows;
              const long long wo = (long long)(row0 / NR + g) * Kt;
              w[i].x = (live[0] && grp) ? __ldg(wcol[0] + wo) : 0.f;
              w[i].y = (live[1] && grp) ? __ldg(wcol[1] + wo) : 0.f;
            }
          };
          float2 wn[4];
          wload(0, wn);
#pragma unroll 1
          for (int rb = 0; rb < 128; rb += 8) {
            const float2 wc[4] = {wn[0], wn[1], wn[2], wn[3]};
            if (rb + 8 < 128) wload(rb + 8, wn);
            const int off = rb % NR;
            const uint32_t lm = NR == 3 ? (0x49u << ((3 - off) % 3)) & 0xFFu : (off == 0 ? 0x55u : 0xAAu);
            const uint32_t jm = NR == 3 ? (0x49u << ((5 - off) % 3)) & 0xFFu : 0u;
            float v0[8], v1[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const bool isL = (lm >> e) & 1u, isJ = (jm >> e) & 1u;
              const int gi = (off + e) / NR;   // group of row rb + e, relative to rb / NR
              const float2 lam = gi == 0 ? wc[0] : (gi == 1 ? wc[1] : (gi == 2 ? wc[2] : wc[3]));
              const float jd0 = NR == 3 ? lam.x * dd[0] : 0.f, jd1 = NR == 3 ? lam.y * dd[1] : 0.f;
              const bool useL0 = isL == !signbit(lam.x), useL1 = isL == !signbit(lam.y);
              v0[e] = isJ ? jd0 : fmaf(lam.x, useL0 ? sl[0] : su[0], -jd0);
              v1[e] = isJ ? jd1 : fmaf(lam.y, useL1 ? sl[1] : su[1], -jd1);
            }
            put8(rb, nrn0, v0);
            if (nu > 1) put8(rb, nrn0 + 256, v1);
          }
        }
        operand_ready();
      }
      // ---- forward stages k = target-1 .. 1 --------------------------------------------------------
      for (int k = target - 1; k >= 1; --k) {
        pf_vec(t, k - 1, false);
        if (!wait_acc()) return false;
        const int N = a.widths[k];             // neurons of hidden layer k-1 (rows of this product)
        const int Np = (N + 63) & ~63;
#pragma unroll
        for (int u = 0; u < kAdjNU; ++u) {
          const int j = nrn0 + 256 * u;
          if (j >= Np) continue;
          const bool live = j < N;
          const long long o = (long long)t * a.H + a.hoff[k - 1] + (live ? j : 0);
          const float sl = live ? a.sL[o] : 0.f, su = live ? a.sU[o] : 0.f, dd = live ? a.D[o] : 0.f;
          __half* lrow = scr + (size_t)(a.soff[k - 1] + (live ? j : 0)) * 128;
          const uint32_t tl = t_lane + 256u * u;
#pragma unroll 1
          for (int r0 = 0; r0 < 128; r0 += GS) {
            const int nch = min(NR, (128 - r0) >> 3);
            float d[GS];
#pragma unroll
            for (int h = 0; h < NR; ++h) {
              if (h < nch) tmem_ld8_nowait(tl + (uint32_t)(r0 + 8 * h), d + 8 * h);
              else
#pragma unroll
                for (int e = 0; e < 8; ++e) d[8 * h + e] = 0.f;   // rows past the tile
            }
            tmem_wait_ld();
            if (NR == 3)
#pragma unroll
              for (int e = 0; e < GS; e += NR) {
                d[e] += d[e + 2];               // lambda of the lower row
                d[e + 1] += d[e + 2];           // lambda of the upper row
              }
            // lambda is kept in FP16 for the backward pass, and the line choice (sign of lambda) is made
            // on that stored value here and there alike
            __half lh[GS];
#pragma unroll
            for (int e = 0; e < GS; ++e) lh[e] = __float2half_rn(d[e]);
            float v[GS];
#pragma unroll
            for (int e = 0; e < GS; e += NR) {
              const bool nl = !(__half_as_ushort(lh[e]) & 0x8000u), nu_ = !(__half_as_ushort(lh[e + 1]) & 0x8000u);
              if (NR == 3) {
                const float jd = d[e + 2] * dd;
                v[e] = fmaf(d[e], nl ? sl : su, -jd);
                v[e + 1] = fmaf(d[e + 1], nu_ ? su : sl, -jd);
                v[e + NR - 1] = jd;
              } else {
                v[e] = d[e] * (nl ? sl : su);
                v[e + 1] = d[e + 1] * (nu_ ? su : sl);
              }
            }
#pragma unroll
            for (int h = 0; h < NR; ++h)
              if (h < nch) put8(r0 + 8 * h, j, v + 8 * h);
            if (live)
#pragma unroll
              for (int h = 0; h < NR; ++h)
                if (h < nch) {
                  uint4 q4;
                  q4.x = (uint32_t)__half_as_ushort(lh[8 * h]) | ((uint32_t)__half_as_ushort(lh[8 * h + 1]) << 16);
                  q4.y = (uint32_t)__half_as_ushort(lh[8 * h + 2]) | ((uint32_t)__half_as_ushort(lh[8 * h + 3]) << 16);
                  q4.z = (uint32_t)__half_as_ushort(lh[8 * h + 4]) | ((uint32_t)__half_as_ushort(lh[8 * h + 5]) << 16);
                  q4.w = (uint32_t)__half_as_ushort(lh[8 * h + 6]) | ((uint32_t)__half_as_ushort(lh[8 * h + 7]) << 16);
                  *reinterpret_cast<uint4*>(lrow + r0 + 8 * h) = q4;
                }
          }
        }
        operand_ready();
      }
      // ---- G_{-1} from lambda_{-1} (neurons = inputs m < n) --------------------------------------------
      {
#pragma unroll
        for (int u = 0; u < kAdjNU; ++u)
          if (nrn0 + 256 * u < n) {
            prefetch_l1(a.dlo + (long long)t * n + nrn0 + 256 * u);
            prefetch_l1(a.dhi + (long long)t * n + nrn0 + 256 * u);
          }
        if (!wait_acc()) return false;
        const int np = (n + 63) & ~63;
#pragma unroll
        for (int u = 0; u < kAdjNU; ++u) {
          const int j = nrn0 + 256 * u;
          if (j >= np) continue;
          const bool live = j < n;
          const float dl = live ? a.dlo[(long long)t * n + j] : 0.f, dh = live ? a.dhi[(long long)t * n + j] : 0.f;
          const float dm = 0.5f * (dl + dh);   // the derivative's value where M = 0 (mean of both sides)
          const uint32_t tl = t_lane + 256u * u;
          float gdl = 0.f, gdh = 0.f;
#pragma unroll 1
          for (int r0 = 0; r0 < 128; r0 += GS) {
            const int nch = min(NR, (128 - r0) >> 3);
            float d[GS];
#pragma unroll
            for (int h = 0; h < NR; ++h) {
              if (h < nch) tmem_ld8_nowait(tl + (uint32_t)(r0 + 8 * h), d + 8 * h);
              else
#pragma unroll
                for (int e = 0; e < 8; ++e) d[8 * h + e] = 0.f;   // rows past the tile
            }
            tmem_wait_ld();
            float v[GS];
#pragma unroll
            for (int e = 0; e < GS; e += NR) {
              const int r = r0 + e;
              // output rows: d = delta = lambda - lambda^J (M itself); hidden rows: d = lambda = M.
              // Rows past 128 (the last group) only hold zeros and are not stored.
              const float glo = r < 128 ? gw[r] * ginv : 0.f, ghi = r + 1 < 128 ? gw[r + 1] * ginv : 0.f;
              const float mlo = d[e], mhi = d[e + 1];
              const float G0 = glo * (mlo > 0.f ? dl : (mlo < 0.f ? dh : dm));
              const float G1 = ghi * (mhi > 0.f ? dh : (mhi < 0.f ? dl : dm));
              gdl = fmaf(glo, fmaxf(mlo, 0.f), fmaf(ghi, fminf(mhi, 0.f), gdl));
              gdh = fmaf(glo, fminf(mlo, 0.f), fmaf(ghi, fmaxf(mhi, 0.f), gdh));
              v[e] = G0;
              v[e + 1] = G1;
              if (NR == 3) v[e + NR - 1] = -(G0 + G1);
            }
#pragma unroll
            for (int h = 0; h < NR; ++h)
              if (h < nch) put8(r0 + 8 * h, j, v + 8 * h);
          }
          if (live && gdl != 0.f) atomicAdd(a.gdlo + (long long)t * n + j, gdl * gscale);
          if (live && gdh != 0.f) atomicAdd(a.gdhi + (long long)t * n + j, gdh * gscale);
        }
        operand_ready();
      }
      // ---- backward stages k = 0 .. target-1 -------------------------------------------------------
      // The thread's neurons go side by side.
      for (int k = 0; k < target; ++k) {
        pf_vec(t, k, true);
        if (!wait_acc()) return false;
        const int N = a.widths[k + 1];            // neurons of hidden layer k
        const bool last = k == target - 1;
        const int Np = (N + 63) & ~63;
        const int nu = (kAdjNU == 2 && nrn0 + 256 < Np) ? 2 : (nrn0 < Np ? 1 : 0);   // neurons of this thread in the layer
        if (nu > 0) {
          bool live[2];
          long long o[2];
          float sl[2], su[2], tlv[2], tu[2], dd[2];
          const __half* lrow[2];
          const float* wcol[2];
#pragma unroll
          for (int u = 0; u < kAdjNU; ++u) {
            const int j = nrn0 + 256 * u;
            live[u] = u < nu && j < N;
            o[u] = (long long)t * a.H + a.hoff[k] + (live[u] ? j : 0);
            sl[u] = live[u] ? a.sL[o[u]] : 0.f;
            su[u] = live[u] ? a.sU[o[u]] : 0.f;
            tlv[u] = live[u] ? a.tL[o[u]] : 0.f;
            tu[u] = live[u] ? a.tU[o[u]] : 0.f;
            dd[u] = live[u] ? a.D[o[u]] : 0.f;
            lrow[u] = scr + (size_t)((last ? 0 : a.soff[k]) + (live[u] ? j : 0)) * 128;
            wcol[u] = a.W_target + (live[u] ? j : 0);
          }
          const float2 dd2 = make_float2(dd[0], dd[1]);
          float2 SL = make_float2(0.f, 0.f), SU = SL, TL = SL, TU = SL, GD = SL;
          float2 wv = SL;   // lambda_{target-1} of the current row group (last stage), carried across chunks
          // 16-row chunks; the roles of a chunk's rows as bit masks (bit e: row rb + e): Jacobian rows, and
          // rows whose lower line is chosen when lambda >= 0 (lower-bound rows)
#pragma unroll 1
          for (int rb = 0; rb < 128; rb += 16) {
            const int off = rb % NR;       // role of row rb (tiles start on a row group)
            // role-0 rows: e = -off mod NR (+ NR, ...); Jacobian rows (NR = 3): e = 2 - off mod 3 (+ 3, ...)
            const uint32_t lm = NR == 3 ? (0x9249u << ((3 - off) % 3)) & 0xFFFFu : (off == 0 ? 0x5555u : 0xAAAAu);
            const uint32_t jm = NR == 3 ? (0x9249u << ((5 - off) % 3)) & 0xFFFFu : 0u;
            float ga0[16], ga1[16], l0[16], l1[16], g[16];
            tmem_ld16_nowait(t_lane + (uint32_t)rb, ga0);
            if (nu > 1) tmem_ld16_nowait(t_lane + 256u + (uint32_t)rb, ga1);
            if (!last) {
#pragma unroll
              for (int e = 0; e < 16; e += 8) {
                const uint4 v = *reinterpret_cast<const uint4*>(lrow[0] + rb + e);
                const uint4 w = nu > 1 ? *reinterpret_cast<const uint4*>(lrow[1] + rb + e) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t vv[4] = {v.x, v.y, v.z, v.w}, ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                  const float2 a2 = __half22float2(*reinterpret_cast<const __half2*>(&vv[h]));
                  const float2 b2 = __half22float2(*reinterpret_cast<const __half2*>(&ww[h]));
                  l0[e + 2 * h] = a2.x; l0[e + 2 * h + 1] = a2.y;
                  l1[e + 2 * h] = b2.x; l1[e + 2 * h + 1] = b2.y;
                }
              }
            } else {
              // lambda_{target-1}: the W_target row of each row's state, loaded at the group's first row
              // (role 0) and carried to the group's other rows, also across chunks
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                if ((lm >> e) & 1u) {
                  const int r = rb + e;
                  const bool grp = r + NR - 1 < nrows;
                  const long long wo = (long long)((row0 + r) / NR) * Kt;
                  wv.x = (live[0] && grp) ? __ldg(wcol[0] + wo) : 0.f;
                  wv.y = (live[1] && grp) ? __ldg(wcol[1] + wo) : 0.f;
                }
                l0[e] = wv.x;
                l1[e] = wv.y;
              }
            }
#pragma unroll
            for (int e = 0; e < 16; e += 4) {
              const float4 v = *reinterpret_cast<const float4*>(gw + rb + e);
              g[e] = v.x * ginv; g[e + 1] = v.y * ginv; g[e + 2] = v.z * ginv; g[e + 3] = v.w * ginv;
            }
            tmem_wait_ld();
            if (nu < 2)
#pragma unroll
              for (int e = 0; e < 16; ++e) ga1[e] = 0.f;
            float G0[16], G1[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const bool isJ = (jm >> e) & 1u, isL = (lm >> e) & 1u;
              // scalar arithmetic: the two neurons' values sit in separate arrays, so packed FP32x2
              // operations would first have to move them into register pairs
              const float x0 = ga0[e], x1 = ga1[e], la = l0[e], lb = l1[e];
              const float p10 = x0 * la, p11 = x1 * lb, p20 = g[e] * la, p21 = g[e] * lb;
              // lower line chosen (sg) / upper line chosen (ng); both 0 on Jacobian rows. The choice is
              // the sign bit of the stored lambda, as in the forward recompute.
              const bool u0 = isL == !signbit(la), u1 = isL == !signbit(lb);
              const float sg0 = !isJ && u0 ? 1.f : 0.f, sg1 = !isJ && u1 ? 1.f : 0.f;
              const float ng0 = !isJ && !u0 ? 1.f : 0.f, ng1 = !isJ && !u1 ? 1.f : 0.f;
              SL.x = fmaf(sg0, p10, SL.x);
              SL.y = fmaf(sg1, p11, SL.y);
              SU.x = fmaf(ng0, p10, SU.x);
              SU.y = fmaf(ng1, p11, SU.y);
              TL.x = fmaf(sg0, p20, TL.x);
              TL.y = fmaf(sg1, p21, TL.y);
              TU.x = fmaf(ng0, p20, TU.x);
              TU.y = fmaf(ng1, p21, TU.y);
              float2 G;
              if (isJ) {
                GD.x += p10;
                GD.y += p11;
                G = make_float2(x0 * dd2.x, x1 * dd2.y);
              } else {
                const float sv0 = u0 ? sl[0] : su[0], sv1 = u1 ? sl[1] : su[1];
                const float tv0 = u0 ? tlv[0] : tu[0], tv1 = u1 ? tlv[1] : tu[1];
                G = make_float2(fmaf(x0, sv0, g[e] * tv0), fmaf(x1, sv1, g[e] * tv1));
              }
              G0[e] = G.x;
              G1[e] = G.y;
            }
            if (!last) {
              put8(rb, nrn0, G0);
              put8(rb + 8, nrn0, G0 + 8);
              if (nu > 1) {
                put8(rb, nrn0 + 256, G1);
                put8(rb + 8, nrn0 + 256, G1 + 8);
              }
            }
          }
          const float gsl[2] = {SL.x, SL.y}, gsu[2] = {SU.x, SU.y}, gtl[2] = {TL.x, TL.y}, gtu[2] = {TU.x, TU.y};
          const float gd[2] = {GD.x, GD.y};
#pragma unroll
          for (int u = 0; u < kAdjNU; ++u)
            if (live[u]) {
              if (gsl[u] != 0.f) atomicAdd(a.gsL + o[u], gsl[u] * gscale);
              if (gsu[u] != 0.f) atomicAdd(a.gsU + o[u], gsu[u] * gscale);
              if (gtl[u] != 0.f) atomicAdd(a.gtL + o[u], gtl[u] * gscale);
              if (gtu[u] != 0.f) atomicAdd(a.gtU + o[u], gtu[u] * gscale);
              if (gd[u] != 0.f) atomicAdd(a.gD + o[u], gd[u] * gscale);
            }
        }
        if (!last) operand_ready();
      }
      return true;
    };

    for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      const int t = item / a.tiles_per_t, tile = item - t * a.tiles_per_t;
      const int row0 = tile * a.rows_per_tile;
      const int nrows = min(a.rows_per_tile, a.rows_total - row0);   // valid rows of this tile
      // ---- row cotangents of the tile (0 past the valid rows) and their scale ----------------------
      float* gw = gws + gb * 128;
      if (etid < 128) {
        float g = 0.f;
        if (etid < nrows) {
          const int grow = row0 + etid, role = grow % a.nroles, idx = grow / a.nroles;
          if (output) {
            const int nx = a.widths[a.L];
            g = role == 0 ? a.g_lo[(long long)t * nx + idx] : (role == 1 ? a.g_hi[(long long)t * nx + idx] : 0.f);
          } else {
            const long long o = (long long)t * a.H + a.hoff[target] + idx;
            g = role == 0 ? a.gl[o] : a.gu[o];
          }
        }
        gw[etid] = g;
        float m = fabsf(g);
#pragma unroll
        for (int dlt = 16; dlt > 0; dlt >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, dlt));
        if (lane == 0) wmax[gb * 4 + (etid >> 5)] = m;
      }
      if (!epi_sync()) { ok = false; break; }
      const float gmax = fmaxf(fmaxf(wmax[gb * 4], wmax[gb * 4 + 1]), fmaxf(wmax[gb * 4 + 2], wmax[gb * 4 + 3]));
      const float gscale = (gmax > 0.f && isfinite(gmax)) ? gmax : 1.f;
      const float ginv = 1.f / gscale;
      gb ^= 1;
      ok = output ? run_item(std::integral_constant<int, 3>(), t, row0, nrows, gw, ginv, gscale)
                  : run_item(std::integral_constant<int, 2>(), t, row0, nrows, gw, ginv, gscale);
      if (!ok) break;
      tc_fence_before();
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

PFN_cuTensorMapEncodeTiled_v12000 adj_encode_fn() {
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

__global__ void round_copy_kernel(const float* W, long long count, uint16_t* out, int fmt) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    out[e] = op_round(W[e], fmt);
}

struct AdjState {
  uint16_t* W[kMaxLayers] = {};   // W_k rounded to the operand format, row-major [widths[k+1], widths[k]]
  CUtensorMap fwd[kMaxLayers];
  CUtensorMap bwd[kMaxLayers];
};

bool encode(CUtensorMap* map, const void* ptr, int rows, int cols, int fmt) {
  auto enc = adj_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
             const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

leb_status adj_tc_prepare(Ctx& c) {
  MlpModel& m = c.mlp;
  if (!m.tc || m.L < 2) return LEB_ERR_UNSUPPORTED;
  for (int i = 0; i < m.L; ++i)
    if (m.widths[i] > 512 || m.widths[i] % 32 != 0) return LEB_ERR_UNSUPPORTED;
  const int fmt = m.prec == LEB_PREC_BF16 ? 1 : 0;
  AdjState* st = new AdjState();
  m.adj = st;
  for (int k = 0; k + 1 < m.L; ++k) {
    const int rows = m.widths[k + 1], cols = m.widths[k];
    if (cudaMalloc(&st->W[k], (size_t)rows * cols * 2) != cudaSuccess) return LEB_ERR_CUDA;
    round_copy_kernel<<<256, 256>>>(m.W[k], (long long)rows * cols, st->W[k], fmt);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    if (!encode(&st->bwd[k], st->W[k], rows, cols, fmt)) return LEB_ERR_UNSUPPORTED;
    if (!encode(&st->fwd[k], tc_weight_t(c, k), cols, rows, fmt)) return LEB_ERR_UNSUPPORTED;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return LEB_ERR_CUDA;
  if (cudaFuncSetAttribute(adjoint_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem) != cudaSuccess)
    return LEB_ERR_CUDA;
  // the register split needs the launch budget it draws on: never launch a kernel compiled below it
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, adjoint_tc_kernel) != cudaSuccess) return LEB_ERR_CUDA;
  if (fa.numRegs < kAdjRegsLaunchMin) return LEB_ERR_UNSUPPORTED;
  return LEB_OK;
}

void adj_tc_release(Ctx& c) {
  AdjState* st = reinterpret_cast<AdjState*>(c.mlp.adj);
  if (!st) return;
  for (int k = 0; k < kMaxLayers; ++k) cudaFree(st->W[k]);
  delete st;
  c.mlp.adj = nullptr;
}

size_t adj_tc_scratch_floats(const Ctx& c) {
  const MlpModel& m = c.mlp;
  size_t stot = 0;
  for (int k = 0; k + 2 < m.L; ++k) stot += m.widths[k + 1];   // lambda_0 .. lambda_{L-3}
  return (size_t)c.sm_count * stot * 64;   // FP16: two per float
}

leb_status adj_tc_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, const float* g_lo,
                        const float* g_hi, int* flags, cudaStream_t s) {
  const MlpModel& m = c.mlp;
  AdjState* st = reinterpret_cast<AdjState*>(m.adj);
  if (!st) return LEB_ERR_UNSUPPORTED;
  AdjTcArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k + 1 < m.L; ++k) {
    a.fwd[k] = st->fwd[k];
    a.bwd[k] = st->bwd[k];
  }
  a.L = m.L;
  for (int i = 0; i <= m.L; ++i) a.widths[i] = m.widths[i];
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
  int o = 0;
  for (int k = 0; k + 2 <= target; ++k) {
    a.soff[k] = o;
    o += m.widths[k + 1];
  }
  a.stot = o > 0 ? o : 1;
  a.W_target = m.W[target];
  a.sL = ws + L.sL;
  a.sU = ws + L.sU;
  a.tL = ws + L.tL;
  a.tU = ws + L.tU;
  a.D = ws + L.D;
  a.dlo = ws + L.dlo;
  a.dhi = ws + L.dhi;
  a.g_lo = g_lo;
  a.g_hi = g_hi;
  a.gl = ws + L.gl;
  a.gu = ws + L.gu;
  a.gsL = ws + L.gsL;
  a.gsU = ws + L.gsU;
  a.gtL = ws + L.gtL;
  a.gtU = ws + L.gtU;
  a.gD = ws + L.gD;
  a.gdlo = ws + L.gdlo;
  a.gdhi = ws + L.gdhi;
  a.scratch = reinterpret_cast<__half*>(ws + L.adj);
  a.flags = flags;
  const int items = T * a.tiles_per_t;
  const int grid = items < c.sm_count ? items : c.sm_count;
  if (grid == 0) return LEB_OK;
  timer_begin(c, s, "adjoint_tc_kernel");
  adjoint_tc_kernel<<<grid, kAdjThreads, kAdjSmem, s>>>(a);
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

}  // namespace leb
